// Stream-K work scheduler: maps (CTA, step) to (problem, tile, k-range, role).
//
// Compiled for host (plan queries, tests) and device (every GEMM kernel), so
// the host enumeration is exactly what the kernels execute.
//
// Decomposition (the method the paper studies, Introduction/Background/
// Methodology, after Osama et al. PPoPP 2023; the paper's "Block2CTile"
// mapping in its Results section is this function's counterpart):
//  * tiles of all problems are concatenated; tile t has I_p k-blocks;
//  * the first `sk_tiles` tiles are Stream-K: their iterations, end to end,
//    are split into `sk_units` contiguous ranges, the first r of length q+1
//    and the rest of length q;
//  * the remaining tiles are data-parallel: tile sk_tiles + j goes to CTA
//    j mod g and is processed after that CTA's Stream-K range;
//  * a range boundary inside a tile splits it: the CTA holding k-block 0 is
//    the owner and sums the partials of CTAs owner+1 .. peer_last in that
//    order; the other CTAs are peers and write one partial each (a CTA can
//    only be a peer in its first segment, so one workspace slot per CTA).
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define SK_HD __host__ __device__ __forceinline__
#else
#define SK_HD inline
#endif

namespace sk {

enum : int32_t { ROLE_WHOLE = 0, ROLE_OWNER = 1, ROLE_PEER = 2, ROLE_DP = 3 };

// Default tile-row group of the rasterisation: group_m consecutive tile rows
// are walked column by column so that CTAs running at the same time share A
// and B panels in L2.
constexpr int32_t GROUP_M_DEFAULT = 8;

struct ProbSched {
  int32_t tiles_m, tiles_n;   // tile grid of the problem
  int32_t iters;              // k-blocks per tile, >= 1
  int32_t pad_;
  int64_t tile_base;          // first global tile index of the problem
  int64_t iter_base;          // first global iteration index of the problem
};

struct Sched {
  int32_t num_problems;
  int32_t g;                  // persistent CTAs (units)
  int32_t sk_units;           // CTAs with a Stream-K range (<= g)
  int32_t r;                  // sk_iters mod sk_units
  int32_t group_m;            // rasterisation group (tile rows), >= 1
  int32_t pad_;
  int64_t q;                  // sk_iters / sk_units
  int64_t total_tiles;
  int64_t sk_tiles;
  int64_t sk_iters;
};

struct Item {
  int32_t problem;
  int32_t tile;               // local tile index (before rasterisation)
  int32_t tm, tn;             // tile coordinates
  int32_t k0, k1;
  int32_t role;
  int32_t peer_first, peer_last;
  int32_t pad_;
  int64_t gtile;
};

struct Cursor {
  int64_t it, end;            // Stream-K progress [it, end)
  int64_t dp;                 // next data-parallel global tile
};

SK_HD int64_t sk_min64(int64_t a, int64_t b) { return a < b ? a : b; }

// Largest p with ps[p].iter_base <= it (problems all have >= 1 tile).
SK_HD int32_t problem_of_iter(const ProbSched *ps, int32_t n, int64_t it) {
  int32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (ps[mid].iter_base <= it) lo = mid; else hi = mid - 1;
  }
  return lo;
}

SK_HD int32_t problem_of_tile(const ProbSched *ps, int32_t n, int64_t t) {
  int32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (ps[mid].tile_base <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Which Stream-K unit holds global iteration `it` (< sk_iters).
SK_HD int32_t unit_of_iter(const Sched &s, int64_t it) {
  int64_t big = (int64_t)s.r * (s.q + 1);
  if (it < big) return (int32_t)(it / (s.q + 1));
  return (int32_t)(s.r + (it - big) / s.q);
}

SK_HD void raster(int32_t lt, int32_t tiles_m, int32_t tiles_n, int32_t group_m, int32_t &tm, int32_t &tn) {
  int32_t per_group = group_m * tiles_n;
  int32_t group = lt / per_group;
  int32_t first_m = group * group_m;
  int32_t gm = tiles_m - first_m;
  if (gm > group_m) gm = group_m;
  int32_t in_group = lt - group * per_group;
  tm = first_m + in_group % gm;
  tn = in_group / gm;
}

SK_HD void cursor_init(const Sched &s, int32_t u, Cursor &c) {
  if (u < s.sk_units) {
    int64_t extra = u < s.r ? u : s.r;
    c.it = (int64_t)u * s.q + extra;
    c.end = c.it + s.q + (u < s.r ? 1 : 0);
  } else {
    c.it = 0;
    c.end = 0;
  }
  c.dp = s.sk_tiles + u;
}

SK_HD bool cursor_next(const Sched &s, const ProbSched *ps, int32_t u, Cursor &c, Item &w) {
  int32_t p, lt;
  if (c.it < c.end) {
    p = problem_of_iter(ps, s.num_problems, c.it);
    const int32_t I = ps[p].iters;
    int64_t local = c.it - ps[p].iter_base;
    lt = (int32_t)(local / I);
    int32_t k0 = (int32_t)(local - (int64_t)lt * I);
    int64_t tile_start = c.it - k0;
    int64_t seg_end = sk_min64(c.end, tile_start + I);
    int32_t k1 = k0 + (int32_t)(seg_end - c.it);
    w.k0 = k0;
    w.k1 = k1;
    w.peer_first = -1;
    w.peer_last = -1;
    if (k0 == 0 && k1 == I) {
      w.role = ROLE_WHOLE;
    } else if (k0 == 0) {
      w.role = ROLE_OWNER;
      w.peer_first = u + 1;
      w.peer_last = unit_of_iter(s, tile_start + I - 1);
    } else {
      w.role = ROLE_PEER;
    }
    w.gtile = ps[p].tile_base + lt;
    c.it = seg_end;
  } else if (c.dp < s.total_tiles) {
    p = problem_of_tile(ps, s.num_problems, c.dp);
    lt = (int32_t)(c.dp - ps[p].tile_base);
    w.k0 = 0;
    w.k1 = ps[p].iters;
    w.role = ROLE_DP;
    w.peer_first = -1;
    w.peer_last = -1;
    w.gtile = c.dp;
    c.dp += s.g;
  } else {
    return false;
  }
  w.problem = p;
  w.tile = lt;
  raster(lt, ps[p].tiles_m, ps[p].tiles_n, s.group_m, w.tm, w.tn);
  w.pad_ = 0;
  return true;
}

}  // namespace sk

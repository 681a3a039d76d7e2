// C-ABI layer of the Stream-K GEMM: argument checks, layout normalisation,
// the Stream-K / hybrid plan, workspace carving, TMA descriptor encoding and
// kernel launch.  See include/skgemm.h for the contract of every entry point.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/skgemm.h"
#include "common.cuh"

using namespace sk;

namespace sk {
cudaError_t launch_transpose16(const void *src, int64_t rows, int64_t cols, int64_t ld_src, void *dst, int64_t ld_dst,
                               int sms, cudaStream_t st);
}

namespace {

// Last failure seen by this thread (sk_last_error).
thread_local std::string t_last_error;

sk_status fail_cuda(const char *what, cudaError_t e) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  t_last_error = buf;
  return SK_ERR_CUDA;
}

sk_status fail_msg(sk_status s, const char *what) {
  t_last_error = what;
  return s;
}

// ------------------------------------------------------------------ device
struct DevInfo {
  bool ready = false;
  int sms = 0;
  int major = 0, minor = 0;
};
std::mutex g_mu;
DevInfo g_dev[64];

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;

sk_status current_device(int *dev, DevInfo *out) {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) return SK_ERR_NO_DEVICE;
  if (d < 0 || d >= 64) return SK_ERR_NO_DEVICE;
  std::lock_guard<std::mutex> lk(g_mu);
  DevInfo &di = g_dev[d];
  if (!di.ready) {
    if (cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, d) != cudaSuccess) return SK_ERR_NO_DEVICE;
    cudaDeviceGetAttribute(&di.major, cudaDevAttrComputeCapabilityMajor, d);
    cudaDeviceGetAttribute(&di.minor, cudaDevAttrComputeCapabilityMinor, d);
    di.ready = true;
  }
  *dev = d;
  *out = di;
  return SK_OK;
}

sk_status encoder(EncodeTiledFn *fn) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_encode) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return fail_msg(SK_ERR_CUDA, "cudaGetDriverEntryPointByVersion(cuTensorMapEncodeTiled) failed");
    g_encode = reinterpret_cast<EncodeTiledFn>(p);
  }
  *fn = g_encode;
  return SK_OK;
}

// --------------------------------------------------------- problem checks
int dtype_bytes(sk_dtype t) {
  switch (t) {
    case SK_F32: return 4;
    case SK_BF16: return 2;
    case SK_E4M3: return 1;
  }
  return 0;
}

bool valid_layout(sk_layout l) { return l == SK_ROW_MAJOR || l == SK_COL_MAJOR; }
bool valid_dtype(sk_dtype t) { return t == SK_F32 || t == SK_BF16 || t == SK_E4M3; }
sk_layout flip(sk_layout l) { return l == SK_ROW_MAJOR ? SK_COL_MAJOR : SK_ROW_MAJOR; }

// Minimum leading dimension of an r x c matrix stored with layout l.
int64_t min_ld(sk_layout l, int64_t r, int64_t c) {
  int64_t e = l == SK_ROW_MAJOR ? c : r;
  return e < 1 ? 1 : e;
}

// Kernel family of a type combination.
enum Family { FAM_F32 = 0, FAM_BF16 = 1, FAM_E4M3 = 2, FAM_NONE = -1 };

Family family_of(const sk_problem &p) {
  if (p.a_type != p.b_type) return FAM_NONE;
  if (p.a_type == SK_F32) return p.c_type == SK_F32 ? FAM_F32 : FAM_NONE;
  if (p.a_type == SK_BF16) return (p.c_type == SK_BF16 || p.c_type == SK_F32) ? FAM_BF16 : FAM_NONE;
  if (p.a_type == SK_E4M3) return (p.c_type == SK_BF16 || p.c_type == SK_F32) ? FAM_E4M3 : FAM_NONE;
  return FAM_NONE;
}

sk_status check_problem(const sk_problem *p) {
  if (!p) return SK_ERR_INVALID_ARG;
  if (p->m < 0 || p->n < 0 || p->k < 0) return SK_ERR_INVALID_ARG;
  if (p->m > INT32_MAX / 2 || p->n > INT32_MAX / 2 || p->k > INT32_MAX / 2) return SK_ERR_UNSUPPORTED;
  if (!valid_dtype(p->a_type) || !valid_dtype(p->b_type) || !valid_dtype(p->c_type)) return SK_ERR_INVALID_ARG;
  if (!valid_layout(p->a_layout) || !valid_layout(p->b_layout) || !valid_layout(p->c_layout))
    return SK_ERR_INVALID_ARG;
  if (family_of(*p) == FAM_NONE) return SK_ERR_UNSUPPORTED;
  if (p->m == 0 || p->n == 0) return SK_OK;
  if (!p->C) return SK_ERR_INVALID_ARG;
  if (p->ldc < min_ld(p->c_layout, p->m, p->n)) return SK_ERR_INVALID_ARG;
  if (p->beta != 0.f && !p->C_in) return SK_ERR_INVALID_ARG;
  if (p->k == 0) return SK_OK;
  if (!p->A || !p->B) return SK_ERR_INVALID_ARG;
  if (p->lda < min_ld(p->a_layout, p->m, p->k)) return SK_ERR_INVALID_ARG;
  if (p->ldb < min_ld(p->b_layout, p->k, p->n)) return SK_ERR_INVALID_ARG;
  return SK_OK;
}

// A problem rewritten so that C is row-major: C col-major (m x n) is the
// row-major C^T (n x m) = B^T A^T, with each transpose a layout flip.
struct Norm {
  int64_t M, N, K;
  const void *A, *B;
  const void *C_in;
  void *C;
  sk_layout a_layout, b_layout;   // of the (possibly swapped) operands
  int64_t lda, ldb, ldc;
  float alpha, beta;
  const float *sa, *sb;
  sk_dtype in_type, c_type;
};

Norm normalise(const sk_problem &p) {
  Norm n;
  n.alpha = p.alpha;
  n.beta = p.beta;
  n.sa = p.scale_a;
  n.sb = p.scale_b;
  n.in_type = p.a_type;
  n.c_type = p.c_type;
  n.C = p.C;
  n.C_in = p.C_in;
  n.ldc = p.ldc;
  n.K = p.k;
  if (p.c_layout == SK_ROW_MAJOR) {
    n.M = p.m;
    n.N = p.n;
    n.A = p.A;
    n.a_layout = p.a_layout;
    n.lda = p.lda;
    n.B = p.B;
    n.b_layout = p.b_layout;
    n.ldb = p.ldb;
  } else {
    n.M = p.n;
    n.N = p.m;
    n.A = p.B;
    n.a_layout = flip(p.b_layout);
    n.lda = p.ldb;
    n.B = p.A;
    n.b_layout = flip(p.a_layout);
    n.ldb = p.lda;
    std::swap(n.sa, n.sb);
  }
  return n;
}

// ------------------------------------------------------------------ config
struct Cfg {
  Family fam;
  int BM, BN, BK, stages;
  bool pair;       // CTA-pair kernel: a unit is a cluster of 2 CTAs, tile 256 x BN
  sk_mode mode;
  int g;           // scheduler units (CTAs, or CTA pairs)
  int min_ipu;
  uint64_t timeout_ns;
  int debug_flags;
  uint64_t *trace;
  uint32_t *cover;
  int raster_group;
  int fixup;       // FIXUP_OWNER, FIXUP_LAST_ARRIVER, FIXUP_SPLIT or FIXUP_SPLIT_CLUSTER
  bool tc32 = false;   // FP32 on the tensor cores (3xTF32) instead of FFMA
  int ctas() const { return pair ? 2 * g : g; }
};

sk_status resolve_cfg(Family fam, const sk_config *c, int sms, Cfg *out) {
  sk_config d;
  std::memset(&d, 0, sizeof(d));
  if (c) d = *c;
  Cfg r;
  r.fam = fam;
  if (d.tile_m != 128 && d.tile_m != 256) return SK_ERR_UNSUPPORTED;   // 0 was resolved by auto_tile
  r.pair = d.tile_m == 256;
  r.BM = d.tile_m;
  if (d.f32_kernel < SK_F32_AUTO || d.f32_kernel > SK_F32_TF32X3) return SK_ERR_INVALID_ARG;
  if (fam == FAM_F32 && d.f32_kernel == SK_F32_TF32X3) {
    // 3xTF32 on the tensor cores: 128 x 128 tiles on one CTA or 256 x 256
    // tiles on a CTA pair (each CTA holds 128 rows of A and 128 of B),
    // 32-deep k-blocks, each stage twice the loaded bytes (high and low parts)
    const int bn = r.pair ? 256 : 128;
    if (d.tile_n != 0 && d.tile_n != bn) return SK_ERR_UNSUPPORTED;
    r.tc32 = true;
    r.BN = bn;
    r.BK = 32;
    const int max_stages = (227 * 1024 - 1024 - 512 - EPI_STAGE_BYTES) / (2 * (128 * 128 + 128 * 128));
    r.stages = d.stages ? d.stages : max_stages;
    if (r.stages < 2 || r.stages > max_stages) return SK_ERR_UNSUPPORTED;
  } else if (fam == FAM_F32) {
    if (r.pair) return SK_ERR_UNSUPPORTED;
    if (d.tile_n != 0 && d.tile_n != 128) return SK_ERR_UNSUPPORTED;
    r.BN = 128;
    r.BK = F32_BK;
    if (d.stages != 0 && d.stages != 2) return SK_ERR_UNSUPPORTED;
    r.stages = 2;
  } else {
    r.BN = d.tile_n ? d.tile_n : 256;
    if (r.BN != 128 && r.BN != 256 && !(r.BN == 512 && r.pair)) return SK_ERR_UNSUPPORTED;   // 256 x 512: pairs
    if (r.pair && r.BN == 128 && fam != FAM_BF16) return SK_ERR_UNSUPPORTED;   // 256 x 128 pairs: BF16
    r.BK = fam == FAM_BF16 ? 64 : 128;
    const int stage_bytes = 128 * 128 + (r.pair ? r.BN / 2 : r.BN) * 128;   // per CTA
    const int max_stages = std::min(8, (227 * 1024 - 1024 - 512 - EPI_STAGE_BYTES) / stage_bytes);
    r.stages = d.stages ? d.stages : max_stages;
    if (r.stages < 2 || r.stages > max_stages) return SK_ERR_UNSUPPORTED;
  }
  if (d.mode < SK_MODE_AUTO || d.mode > SK_MODE_HYBRID2) return SK_ERR_INVALID_ARG;
  r.mode = d.mode == SK_MODE_AUTO ? SK_MODE_HYBRID2 : d.mode;
  if (sms <= 0) return SK_ERR_INVALID_ARG;
  if (d.num_ctas < 0 || d.num_ctas > sms) return SK_ERR_INVALID_ARG;
  if (sms > WS_MAX_CTAS) return SK_ERR_UNSUPPORTED;   // the workspace's flag region
  const int ctas = d.num_ctas ? d.num_ctas : sms;
  r.g = r.pair ? ctas / 2 : ctas;
  if (r.g < 1) return SK_ERR_INVALID_ARG;
  if (d.min_iters_per_unit < 0) return SK_ERR_INVALID_ARG;
  r.min_ipu = d.min_iters_per_unit ? d.min_iters_per_unit : 4;
  r.timeout_ns = d.timeout_ns ? d.timeout_ns : 2000000000ull;
  r.debug_flags = d.debug_flags;
  r.trace = d.trace;
  r.cover = d.coverage;
  if (d.raster_group < 0 || d.raster_group > 64) return SK_ERR_INVALID_ARG;
  r.raster_group = d.raster_group ? d.raster_group : GROUP_M_DEFAULT;
  if (d.fixup != SK_FIXUP_OWNER && d.fixup != SK_FIXUP_LAST_ARRIVER && d.fixup != SK_FIXUP_SPLIT &&
      d.fixup != SK_FIXUP_SPLIT_CLUSTER)
    return SK_ERR_INVALID_ARG;
  // the cluster split: BF16 or 3xTF32 on 128-row tiles or 256 x 256 pairs
  if (d.fixup == SK_FIXUP_SPLIT_CLUSTER &&
      (!(fam == FAM_BF16 || (fam == FAM_F32 && r.tc32)) || (r.pair && r.BN != 256)))
    return SK_ERR_UNSUPPORTED;
  r.fixup = d.fixup == SK_FIXUP_LAST_ARRIVER ? FIXUP_LAST_ARRIVER
            : d.fixup == SK_FIXUP_SPLIT      ? FIXUP_SPLIT
            : d.fixup == SK_FIXUP_SPLIT_CLUSTER ? FIXUP_SPLIT_CLUSTER
                                             : FIXUP_OWNER;
  *out = r;
  return SK_OK;
}

// Workspace bytes (layout in common.cuh): the status word, the fixed flag
// region, and per CTA one partial slot (128 rows x BN FP32); the
// last-arriver fixup adds a second slot per CTA.
size_t ws_base_bytes(const Cfg &c) {
  // (the cluster split exchanges partials between shared memories: no slots)
  const size_t slots = c.fixup == FIXUP_SPLIT_CLUSTER ? 0 : (size_t)c.ctas() * 128 * c.BN * 4;
  return WS_FLAG_OFFSET + WS_FLAG_BYTES + (c.fixup == FIXUP_LAST_ARRIVER ? 2 : 1) * slots;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Groups of more than MAXP_GROUPED problems keep their problem table in the
// workspace, after the partial slots: the kernel's per-problem records
// (tensor maps included), then the per-problem schedule records.
size_t table_bytes(const Cfg &c, size_t nprob) {
  if (nprob <= (size_t)MAXP_GROUPED) return 0;
  const size_t rec = (c.fam == FAM_F32 && !c.tc32) ? sizeof(SimtProblem) : sizeof(TcProblem);
  return round256(nprob * rec) + round256(nprob * sizeof(ProbSched));
}

size_t ws_bytes_for(const Cfg &c, size_t nprob = 0) { return ws_base_bytes(c) + table_bytes(c, nprob); }

Workspace carve(void *ws, const Cfg &c) {
  uint8_t *b = static_cast<uint8_t *>(ws);
  Workspace w;
  w.status = reinterpret_cast<uint32_t *>(b);
  w.flags = reinterpret_cast<uint32_t *>(b + WS_FLAG_OFFSET);
  w.partials = reinterpret_cast<float *>(b + WS_FLAG_OFFSET + WS_FLAG_BYTES);
  w.owner_partials = c.fixup == FIXUP_LAST_ARRIVER ? w.partials + (size_t)c.ctas() * 128 * c.BN : nullptr;
  return w;
}


// -------------------------------------------------------------------- plan
struct PlanOut {
  Sched s;
  std::vector<ProbSched> ps;
  std::vector<int> orig_index;   // problem index in the caller's array
  int grid;
  double predicted_ns = 0;
};

// MAC-loop iterations (k-blocks of every tile) of all problems of a plan.
int64_t total_iters(const PlanOut &pl) {
  if (pl.ps.empty()) return 0;
  const ProbSched &q = pl.ps.back();
  return q.iter_base + (int64_t)q.tiles_m * q.tiles_n * q.iters;
}

int64_t count_sk_tiles(int64_t T, int64_t g, sk_mode mode) {
  switch (mode) {
    case SK_MODE_DP: return 0;
    case SK_MODE_SK: return T;
    case SK_MODE_HYBRID1: return T % g;
    case SK_MODE_HYBRID2:
      if (T <= g) return T;
      if (T % g == 0) return 0;
      return g + T % g;
    default: return T;
  }
}

// Builds the plan over the problems with m, n, k >= 1 (in their order).
void build_plan(const std::vector<Norm> &probs, const std::vector<int> &idx, const Cfg &c, PlanOut *out) {
  out->ps.clear();
  out->orig_index.clear();
  int64_t tiles = 0, iters = 0;
  for (size_t i = 0; i < probs.size(); ++i) {
    const Norm &n = probs[i];
    ProbSched p;
    p.tiles_m = (int32_t)((n.M + c.BM - 1) / c.BM);
    p.tiles_n = (int32_t)((n.N + c.BN - 1) / c.BN);
    p.iters = (int32_t)((n.K + c.BK - 1) / c.BK);
    p.pad_ = 0;
    p.tile_base = tiles;
    p.iter_base = iters;
    const int64_t t = (int64_t)p.tiles_m * p.tiles_n;
    tiles += t;
    iters += t * p.iters;
    out->ps.push_back(p);
    out->orig_index.push_back(idx[i]);
  }
  Sched &s = out->s;
  s.num_problems = (int32_t)out->ps.size();
  s.g = c.g;
  s.group_m = c.raster_group;
  s.pad_ = 0;
  s.total_tiles = tiles;
  s.sk_tiles = count_sk_tiles(tiles, c.g, c.mode);
  // iterations of the leading sk_tiles tiles
  int64_t ski = 0;
  for (const ProbSched &p : out->ps) {
    const int64_t t = (int64_t)p.tiles_m * p.tiles_n;
    const int64_t lo = p.tile_base, hi = p.tile_base + t;
    const int64_t take = std::max<int64_t>(0, std::min(hi, s.sk_tiles) - lo);
    ski += take * p.iters;
  }
  s.sk_iters = ski;
  if (ski > 0) {
    int64_t units = ski / std::max(1, c.min_ipu);
    units = std::max<int64_t>(1, std::min<int64_t>(c.g, units));
    s.sk_units = (int32_t)units;
    s.q = ski / units;
    s.r = (int32_t)(ski % units);
  } else {
    s.sk_units = 0;
    s.q = 0;
    s.r = 0;
  }
  const int64_t dp = tiles - s.sk_tiles;
  const int64_t units = std::max<int64_t>(s.sk_units, std::min<int64_t>(c.g, dp));
  out->grid = (int)(c.pair ? 2 * units : units);
}

// ----------------------------------------------------------- runtime model
// Analytic makespan of a plan, used to choose the tile and the DP/SK split
// when the caller leaves them to the library (the paper's Results and
// Future Work name such a predictive load-balancing model, "Block2Time").
//
// Each unit is simulated as the kernel runs it: an MMA chain (k-blocks x
// t_iter + t_mac_item per item) feeding an epilogue chain through two TMEM
// accumulators, so item i's MMAs wait for the epilogue of item i-2 (i-1
// for 256 x 512 pairs, whose one accumulator fills TMEM).  The
// epilogue of an item costs
//   whole / DP tile : t_store
//   peer            : t_spill                      (and records when the
//                                                   partial is visible)
//   owner           : t_fix_base + peers x t_fix_peer + t_store, after every
//                     peer's partial is visible; t_fix_peer is the staged
//                     (last item) or the plain (more work follows) rate.
// The FP32 SIMT kernel has no separate epilogue warps: its chains are one.
// When the plan's DRAM bytes at HBM bandwidth exceed the longest MMA chain
// (see plan_dram_bytes: Stream-K ranges lose the L2 sharing of DP waves),
// every MMA chain is stretched by that ratio; the fixup tail still follows.
// The kernel's time is the latest unit end plus a launch cost.
// Coefficients: least-squares fit (log time) to every default-stage
// candidate of 26 BF16 shapes timed on GB300, the tile-aligned unit counts
// included (the choice among the measured candidates then costs 0.4 % on
// average, 3.4 % at worst, against the measured best).
// 256 x 128 pair tiles (explicit requests only): each CTA needs 24 KB of
// operands per 256-cycle k-block, beyond what L2 delivers to one SM, so a
// k-block costs about what a 256 x 256 one does (measured 8192^3: 986 us).
#define PAIR128_COEFFS 520.0, 1190.0, 5270.0, 4000.0, 3500.0, 0.0, 2600.0, 3000.0
// 3xTF32 (128 x 128 tiles, 32-deep k-blocks: three TF32 MMAs of half the
// BF16 rate per k-block plus the in-kernel split of the stage; the
// epilogue warps also do the split, so an epilogue does not overlap the
// next item's MMAs).
#define TF32X3_COEFFS 700.0, 900.0, 5160.0, 4500.0, 3020.0, 0.0, 3210.0, 790.0
// 3xTF32 on CTA pairs (256 x 256 tiles): twelve M = 256 TF32 MMAs per
// 32-deep k-block (1536 cycles), the split spread over both CTAs' epilogue
// warps.  The per-k-block costs of both 3xTF32 families are refitted to
// seven FP32 shapes timed on GB300 (384x384x2048 to 8192x4096x4096): the
// model then ranks the two tiles as measured on all seven (pairs win from
// 1024x1024x4096 up, e.g. 4096^3 505 against 643 us).
#define TF32X3_PAIR_COEFFS 1100.0, 1190.0, 8500.0, 5510.0, 5030.0, 0.0, 3450.0, 4030.0
// 256 x 512 pairs: a k-block (two N = 256 MMAs) measured 0.573 us against
// 0.650 us for two 256 x 256 k-blocks (per-CTA timeline, 8192^3 DP, same
// clock); TMEM holds one 512-column accumulator, so a tile's MMAs wait for
// the previous tile's epilogue and for its last MMAs to drain.  A fit of
// launch + items x (k-blocks x t_iter + t_item) to 14 DP shapes (K 1024 to
// 16384, 1 to 27 tiles per pair) gave t_iter 560 ns, t_item 6.8 us and a
// 7.9 us launch (2 % rms); against the 256 x 256 pair's coefficients the
// values below pick the faster of the two tiles on all 21 shapes measured
// both ways (the wide tile on 8192^3, 8192 x 8192 x {12288, 16384},
// 6144 x 6144 x 12288, 16384 x 16384 x 8192 and 3072 x 3072 x 16384, by
// 2-16 %; the pair on K = 4096 shapes, on 13.5 tiles per pair -- 8192 x
// 16384 x 8192 both ways round -- and on short or small shapes).  Partials
// are twice a 256 x 256 pair's.
#define PAIR512_COEFFS 555.0, 1500.0, 7920.0, 5000.0, 10060.0, 0.0, 6900.0, 8060.0

struct ModelCoeffs {
  double iter_ns;            // one k-block of one tile (effective; fitted with t_mac_item)
  double mac_item_ns;        // per work item on the MMA chain (tile switch, pipeline refill)
  double launch_ns;          // launch and prologue
  double store_ns;           // epilogue of a finished tile (TMEM -> C)
  double spill_ns;           // a peer's partial to the workspace
  double fix_base_ns;        // owner fixup, fixed part
  double fix_peer_last_ns;   // per peer partial, staged fixup (the CTA's last item)
  double fix_peer_mid_ns;    // per peer partial, plain fixup (more work follows)
  bool serial;               // epilogue on the same threads as the MMA chain
  bool one_acc = false;      // one TMEM accumulator: an item's MMAs wait for the previous epilogue
};

ModelCoeffs model_coeffs(const Cfg &c) {
  if (c.fam == FAM_F32 && c.tc32) return c.pair ? ModelCoeffs{TF32X3_PAIR_COEFFS, false} : ModelCoeffs{TF32X3_COEFFS, false};
  if (c.fam == FAM_F32) return {1700.0, 500.0, 6000.0, 1000.0, 2000.0, 1000.0, 1000.0, 1000.0, true};
  if (c.pair && c.BN == 128) return {PAIR128_COEFFS, false};
  if (c.pair && c.BN == 512) return {PAIR512_COEFFS, false, true};
  if (c.pair) return {302.0, 1190.0, 5270.0, 5510.0, 5030.0, 0.0, 3450.0, 4030.0, false};
  if (c.BN == 256) return {375.0, 760.0, 6520.0, 3030.0, 3920.0, 1760.0, 3320.0, 3790.0, false};
  return {284.0, 636.0, 5160.0, 3900.0, 3020.0, 0.0, 3210.0, 790.0, false};
}

// The split reduce needs every unit to hold exactly one range inside one
// tile, so that a tile's units finish together: all tiles Stream-K, every
// unit used, equal ranges (no remainder) that divide every tile's k-blocks.
bool split_eligible(const PlanOut &pl) {
  const Sched &s = pl.s;
  if (s.num_problems <= 0 || s.sk_tiles != s.total_tiles || s.sk_units != s.g || s.r != 0 || s.q <= 0) return false;
  for (const ProbSched &p : pl.ps)
    if (p.iters % s.q != 0) return false;
  return true;
}

// The cluster split additionally needs one problem (the single-problem
// kernels), every tile split into exactly two ranges (2 units per tile),
// and a tile shape with a cluster-split kernel.
// Units per tile of a cluster-split plan (2, 4 or 8; a cluster holds at
// most 8 CTAs), or 0 if the plan cannot run as one: one problem, every
// tile split into equal tile-aligned ranges (split_eligible), a tile shape
// with a cluster-split kernel, and an operand ring that holds this CTA's
// incoming blocks ((k - 1) partials of its units) and its outgoing ones.
int xs_units_per_tile(const PlanOut &pl, const Cfg &c, const std::vector<Norm> &work) {
  if (pl.s.num_problems != 1 || pl.s.total_tiles <= 0 || !split_eligible(pl)) return 0;
  if (!(c.fam == FAM_BF16 || (c.fam == FAM_F32 && c.tc32)) || (c.pair && c.BN != 256)) return 0;
  if (pl.s.g % pl.s.total_tiles != 0) return 0;
  const int k = (int)(pl.s.g / pl.s.total_tiles);
  if (k != 2 && k != 4 && k != 8) return 0;
  if ((c.pair ? 2 : 1) * k > 8) return 0;
  const int uw = work[0].c_type == SK_F32 ? 1 : 2;   // 32-column chunks per unit
  const int ns = 4 * (c.BN / 32) / uw;
  const int blk = uw * 4096;
  const int own_max = (ns + k - 1) / k, own_min = ns / k;
  if (own_max > XS_MAX_UNITS) return 0;   // one data barrier per own unit
  const int stage = (128 * 128 + (c.pair ? c.BN / 2 : c.BN) * 128) * (c.tc32 ? 2 : 1);
  if ((int64_t)c.stages * stage < (int64_t)((k - 1) * own_max + (ns - own_min)) * blk) return 0;
  return k;
}

double algorithmic_dram_bytes(const std::vector<Norm> &work) {
  double b = 0;
  for (const Norm &n : work) {
    const double es = dtype_bytes(n.in_type), cs = dtype_bytes(n.c_type);
    b += (double)(n.M * n.K + n.K * n.N) * es + (double)n.M * n.N * cs * (n.beta != 0.f ? 2.0 : 1.0);
  }
  return b;
}

constexpr double kHbmBytesPerNs = 6500.0;   // measured copy bandwidth ~6.76 TB/s, rounded down
constexpr double kL2OperandBytes = 100e6;   // L2 the operands can hold (of 126 MB; the rest serves C and partials)

// DRAM bytes the plan's operand loads are expected to cost.
//  * DP tiles run in waves of g consecutive tiles that share A/B panels in
//    L2: each wave reads the distinct row panels and column panels of its
//    tiles once.
//  * Stream-K units run far-apart parts of the tile list at the same time;
//    their k-slices come from DRAM once each if the SK tiles' panels fit
//    in L2 together.  Otherwise an operand keeps what fits of its share of
//    L2 (half, or what the other operand leaves) and the rest of its
//    panels is re-read by every tile that streams it.
// Output (and C_in) bytes are added for every tile.
double plan_dram_bytes(const std::vector<Norm> &work, const PlanOut &pl, const Cfg &c) {
  const Sched &s = pl.s;
  const double es = dtype_bytes(work[0].in_type);
  auto panel_key = [](int32_t p, int32_t idx) { return ((uint64_t)(uint32_t)p << 32) | (uint32_t)idx; };
  auto tile_of = [&](int64_t gt, int32_t &p, int32_t &tm, int32_t &tn) {
    p = problem_of_tile(pl.ps.data(), s.num_problems, gt);
    raster((int32_t)(gt - pl.ps[p].tile_base), pl.ps[p].tiles_m, pl.ps[p].tiles_n, s.group_m, tm, tn);
  };
  double bytes = 0;
  // Stream-K part
  if (s.sk_tiles > 0) {
    std::vector<uint64_t> rows, cols;
    double streamed_a = 0, streamed_b = 0;
    for (int64_t t = 0; t < s.sk_tiles; ++t) {
      int32_t p, tm, tn;
      tile_of(t, p, tm, tn);
      rows.push_back(panel_key(p, tm));
      cols.push_back(panel_key(p, tn));
      streamed_a += (double)pl.ps[p].iters * c.BK * c.BM * es;
      streamed_b += (double)pl.ps[p].iters * c.BK * c.BN * es;
    }
    std::sort(rows.begin(), rows.end());
    rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    double unique_a = 0, unique_b = 0;
    for (uint64_t r : rows) unique_a += (double)c.BM * work[r >> 32].K * es;
    for (uint64_t q : cols) unique_b += (double)c.BN * work[q >> 32].K * es;
    if (unique_a + unique_b <= kL2OperandBytes) {
      bytes += unique_a + unique_b;
    } else {
      double budget_a = kL2OperandBytes / 2, budget_b = kL2OperandBytes / 2;
      if (unique_a < budget_a) budget_b = kL2OperandBytes - unique_a;
      else if (unique_b < budget_b) budget_a = kL2OperandBytes - unique_b;
      auto operand = [](double unique, double streamed, double budget) {
        return unique <= budget ? unique : unique + (streamed - unique) * (1.0 - budget / unique);
      };
      bytes += operand(unique_a, streamed_a, budget_a) + operand(unique_b, streamed_b, budget_b);
    }
  }
  // data-parallel waves
  std::vector<uint64_t> rows, cols;
  const int64_t dp = s.total_tiles - s.sk_tiles;
  for (int64_t w0 = 0; w0 < dp; w0 += s.g) {
    rows.clear();
    cols.clear();
    const int64_t w1 = std::min<int64_t>(dp, w0 + s.g);
    for (int64_t j = w0; j < w1; ++j) {
      int32_t p, tm, tn;
      tile_of(s.sk_tiles + j, p, tm, tn);
      rows.push_back(panel_key(p, tm));
      cols.push_back(panel_key(p, tn));
    }
    std::sort(rows.begin(), rows.end());
    rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    for (uint64_t r : rows) bytes += (double)c.BM * work[r >> 32].K * es;
    for (uint64_t q : cols) bytes += (double)c.BN * work[q >> 32].K * es;
  }
  for (const Norm &n : work)
    bytes += (double)n.M * n.N * dtype_bytes(n.c_type) * (n.beta != 0.f ? 2.0 : 1.0);
  return bytes;
}

// Cluster split: writing half an accumulator into the partner's shared
// memory, as a fraction of a full spill to the workspace (estimate).
constexpr double kXsExchangeFrac = 0.35;

constexpr double kGroupedIterFactor = 1.07;

double predict_ns(const std::vector<Norm> &work, const PlanOut &pl, const Cfg &c) {
  ModelCoeffs k = model_coeffs(c);
  const Sched &s = pl.s;
  if (s.num_problems <= 0) return k.launch_ns;
  // The grouped kernel (problem table, per-item tensor-map selection) runs a
  // k-block about 7 % slower than the single-problem one: the two backward
  // GEMMs of 8192 x 11008 x 4096 took 842 us as one grouped launch and
  // 784 us as two single launches on the same tiles.
  if (work.size() > 1) k.iter_ns *= kGroupedIterFactor;
  std::vector<std::vector<Item>> items((size_t)c.g);
  double longest_mac = 0;
  for (int u = 0; u < c.g; ++u) {
    Cursor cur;
    cursor_init(s, u, cur);
    Item w;
    double mac = 0;
    while (cursor_next(s, pl.ps.data(), u, cur, w)) {
      items[u].push_back(w);
      mac += (w.k1 - w.k0) * k.iter_ns + k.mac_item_ns;
    }
    longest_mac = std::max(longest_mac, mac);
  }
  const double dram_ns = std::max(algorithmic_dram_bytes(work), plan_dram_bytes(work, pl, c)) / kHbmBytesPerNs;
  const double stretch = longest_mac > 0 ? std::max(1.0, dram_ns / longest_mac) : 1.0;
  // Two passes: the first finds when each peer's partial is visible (a
  // peer segment is a unit's first item, so it depends on no owner), the
  // second lets owners wait for them.
  std::vector<double> spill_done((size_t)c.g, 0.0);
  double end = 0;
  for (int pass = 0; pass < 2; ++pass) {
    end = 0;
    for (int u = 0; u < c.g; ++u) {
      const std::vector<Item> &its = items[u];
      double mac_prev = 0, epi_prev = 0, epi_prev2 = 0;
      for (size_t i = 0; i < its.size(); ++i) {
        const Item &w = its[i];
        const bool last = i + 1 == its.size();
        const double mac_start = k.serial ? epi_prev : std::max(mac_prev, k.one_acc ? epi_prev : epi_prev2);
        const double mac_end = mac_start + (w.k1 - w.k0) * k.iter_ns * stretch + k.mac_item_ns;
        double start = std::max(mac_end, epi_prev);
        double e;
        if (c.fixup == FIXUP_SPLIT_CLUSTER && (w.role == ROLE_PEER || w.role == ROLE_OWNER)) {
          // the kc contributors (units o .. o + kc - 1, one cluster) each
          // signal a free ring when their accumulator is complete, write
          // the (kc - 1) / kc of it the others sum into their shared
          // memories, then sum and store their 1 / kc of the tile
          const int kc = (int)(s.g / s.total_tiles);
          const int o = u - u % kc;
          spill_done[u] = start;
          if (pass > 0)
            for (int p = o; p < o + kc; ++p) start = std::max(start, spill_done[p]);
          e = kXsExchangeFrac * k.spill_ns * 2.0 * (kc - 1) / kc + k.store_ns / kc +
              (kc > 2 ? k.fix_peer_last_ns * (kc - 2) / kc : 0.0);
        } else if (c.fixup == FIXUP_SPLIT && (w.role == ROLE_PEER || w.role == ROLE_OWNER)) {
          // all contributors spill, wait for each other, then each reads
          // about one partial's bytes and stores its share of the tile
          int o = u, pl_ = w.peer_last;
          if (w.role == ROLE_PEER) {
            const ProbSched &q = pl.ps[w.problem];
            const int64_t ts = q.iter_base + (int64_t)w.tile * q.iters;
            o = unit_of_iter(s, ts);
            pl_ = unit_of_iter(s, ts + q.iters - 1);
          }
          // (tensor-core kernel: the tile's columns x row quarters are cut
          // into NS units dealt out in order, a unit's partials summed by
          // one warp; each contributor spills all but its own units, which
          // stay in TMEM, and its busiest warp reads the other kc - 1
          // partials of its units.  FP32 FFMA kernel: each spills
          // everything and reads kc partials of its share.)
          const int kc = pl_ - o + 1;
          const int jx = u - o;
          double own_cta, own_warp;
          if (k.serial) {
            own_cta = own_warp = (double)((jx + 1) * 4096 / kc - jx * 4096 / kc) / 4096;
          } else {
            const int ns = 4 * (c.BN / 32) / (work[w.problem].c_type == SK_F32 ? 1 : 2);
            const int n_u = (jx + 1) * ns / kc - jx * ns / kc;
            own_cta = (double)n_u / ns;
            own_warp = (double)((n_u + 3) / 4) / (ns / 4);
          }
          spill_done[u] = start + k.spill_ns * (k.serial ? 1.0 : 1.0 - own_cta);
          double ready = spill_done[u];
          if (pass > 0)
            for (int p = o; p <= pl_; ++p) ready = std::max(ready, spill_done[p]);
          start = ready;
          e = own_cta > 0
                  ? k.fix_base_ns + k.fix_peer_last_ns * (k.serial ? kc : kc - 1) * own_warp + k.store_ns * own_warp
                  : 0.0;
        } else if (w.role == ROLE_PEER) {
          e = k.spill_ns;
          spill_done[u] = start + e;
        } else if (w.role == ROLE_OWNER) {
          if (pass > 0)
            for (int p = w.peer_first; p <= w.peer_last; ++p) start = std::max(start, spill_done[p]);
          e = k.fix_base_ns + (w.peer_last - w.peer_first + 1) * (last ? k.fix_peer_last_ns : k.fix_peer_mid_ns) +
              k.store_ns;
        } else {
          e = k.store_ns;
        }
        mac_prev = mac_end;
        epi_prev2 = epi_prev;
        epi_prev = start + e;
      }
      end = std::max(end, epi_prev);
    }
  }
  return k.launch_ns + end;
}

// --------------------------------------------------------------- launches
sk_status cuda_err(cudaError_t e, const char *what = "CUDA call") {
  return e == cudaSuccess ? SK_OK : fail_cuda(what, e);
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

sk_status check_tc_alignment(const Norm &n) {
  const int es = dtype_bytes(n.in_type);
  if (!aligned16(n.A) || !aligned16(n.B)) return SK_ERR_UNSUPPORTED;
  if ((n.lda * es) % 16 != 0 || (n.ldb * es) % 16 != 0) return SK_ERR_UNSUPPORTED;
  if ((n.in_type == SK_E4M3 || n.in_type == SK_F32) && (n.a_layout != SK_ROW_MAJOR || n.b_layout != SK_COL_MAJOR))
    return SK_ERR_UNSUPPORTED;
  return SK_OK;
}

// The pair kernel reads MN-major (transposed) BF16 operands too; E4M3 is
// K-major only (checked by check_tc_alignment).
sk_status check_pair_layout(const Norm &n) {
  (void)n;
  return SK_OK;
}

sk_status encode_operand(EncodeTiledFn enc, CUtensorMap *m, const void *base, sk_dtype t, bool kmajor, int64_t rows,
                         int64_t K, int64_t ld, int box_rows, int BK) {
  const int es = dtype_bytes(t);
  const CUtensorMapDataType dt = t == SK_BF16  ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                 : t == SK_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                               : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  cuuint64_t dims[2], strides[1];
  cuuint32_t box[2], estr[2] = {1, 1};
  if (kmajor) {   // element (r, k) at base[r*ld + k]
    dims[0] = (cuuint64_t)K;
    dims[1] = (cuuint64_t)rows;
    box[0] = (cuuint32_t)BK;
    box[1] = (cuuint32_t)box_rows;
  } else {        // element (r, k) at base[r + k*ld]
    dims[0] = (cuuint64_t)rows;
    dims[1] = (cuuint64_t)K;
    box[0] = 64;
    box[1] = (cuuint32_t)BK;
  }
  strides[0] = (cuuint64_t)ld * es;
  CUresult r = enc(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[128];
    std::snprintf(buf, sizeof(buf), "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return fail_msg(SK_ERR_CUDA, buf);
  }
  return SK_OK;
}

static_assert(sizeof(TcParams<MAXP_GROUPED>) <= 32000, "kernel parameter block too large");
// table records are uploaded in whole 16-byte words
static_assert(sizeof(TcProblem) % 16 == 0 && sizeof(SimtProblem) % 16 == 0 && sizeof(ProbSched) % 16 == 0,
              "problem records must be multiples of 16 bytes");

template <int MAXP>
sk_status launch_tc_family(const std::vector<Norm> &probs, const PlanOut &pl, const Cfg &c, Workspace ws,
                           void *table, cudaStream_t st) {
  EncodeTiledFn enc;
  sk_status rc = encoder(&enc);
  if (rc != SK_OK) return rc;
  // Heap-allocated: the grouped parameter block is ~22 KB.
  TcParams<MAXP> *P = new TcParams<MAXP>();
  std::memset(P, 0, sizeof(*P));
  const size_t np = probs.size();
  // More problems than the parameter block holds: build the records on the
  // host and upload them to the workspace's table region.
  const bool gtab = np > (size_t)MAXP;
  std::vector<TcProblem> big(gtab ? np : 0);
  std::vector<ProbSched> big_ps(gtab ? np : 0);
  if (gtab) std::memset(static_cast<void *>(big.data()), 0, np * sizeof(TcProblem));
  for (size_t i = 0; i < np; ++i) {
    const Norm &n = probs[i];
    TcProblem &tp = gtab ? big[i] : P->prob[i];
    const bool a_k = n.a_layout == SK_ROW_MAJOR;   // A(i,k) at A[i*lda + k]
    const bool b_k = n.b_layout == SK_COL_MAJOR;   // B(k,j) at B[k + j*ldb]
    rc = encode_operand(enc, &tp.tmap_a, n.A, n.in_type, a_k, n.M, n.K, n.lda, 128, c.BK);
    if (rc == SK_OK)
      // (B rows per load: a pair CTA's half of one MMA's columns, at most 128)
    rc = encode_operand(enc, &tp.tmap_b, n.B, n.in_type, b_k, n.N, n.K, n.ldb, c.pair ? std::min(c.BN / 2, 128) : c.BN,
                        c.BK);
    if (rc != SK_OK) {
      delete P;
      return rc;
    }
    tp.C = n.C;
    tp.C_in = n.C_in;
    tp.ldc = n.ldc;
    {
      // TMA stores of C: beta == 0, 16-byte aligned base and row pitch.
      const int ces = n.c_type == SK_F32 ? 4 : 2;
      tp.c_tma = MAXP == 1 && n.beta == 0.f && aligned16(n.C) && (n.ldc * ces) % 16 == 0;
      if (tp.c_tma) {
        cuuint64_t dims[2] = {(cuuint64_t)n.N, (cuuint64_t)n.M};
        cuuint64_t strides[1] = {(cuuint64_t)n.ldc * ces};
        cuuint32_t box[2] = {(cuuint32_t)(128 / ces), 32};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = enc(&P->tmap_c[0], n.c_type == SK_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                         2, n.C, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) tp.c_tma = 0;   // fall back to plain stores
      }
    }
    tp.M = (int32_t)n.M;
    tp.N = (int32_t)n.N;
    tp.K = (int32_t)n.K;
    tp.alpha = n.alpha;
    tp.beta = n.beta;
    tp.a_mn = a_k ? 0 : 1;
    tp.b_mn = b_k ? 0 : 1;
    const int ces = n.c_type == SK_F32 ? 4 : 2;
    tp.c_vec = aligned16(n.C) && (n.beta == 0.f || aligned16(n.C_in)) && ((n.ldc * ces) % 16 == 0);
    tp.scale_a = n.sa;
    tp.scale_b = n.sb;
    if (gtab)
      big_ps[i] = pl.ps[i];
    else
      P->ps[i] = pl.ps[i];
  }
  if (gtab) {
    uint8_t *tb = static_cast<uint8_t *>(table);
    const size_t rec_bytes = round256(np * sizeof(TcProblem));
    cudaError_t ue = launch_upload(tb, big.data(), np * sizeof(TcProblem), st);
    if (ue == cudaSuccess) ue = launch_upload(tb + rec_bytes, big_ps.data(), np * sizeof(ProbSched), st);
    if (ue != cudaSuccess) {
      delete P;
      return cuda_err(ue, "problem table upload");
    }
    P->gprob = reinterpret_cast<const TcProblem *>(tb);
    P->gps = reinterpret_cast<const ProbSched *>(tb + rec_bytes);
  }
  P->sched = pl.s;
  P->ws = ws;
  P->timeout_ns = c.timeout_ns;
  P->stages = c.stages;
  P->debug_flags = c.debug_flags;
  P->trace = c.trace;
  P->cover = c.cover;
  P->cover_iters = total_iters(pl);
  P->fixup = c.fixup;
  P->xs_k = c.fixup == FIXUP_SPLIT_CLUSTER ? (int32_t)(pl.s.g / std::max<int64_t>(1, pl.s.total_tiles)) : 0;
  const bool f32out = probs[0].c_type == SK_F32;
  cudaError_t e = cudaErrorInvalidValue;
  if (c.fam == FAM_BF16) {
    if (c.pair && c.BN == 512) {
      if constexpr (MAXP == 1)
        e = f32out ? launch_tc<IN_BF16, float, 512, 1, true>(*P, pl.grid, st)
                   : launch_tc<IN_BF16, __nv_bfloat16, 512, 1, true>(*P, pl.grid, st);
      else
        e = cudaErrorNotSupported;
    } else if (c.pair && c.BN == 256)
      e = f32out ? launch_tc<IN_BF16, float, 256, MAXP, true>(*P, pl.grid, st)
                 : launch_tc<IN_BF16, __nv_bfloat16, 256, MAXP, true>(*P, pl.grid, st);
    else if (c.pair)
      e = f32out ? launch_tc<IN_BF16, float, 128, MAXP, true>(*P, pl.grid, st)
                 : launch_tc<IN_BF16, __nv_bfloat16, 128, MAXP, true>(*P, pl.grid, st);
    else if (c.BN == 256)
      e = f32out ? launch_tc<IN_BF16, float, 256, MAXP, false>(*P, pl.grid, st)
                 : launch_tc<IN_BF16, __nv_bfloat16, 256, MAXP, false>(*P, pl.grid, st);
    else
      e = f32out ? launch_tc<IN_BF16, float, 128, MAXP, false>(*P, pl.grid, st)
                 : launch_tc<IN_BF16, __nv_bfloat16, 128, MAXP, false>(*P, pl.grid, st);
  } else if (c.fam == FAM_F32) {
    e = c.pair ? launch_tc<IN_TF32X3, float, 256, MAXP, true>(*P, pl.grid, st)
               : launch_tc<IN_TF32X3, float, 128, MAXP, false>(*P, pl.grid, st);
  } else if (c.fam == FAM_E4M3) {
    if constexpr (MAXP == 1) {
      if (c.pair && c.BN == 512)
        e = f32out ? launch_tc<IN_E4M3, float, 512, 1, true>(*P, pl.grid, st)
                   : launch_tc<IN_E4M3, __nv_bfloat16, 512, 1, true>(*P, pl.grid, st);
      else if (c.pair)
        e = f32out ? launch_tc<IN_E4M3, float, 256, 1, true>(*P, pl.grid, st)
                   : launch_tc<IN_E4M3, __nv_bfloat16, 256, 1, true>(*P, pl.grid, st);
      else if (c.BN == 256)
        e = f32out ? launch_tc<IN_E4M3, float, 256, 1, false>(*P, pl.grid, st)
                   : launch_tc<IN_E4M3, __nv_bfloat16, 256, 1, false>(*P, pl.grid, st);
      else
        e = f32out ? launch_tc<IN_E4M3, float, 128, 1, false>(*P, pl.grid, st)
                   : launch_tc<IN_E4M3, __nv_bfloat16, 128, 1, false>(*P, pl.grid, st);
    } else {
      delete P;
      return SK_ERR_UNSUPPORTED;
    }
  }
  delete P;
  return cuda_err(e, "tcgen05 GEMM launch");
}

template <int MAXP>
sk_status launch_f32_family(const std::vector<Norm> &probs, const PlanOut &pl, const Cfg &c, Workspace ws,
                            void *table, cudaStream_t st) {
  SimtParams<MAXP> *P = new SimtParams<MAXP>();
  std::memset(P, 0, sizeof(*P));
  const size_t np = probs.size();
  const bool gtab = np > (size_t)MAXP;
  std::vector<SimtProblem> big(gtab ? np : 0);
  std::vector<ProbSched> big_ps(gtab ? np : 0);
  for (size_t i = 0; i < np; ++i) {
    const Norm &n = probs[i];
    SimtProblem &sp = gtab ? big[i] : P->prob[i];
    sp.A = static_cast<const float *>(n.A);
    sp.B = static_cast<const float *>(n.B);
    sp.C_in = static_cast<const float *>(n.C_in);
    sp.C = static_cast<float *>(n.C);
    if (n.a_layout == SK_ROW_MAJOR) {
      sp.a_rs = n.lda;
      sp.a_cs = 1;
    } else {
      sp.a_rs = 1;
      sp.a_cs = n.lda;
    }
    if (n.b_layout == SK_ROW_MAJOR) {
      sp.b_rs = n.ldb;
      sp.b_cs = 1;
    } else {
      sp.b_rs = 1;
      sp.b_cs = n.ldb;
    }
    sp.ldc = n.ldc;
    sp.M = (int32_t)n.M;
    sp.N = (int32_t)n.N;
    sp.K = (int32_t)n.K;
    sp.alpha = n.alpha;
    sp.beta = n.beta;
    sp.a_kmajor = n.a_layout == SK_ROW_MAJOR;
    sp.b_kmajor = n.b_layout == SK_COL_MAJOR;
    sp.a_vec = aligned16(n.A) && (n.lda % 4 == 0);
    sp.b_vec = aligned16(n.B) && (n.ldb % 4 == 0);
    sp.c_vec = aligned16(n.C) && (n.beta == 0.f || aligned16(n.C_in)) && (n.ldc % 4 == 0);
    if (gtab)
      big_ps[i] = pl.ps[i];
    else
      P->ps[i] = pl.ps[i];
  }
  if (gtab) {
    uint8_t *tb = static_cast<uint8_t *>(table);
    const size_t rec_bytes = round256(np * sizeof(SimtProblem));
    cudaError_t ue = launch_upload(tb, big.data(), np * sizeof(SimtProblem), st);
    if (ue == cudaSuccess) ue = launch_upload(tb + rec_bytes, big_ps.data(), np * sizeof(ProbSched), st);
    if (ue != cudaSuccess) {
      delete P;
      return cuda_err(ue, "problem table upload");
    }
    P->gprob = reinterpret_cast<const SimtProblem *>(tb);
    P->gps = reinterpret_cast<const ProbSched *>(tb + rec_bytes);
  }
  P->sched = pl.s;
  P->ws = ws;
  P->timeout_ns = c.timeout_ns;
  P->debug_flags = c.debug_flags;
  P->fixup = c.fixup;
  cudaError_t e = launch_simt_f32<MAXP>(*P, pl.grid, st);
  delete P;
  return cuda_err(e, "FP32 GEMM launch");
}

// Fills the fields the caller left to the library (tile_m = 0, tile_n = 0,
// mode = AUTO) with the candidate the runtime model predicts fastest.
// Decisions are cached per problem set and config.
//
// Co-resident clusters of the cluster-split kernel with k units per
// cluster for config c on device `dev`, cached; with no device (dev < 0:
// plan queries given an SM count) every SM is assumed usable.
int xs_capacity(int dev, const Cfg &c, bool f32out, int sms, int k) {
  const int per = (c.pair ? 2 : 1) * k;
  if (dev < 0 || dev >= 64) return sms / per;
  static std::mutex mu;
  static int cache[64][2][2][2][2][4][16] = {};
  std::lock_guard<std::mutex> lk(mu);
  const int ki = k == 2 ? 0 : k == 4 ? 1 : k == 8 ? 2 : 3;
  int &slot = cache[dev][c.tc32 ? 1 : 0][c.pair ? 1 : 0][c.BN == 256 ? 1 : 0][f32out ? 1 : 0][ki][c.stages & 15];
  if (slot == 0) {
    int n;
    if (c.tc32)
      n = c.pair ? xs_max_clusters<IN_TF32X3, float, 256, true>(c.stages, k)
                 : xs_max_clusters<IN_TF32X3, float, 128, false>(c.stages, k);
    else if (c.pair)
      n = f32out ? xs_max_clusters<IN_BF16, float, 256, true>(c.stages, k)
                 : xs_max_clusters<IN_BF16, __nv_bfloat16, 256, true>(c.stages, k);
    else if (c.BN == 256)
      n = f32out ? xs_max_clusters<IN_BF16, float, 256, false>(c.stages, k)
                 : xs_max_clusters<IN_BF16, __nv_bfloat16, 256, false>(c.stages, k);
    else
      n = f32out ? xs_max_clusters<IN_BF16, float, 128, false>(c.stages, k)
                 : xs_max_clusters<IN_BF16, __nv_bfloat16, 128, false>(c.stages, k);
    slot = n > 0 ? n : -1;
  }
  return slot > 0 ? slot : 0;
}

// Whether plan `pl` of config `c` can run as a cluster split here: a
// single-problem launch, eligible (xs_units_per_tile), and, where the
// library chooses it (one_wave), one co-resident cluster per tile so the
// plan runs in one wave.  (Clusters never wait on one another, so an
// explicit request runs correctly in several waves too.)
bool xs_runnable(const PlanOut &pl, const Cfg &c, const std::vector<Norm> &work, bool single, int dev, int sms,
                 bool one_wave) {
  const int k = xs_units_per_tile(pl, c, work);
  return single && k > 0 &&
         (!one_wave || xs_capacity(dev, c, work[0].c_type == SK_F32, sms, k) >= pl.s.total_tiles);
}

sk_status choose_auto(Family fam, const std::vector<Norm> &work, const std::vector<int> &idx, int sms, int dev,
                      bool single, sk_config *d) {
  const bool free_tile_m = d->tile_m == 0;
  const bool free_tile_n = d->tile_n == 0 && fam != FAM_F32;
  const bool free_mode = d->mode == SK_MODE_AUTO;
  if (!free_tile_m && !free_tile_n && !free_mode) return SK_OK;
  if (work.empty()) {
    if (free_tile_m) d->tile_m = 128;
    if (free_mode) d->mode = SK_MODE_HYBRID2;
    return SK_OK;
  }
  // cache key
  std::string key;
  {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|", (int)fam, sms, d->tile_m, d->tile_n,
                  d->stages, (int)d->mode, d->num_ctas, d->min_iters_per_unit, d->raster_group, (int)d->fixup,
                  (int)d->f32_kernel, d->debug_flags & DEBUG_SKIP_PEER_FLAG, dev, single ? 1 : 0);
    key = buf;
    for (const Norm &n : work) {
      std::snprintf(buf, sizeof(buf), "%lld,%lld,%lld,%d,%d,%d,%d;", (long long)n.M, (long long)n.N,
                    (long long)n.K, (int)n.a_layout, (int)n.b_layout, (int)n.c_type, n.beta != 0.f);
      key += buf;
    }
  }
  // The cache holds only the chosen fields; everything else (timeouts,
  // test flags, ...) stays the caller's.
  struct Choice {
    int tile_m, tile_n;
    sk_mode mode;
    int num_ctas;
    sk_fixup fixup;
  };
  static std::mutex mu;
  static std::map<std::string, Choice> cache;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      d->tile_m = it->second.tile_m;
      d->tile_n = it->second.tile_n;
      d->mode = it->second.mode;
      d->num_ctas = it->second.num_ctas;
      d->fixup = it->second.fixup;
      return SK_OK;
    }
  }
  const bool pair_ok = (fam != FAM_F32 || d->f32_kernel == SK_F32_TF32X3) && (d->num_ctas > 0 ? d->num_ctas : sms) >= 2;
  std::vector<int> tms, tns;
  std::vector<sk_mode> modes;
  if (free_tile_m) {
    tms.push_back(128);
    if (pair_ok && (d->tile_n == 0 || d->tile_n == 256)) tms.push_back(256);
  } else {
    tms.push_back(d->tile_m);
  }
  if (free_mode) modes = {SK_MODE_HYBRID2, SK_MODE_DP, SK_MODE_SK, SK_MODE_HYBRID1};
  else modes = {d->mode};
  double best = 1e300;
  sk_config best_cfg = *d;
  bool found = false;
  sk_status last_rc = SK_ERR_UNSUPPORTED;
  for (int tm : tms) {
    tns.clear();
    if (fam == FAM_F32) tns.push_back(d->tile_n);
    else if (!free_tile_n) tns.push_back(d->tile_n);
    else if (tm == 256) {
      tns.push_back(256);   // 256 x 128 pairs: only when asked for (never faster)
      if (single && fam != FAM_F32) tns.push_back(512);
    }
    else tns = {256, 128};
    for (int tn : tns) {
      for (sk_mode md : modes) {
        // (the library picks 256 x 512 pairs for data-parallel plans only:
        // their Stream-K partials are twice a 256 x 256 pair's and measured
        // slower on every shape tried)
        if (tn == 512 && free_tile_n && md != SK_MODE_DP) continue;
        sk_config t = *d;
        t.tile_m = tm;
        t.tile_n = tn;
        t.mode = md;
        Cfg c;
        const sk_status rc = resolve_cfg(fam, &t, sms, &c);
        if (rc != SK_OK) {
          last_rc = rc;   // an invalid request stays invalid for every candidate
          continue;
        }
        PlanOut pl;
        build_plan(work, idx, c, &pl);
        if (c.fixup == FIXUP_SPLIT && !split_eligible(pl)) {
          // an explicit split reduce needs a plan it can run
          last_rc = fail_msg(SK_ERR_UNSUPPORTED, "split reduce: every unit must hold one tile-aligned range");
          continue;
        }
        if (c.fixup == FIXUP_SPLIT_CLUSTER && !xs_runnable(pl, c, work, single, dev, sms, false)) {
          last_rc = fail_msg(SK_ERR_UNSUPPORTED,
                             "cluster split: one BF16 or 3xTF32 problem, 2, 4 or 8 tile-aligned units per tile (at most 8 CTAs)");
          continue;
        }
        double ns = predict_ns(work, pl, c);
        if (ns < best * 0.999) {   // keep the earlier candidate on near-ties
          best = ns;
          best_cfg = t;
          found = true;
        }
        // With fewer tiles than units and every tile split (Stream-K), a
        // unit count that is a multiple of the tile count cuts every tile
        // into equal parts whose units finish together: each owner waits
        // for and adds the fewest partials.  Tried when the caller left the
        // count to the library.
        const int64_t T = pl.s.total_tiles;
        if (d->num_ctas == 0 && pl.s.sk_tiles == T && T > 0 && 2 * T <= c.g) {
          const int g_alt = (int)(c.g / T * T);   // k = g_alt / T >= 2 units per tile
          // Tries `units` units (a multiple of T) with the owner fixup unless
          // it is the plan already evaluated, and, if the caller left the
          // fixup at its default, with every contributor summing a share
          // (the split reduce) where each unit then holds one range.
          auto try_units = [&](int units, bool owner_too) {
            sk_config t2 = t;
            t2.num_ctas = c.pair ? 2 * units : units;
            Cfg c2;
            PlanOut pl2;
            if (units == c.g) {
              c2 = c;
              pl2 = pl;
            } else {
              if (resolve_cfg(fam, &t2, sms, &c2) != SK_OK) return;
              build_plan(work, idx, c2, &pl2);
              if (owner_too) {
                const double ns2 = predict_ns(work, pl2, c2);
                if (ns2 < best * 0.999) {
                  best = ns2;
                  best_cfg = t2;
                }
              }
            }
            if (d->fixup != SK_FIXUP_OWNER || (d->debug_flags & DEBUG_SKIP_PEER_FLAG) || !split_eligible(pl2)) return;
            // the split reduce through the workspace, and, with two units
            // per tile, through the clusters' shared memories
            for (sk_fixup fx : {SK_FIXUP_SPLIT, SK_FIXUP_SPLIT_CLUSTER}) {
              sk_config t3 = t2;
              t3.fixup = fx;
              Cfg c3;
              if (resolve_cfg(fam, &t3, sms, &c3) != SK_OK) continue;
              // (the library picks the cluster split with two units per tile
              // only: with 4 or 8 it measured no faster than the split reduce
              // through the workspace)
              if (fx == SK_FIXUP_SPLIT_CLUSTER &&
                  (pl2.s.g != 2 * pl2.s.total_tiles || !xs_runnable(pl2, c3, work, single, dev, sms, true)))
                continue;
              const double ns3 = predict_ns(work, pl2, c3);
              if (ns3 < best * 0.999) {
                best = ns3;
                best_cfg = t3;
              }
            }
          };
          try_units(g_alt, true);
          // The split reduce needs the per-unit range q = (all k-blocks) /
          // units to divide every tile's k-blocks: if g_alt misses that,
          // the largest smaller multiple of T that meets it.
          if (d->fixup == SK_FIXUP_OWNER && !(d->debug_flags & DEBUG_SKIP_PEER_FLAG)) {
            int64_t total = 0;
            for (const ProbSched &q : pl.ps) total += (int64_t)q.tiles_m * q.tiles_n * q.iters;
            auto eligible = [&](int64_t units) {
              if (total % units != 0) return false;
              const int64_t qq = total / units;
              for (const ProbSched &q : pl.ps)
                if (q.iters % qq != 0) return false;
              return true;
            };
            if (!eligible(g_alt))
              for (int kk = (int)(g_alt / T) - 1; kk >= 2; --kk)
                if (eligible(kk * T)) {
                  try_units((int)(kk * T), false);
                  break;
                }
            // the cluster split with two units per tile
            if (2 * T <= c.g && 2 * T != g_alt) try_units((int)(2 * T), true);
          }
        }
      }
    }
  }
  if (!found) return last_rc;
  d->tile_m = best_cfg.tile_m;
  d->tile_n = best_cfg.tile_n;
  d->mode = best_cfg.mode;
  d->num_ctas = best_cfg.num_ctas;
  d->fixup = best_cfg.fixup;
  std::lock_guard<std::mutex> lk(mu);
  if (cache.size() > 4096) cache.clear();
  cache[key] = Choice{best_cfg.tile_m, best_cfg.tile_n, best_cfg.mode, best_cfg.num_ctas, best_cfg.fixup};
  return SK_OK;
}

// Normalises the problems, picks the tile (tile_m = 0: auto) and resolves
// the config.  `work` gets the problems with m, n, k >= 1; `scale_only` the
// ones with k == 0 (C = beta * C_in).
sk_status prepare(const sk_problem *problems, int count, const sk_config *cfg, int sms, int maxp, int dev,
                  bool single, Cfg *c, std::vector<Norm> *work, std::vector<int> *idx,
                  std::vector<Norm> *scale_only) {
  if (!problems || count < 1 || count > maxp) return SK_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    sk_status rc = check_problem(&problems[i]);
    if (rc != SK_OK) return rc;
  }
  const Family fam = family_of(problems[0]);
  for (int i = 1; i < count; ++i)
    if (problems[i].a_type != problems[0].a_type || problems[i].c_type != problems[0].c_type)
      return SK_ERR_UNSUPPORTED;
  for (int i = 0; i < count; ++i) {
    const sk_problem &p = problems[i];
    if (p.m == 0 || p.n == 0) continue;
    Norm n = normalise(p);
    if (p.k == 0) {
      if (scale_only) scale_only->push_back(n);
      continue;
    }
    work->push_back(n);
    idx->push_back(i);
  }
  sk_config d;
  std::memset(&d, 0, sizeof(d));
  if (cfg) d = *cfg;
  if (fam == FAM_F32 && d.f32_kernel == SK_F32_AUTO) {
    // 3xTF32 where every problem's operands suit TMA and the K-major
    // descriptors; FFMA otherwise
    bool tc_ok = true;
    for (const Norm &n : *work) tc_ok = tc_ok && check_tc_alignment(n) == SK_OK;
    d.f32_kernel = tc_ok ? SK_F32_TF32X3 : SK_F32_FFMA;
  }
  sk_status rc = choose_auto(fam, *work, *idx, sms, dev, single, &d);
  if (rc != SK_OK) return rc;
  rc = resolve_cfg(fam, &d, sms, c);
  if (rc != SK_OK) return rc;
  if (c->BN == 512 && !single) return fail_msg(SK_ERR_UNSUPPORTED, "256 x 512 tiles: single-problem calls only");
  for (const Norm &n : *work) {
    if (fam != FAM_F32 || c->tc32) {
      rc = check_tc_alignment(n);
      if (rc != SK_OK) return rc;
    }
    if (c->pair) {
      rc = check_pair_layout(n);
      if (rc != SK_OK) return rc;
    }
  }
  return SK_OK;
}

// Co-resident CTA pairs of the pair kernel that this call would launch
// (cached per device and variant).
int pair_clusters(int dev, const Cfg &c, bool f32out, bool grouped) {
  static std::mutex mu;
  static int cache[64][3][3][2][2][16] = {};
  const int fi = c.fam == FAM_E4M3 ? 1 : c.fam == FAM_F32 ? 2 : 0;
  const int bi = c.BN == 128 ? 1 : c.BN == 512 ? 2 : 0;
  const int st = c.stages & 15;
  std::lock_guard<std::mutex> lk(mu);
  int &slot = cache[dev][fi][bi][f32out][grouped][st];
  if (slot == 0) {
    int n = 0;
    if (c.BN == 512) {   // single-problem BF16 / E4M3 pairs
      if (!grouped && c.fam == FAM_BF16)
        n = f32out ? pair_max_clusters<IN_BF16, float, 512, 1>(c.stages)
                   : pair_max_clusters<IN_BF16, __nv_bfloat16, 512, 1>(c.stages);
      else if (!grouped && c.fam == FAM_E4M3)
        n = f32out ? pair_max_clusters<IN_E4M3, float, 512, 1>(c.stages)
                   : pair_max_clusters<IN_E4M3, __nv_bfloat16, 512, 1>(c.stages);
    } else if (c.fam == FAM_BF16 && c.BN == 128) {
      if (grouped)
        n = f32out ? pair_max_clusters<IN_BF16, float, 128, MAXP_GROUPED>(c.stages)
                   : pair_max_clusters<IN_BF16, __nv_bfloat16, 128, MAXP_GROUPED>(c.stages);
      else
        n = f32out ? pair_max_clusters<IN_BF16, float, 128, 1>(c.stages)
                   : pair_max_clusters<IN_BF16, __nv_bfloat16, 128, 1>(c.stages);
    } else if (c.fam == FAM_BF16) {
      if (grouped)
        n = f32out ? pair_max_clusters<IN_BF16, float, 256, MAXP_GROUPED>(c.stages)
                   : pair_max_clusters<IN_BF16, __nv_bfloat16, 256, MAXP_GROUPED>(c.stages);
      else
        n = f32out ? pair_max_clusters<IN_BF16, float, 256, 1>(c.stages)
                   : pair_max_clusters<IN_BF16, __nv_bfloat16, 256, 1>(c.stages);
    } else if (c.fam == FAM_F32) {
      n = grouped ? pair_max_clusters<IN_TF32X3, float, 256, MAXP_GROUPED>(c.stages)
                  : pair_max_clusters<IN_TF32X3, float, 256, 1>(c.stages);
    } else {
      n = f32out ? pair_max_clusters<IN_E4M3, float, 256, 1>(c.stages)
                 : pair_max_clusters<IN_E4M3, __nv_bfloat16, 256, 1>(c.stages);
    }
    slot = n > 0 ? n : -1;
  }
  return slot;
}

// Shared driver of sk_gemm / sk_gemm_grouped / sk_gemm_backward.
sk_status run(const sk_problem *problems, int count, const sk_config *cfg, void *ws, size_t ws_bytes,
              cudaStream_t st, int maxp) {
  t_last_error.clear();
  if (!problems || count < 1 || count > maxp) return SK_ERR_INVALID_ARG;
  int dev;
  DevInfo di;
  sk_status rc = current_device(&dev, &di);
  if (rc != SK_OK) return rc;
  if (!(di.major == 10 && di.minor == 3)) return SK_ERR_NO_DEVICE;   // built for sm_103a only
  // Make the device's primary context current on this thread: the
  // tensor-map encoder is a driver call and fails with "invalid context" on
  // threads (e.g. the autograd engine's) that have not touched the driver.
  {
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) return fail_cuda("cudaSetDevice", e);
  }
  // Validate everything before launching anything.
  Cfg c;
  std::vector<Norm> work, scale_only;
  std::vector<int> idx;
  rc = prepare(problems, count, cfg, di.sms, maxp, dev, count == 1 && maxp == 1, &c, &work, &idx, &scale_only);
  if (rc != SK_OK) return rc;
  const bool grouped = !(work.size() == 1 && maxp == 1);
  if (c.pair && !work.empty()) {
    // All units must be co-resident (owners wait on peers): never more
    // pairs than the GPU can hold at once.
    const int maxc = pair_clusters(dev, c, work[0].c_type == SK_F32, grouped);
    if (maxc <= 0) return fail_msg(SK_ERR_UNSUPPORTED, "the CTA-pair kernel cannot be made resident");
    c.g = std::min(c.g, maxc);
  }
  if (!work.empty()) {
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return SK_ERR_INVALID_ARG;
    if (ws_bytes < ws_bytes_for(c, work.size())) return SK_ERR_WORKSPACE_TOO_SMALL;
  }
  for (const Norm &n : scale_only) {
    rc = cuda_err(launch_scale(n.C, n.C_in, n.ldc, n.M, n.N, n.beta, n.c_type == SK_F32, st), "k=0 scale launch");
    if (rc != SK_OK) return rc;
  }
  if (work.empty()) return SK_OK;
  PlanOut pl;
  build_plan(work, idx, c, &pl);
  if (c.fixup == FIXUP_SPLIT && !split_eligible(pl))
    return fail_msg(SK_ERR_UNSUPPORTED, "split reduce: every unit must hold one tile-aligned range");
  if (c.fixup == FIXUP_SPLIT_CLUSTER && !xs_runnable(pl, c, work, !grouped, dev, di.sms, false))
    return fail_msg(SK_ERR_UNSUPPORTED,
                    "cluster split: one BF16 or 3xTF32 problem, 2, 4 or 8 tile-aligned units per tile (at most 8 CTAs)");
  Workspace w = carve(ws, c);
  void *table = static_cast<uint8_t *>(ws) + ws_base_bytes(c);   // used for groups beyond MAXP_GROUPED
  if (c.fam == FAM_F32 && !c.tc32) {
    return grouped ? launch_f32_family<MAXP_GROUPED>(work, pl, c, w, table, st)
                   : launch_f32_family<1>(work, pl, c, w, table, st);
  }
  return grouped ? launch_tc_family<MAXP_GROUPED>(work, pl, c, w, table, st)
                 : launch_tc_family<1>(work, pl, c, w, table, st);
}

// Plan for queries: honours num_sms > 0 without touching a device (the
// pair kernel is then assumed to fit num_sms / 2 pairs).
sk_status plan_for_query(const sk_problem *problems, int count, const sk_config *cfg, int num_sms, Cfg *c,
                         PlanOut *pl) {
  int sms = num_sms;
  int dev = -1;
  if (sms <= 0) {
    DevInfo di;
    sk_status rc = current_device(&dev, &di);
    if (rc != SK_OK) return rc;
    sms = di.sms;
  }
  std::vector<Norm> work;
  std::vector<int> idx;
  sk_status rc = prepare(problems, count, cfg, sms, MAX_PROBLEMS, dev, count == 1, c, &work, &idx, nullptr);
  if (rc != SK_OK) return rc;
  if (c->pair && dev >= 0 && !work.empty()) {
    const int maxc = pair_clusters(dev, *c, work[0].c_type == SK_F32, count > 1);
    if (maxc > 0) c->g = std::min(c->g, maxc);
  }
  build_plan(work, idx, *c, pl);
  if (c->fixup == FIXUP_SPLIT && !work.empty() && !split_eligible(*pl)) return SK_ERR_UNSUPPORTED;
  if (c->fixup == FIXUP_SPLIT_CLUSTER && !work.empty() && !xs_runnable(*pl, *c, work, count == 1, dev, sms, false))
    return SK_ERR_UNSUPPORTED;
  pl->predicted_ns = work.empty() ? 0.0 : predict_ns(work, *pl, *c);
  return SK_OK;
}

}  // namespace

extern "C" {

const char *sk_version(void) { return "skgemm 0.1 (sm_103a)"; }

const char *sk_last_error(void) { return t_last_error.c_str(); }

const char *sk_status_string(sk_status s) {
  switch (s) {
    case SK_OK: return "SK_OK";
    case SK_ERR_INVALID_ARG: return "SK_ERR_INVALID_ARG";
    case SK_ERR_UNSUPPORTED: return "SK_ERR_UNSUPPORTED";
    case SK_ERR_WORKSPACE_TOO_SMALL: return "SK_ERR_WORKSPACE_TOO_SMALL";
    case SK_ERR_TIMEOUT: return "SK_ERR_TIMEOUT";
    case SK_ERR_CUDA: return "SK_ERR_CUDA";
    case SK_ERR_NO_DEVICE: return "SK_ERR_NO_DEVICE";
  }
  return "SK_ERR_UNKNOWN";
}

sk_status sk_workspace_size(const sk_problem *problems, int count, const sk_config *cfg, size_t *bytes) {
  if (!bytes) return SK_ERR_INVALID_ARG;
  Cfg c;
  PlanOut pl;
  sk_status rc = plan_for_query(problems, count, cfg, cfg && cfg->num_ctas > 0 ? cfg->num_ctas : 0, &c, &pl);
  if (rc != SK_OK) return rc;
  *bytes = ws_bytes_for(c, (size_t)pl.s.num_problems);
  return SK_OK;
}

sk_status sk_workspace_init(void *ws, size_t ws_bytes, sk_stream_t stream) {
  if (!ws || ws_bytes < 256) return SK_ERR_INVALID_ARG;
  return cuda_err(cudaMemsetAsync(ws, 0, ws_bytes, reinterpret_cast<cudaStream_t>(stream)), "cudaMemsetAsync");
}

sk_status sk_gemm(const sk_problem *problem, const sk_config *cfg, void *ws, size_t ws_bytes, sk_stream_t stream) {
  return run(problem, 1, cfg, ws, ws_bytes, reinterpret_cast<cudaStream_t>(stream), 1);
}

sk_status sk_gemm_grouped(const sk_problem *problems, int count, const sk_config *cfg, void *ws, size_t ws_bytes,
                          sk_stream_t stream) {
  return run(problems, count, cfg, ws, ws_bytes, reinterpret_cast<cudaStream_t>(stream), MAX_PROBLEMS);
}

}  // extern "C"

namespace {

// The two GEMMs of the backward of C = A B: dA = dC B^T (m x k) and
// dB = A^T dC (k x n), each operand read in the storage order it has (a
// forward K-major operand is MN-major here and vice versa).
int backward_problems(const sk_problem *fwd, const void *dC, int64_t lddc, void *dA, int64_t ldda, void *dB,
                      int64_t lddb, sk_problem pr[2]) {
  int n = 0;
  if (dA) {   // dA (m x k) = dC (m x n) * B^T (n x k)
    sk_problem p;
    std::memset(&p, 0, sizeof(p));
    p.m = fwd->m;
    p.n = fwd->k;
    p.k = fwd->n;
    p.a_type = p.b_type = SK_BF16;
    p.c_type = fwd->a_type;
    p.A = dC;
    p.a_layout = SK_ROW_MAJOR;
    p.lda = lddc;
    p.B = fwd->B;
    p.b_layout = flip(fwd->b_layout);
    p.ldb = fwd->ldb;
    p.C = dA;
    p.c_layout = fwd->a_layout;
    p.ldc = ldda;
    p.alpha = 1.f;
    p.beta = 0.f;
    pr[n++] = p;
  }
  if (dB) {   // dB (k x n) = A^T (k x m) * dC (m x n)
    sk_problem p;
    std::memset(&p, 0, sizeof(p));
    p.m = fwd->k;
    p.n = fwd->n;
    p.k = fwd->m;
    p.a_type = p.b_type = SK_BF16;
    p.c_type = fwd->b_type;
    p.A = fwd->A;
    p.a_layout = flip(fwd->a_layout);
    p.lda = fwd->lda;
    p.B = dC;
    p.b_layout = SK_ROW_MAJOR;
    p.ldb = lddc;
    p.C = dB;
    p.c_layout = fwd->b_layout;
    p.ldc = lddb;
    p.alpha = 1.f;
    p.beta = 0.f;
    pr[n++] = p;
  }
  return n;
}

int64_t round8(int64_t v) { return (v + 7) & ~(int64_t)7; }

// K-major copies the backward GEMMs can read instead of MN-major operands
// (MN-major operands measured ~1.4x slower per GEMM: with them the kernel
// moves more bytes through each SM's shared memory).  For each MN-major
// operand: its rows x cols storage, and the copy's leading dimension.
struct FlipCopy {
  int prob, operand;          // problem index, 0 = A, 1 = B
  const void *src;
  int64_t rows, cols, ld_src;   // storage of the MN-major operand (row-major rows x cols)
  int64_t ld_dst;               // the copy: cols x rows row-major
  size_t offset;                // in the workspace, after the GEMM's own bytes
};

// Workspace bytes of the backward's GEMMs: the largest of the grouped plan
// and, with two problems, each single-problem plan (the call runs one or
// the other; the operand copies go after all of them).
sk_status backward_gemm_ws(const sk_problem *pr, int n, const sk_config *cfg, size_t *bytes) {
  size_t b = 0;
  sk_status rc = sk_workspace_size(pr, n, cfg, &b);
  if (n == 1) {
    *bytes = b;
    return rc;
  }
  // two problems: the grouped plan may be refused (a configuration only
  // single launches take); the single plans must both resolve
  if (rc != SK_OK) b = 0;
  for (int i = 0; i < n; ++i) {
    size_t bi = 0;
    const sk_status ri = sk_workspace_size(&pr[i], 1, cfg, &bi);
    if (ri != SK_OK) return ri;
    b = std::max(b, bi);
  }
  *bytes = b;
  return SK_OK;
}

// Plans the copies for problems pr[0..n) after `base` bytes of workspace;
// returns the total workspace bytes the K-major path needs.
size_t plan_flips(const sk_problem *pr, int n, size_t base, std::vector<FlipCopy> *out) {
  size_t off = round256(base);
  for (int i = 0; i < n; ++i) {
    const sk_problem &p = pr[i];
    if (p.a_layout == SK_COL_MAJOR) {   // A(i,k) at A[i + k*lda]: storage k rows x m cols
      FlipCopy f{i, 0, p.A, p.k, p.m, p.lda, round8(p.k), off};
      off = round256(off + (size_t)f.cols * f.ld_dst * 2);
      out->push_back(f);
    }
    if (p.b_layout == SK_ROW_MAJOR) {   // B(k,j) at B[k*ldb + j]: storage k rows x n cols
      FlipCopy f{i, 1, p.B, p.k, p.n, p.ldb, round8(p.k), off};
      off = round256(off + (size_t)f.cols * f.ld_dst * 2);
      out->push_back(f);
    }
  }
  return off;
}

}  // namespace

extern "C" {

sk_status sk_gemm_backward_workspace_size(const sk_problem *fwd, int need_dA, int need_dB, const sk_config *cfg,
                                          size_t *bytes) {
  if (!fwd || !bytes) return SK_ERR_INVALID_ARG;
  if (fwd->a_type != SK_BF16 || fwd->b_type != SK_BF16 || fwd->c_type != SK_BF16) return SK_ERR_UNSUPPORTED;
  if (fwd->m < 0 || fwd->n < 0 || fwd->k < 0) return SK_ERR_INVALID_ARG;
  // shapes only: placeholder (non-null) addresses
  static const unsigned char dummy[16] = {};
  sk_problem f = *fwd;
  if (!f.A) f.A = dummy;
  if (!f.B) f.B = dummy;
  sk_problem pr[2];
  const int n = backward_problems(&f, dummy, f.n > 0 ? f.n : 1, need_dA ? (void *)dummy : nullptr,
                                  f.a_layout == SK_ROW_MAJOR ? f.k : f.m, need_dB ? (void *)dummy : nullptr,
                                  f.b_layout == SK_ROW_MAJOR ? f.n : f.k, pr);
  if (n == 0) {
    *bytes = 256;
    return SK_OK;
  }
  size_t base = 0;
  sk_status rc = backward_gemm_ws(pr, n, cfg, &base);
  if (rc != SK_OK) return rc;
  std::vector<FlipCopy> flips;
  *bytes = plan_flips(pr, n, base, &flips);
  return SK_OK;
}

sk_status sk_gemm_backward(const sk_problem *fwd, const void *dC, int64_t lddc, void *dA, int64_t ldda, void *dB,
                           int64_t lddb, const sk_config *cfg, void *ws, size_t ws_bytes, sk_stream_t stream) {
  if (!fwd) return SK_ERR_INVALID_ARG;
  if (fwd->a_type != SK_BF16 || fwd->b_type != SK_BF16 || fwd->c_type != SK_BF16) return SK_ERR_UNSUPPORTED;
  if (fwd->m < 0 || fwd->n < 0 || fwd->k < 0) return SK_ERR_INVALID_ARG;
  sk_problem pr[2];
  const int n = backward_problems(fwd, dC, lddc, dA, ldda, dB, lddb, pr);
  if (n == 0) return SK_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // With room in the workspace past the GEMM's own bytes, the MN-major
  // operands are first copied to K-major layout there (one transpose
  // launch each), and the GEMMs read the copies.
  size_t base = 0;
  if (ws && backward_gemm_ws(pr, n, cfg, &base) == SK_OK) {
    std::vector<FlipCopy> flips;
    const size_t need = plan_flips(pr, n, base, &flips);
    bool degenerate = false;
    for (int i = 0; i < n; ++i) degenerate |= pr[i].m == 0 || pr[i].n == 0 || pr[i].k == 0;
    if (!flips.empty() && need <= ws_bytes && !degenerate) {
      int dev = 0, sms = 0;
      if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail_msg(SK_ERR_NO_DEVICE, "no CUDA device");
      for (const FlipCopy &f : flips) {
        void *dst = static_cast<uint8_t *>(ws) + f.offset;
        sk_status rc = cuda_err(launch_transpose16(f.src, f.rows, f.cols, f.ld_src, dst, f.ld_dst, sms, st),
                                "operand transpose launch");
        if (rc != SK_OK) return rc;
        sk_problem &p = pr[f.prob];
        if (f.operand == 0) {   // A(i,k) now at copy[i*ld + k]
          p.A = dst;
          p.a_layout = SK_ROW_MAJOR;
          p.lda = f.ld_dst;
        } else {                // B(k,j) now at copy[j*ld + k]
          p.B = dst;
          p.b_layout = SK_COL_MAJOR;
          p.ldb = f.ld_dst;
        }
      }
    }
  }
  // One grouped launch (Stream-K across both problems) or two single-problem
  // launches (the single-problem kernels, wider tiles), whichever the
  // runtime model predicts faster; both write the same results' values up to
  // the summation order of each plan.
  if (n == 2) {
    // (a configuration only single launches take -- 256 x 512 tiles --
    // runs as two single launches too)
    sk_plan_info g, s0, s1;
    const bool grouped_ok = sk_plan_query(pr, 2, cfg, 0, &g) == SK_OK;
    if (sk_plan_query(&pr[0], 1, cfg, 0, &s0) == SK_OK && sk_plan_query(&pr[1], 1, cfg, 0, &s1) == SK_OK &&
        (!grouped_ok || s0.predicted_us + s1.predicted_us < g.predicted_us)) {
      sk_status rc = run(&pr[0], 1, cfg, ws, ws_bytes, st, 1);
      if (rc != SK_OK) return rc;
      return run(&pr[1], 1, cfg, ws, ws_bytes, st, 1);
    }
  }
  return run(pr, n, cfg, ws, ws_bytes, st, MAX_PROBLEMS);
}

sk_status sk_transpose16(const void *src, int64_t rows, int64_t cols, int64_t ld_src, void *dst, int64_t ld_dst,
                         sk_stream_t stream) {
  if (rows < 0 || cols < 0 || ((rows > 0 && cols > 0) && (!src || !dst))) return SK_ERR_INVALID_ARG;
  if (ld_src < cols || ld_dst < rows) return SK_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(src) & 1u) || (reinterpret_cast<uintptr_t>(dst) & 1u)) return SK_ERR_INVALID_ARG;
  if (rows == 0 || cols == 0) return SK_OK;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail_msg(SK_ERR_NO_DEVICE, "no CUDA device");
  return cuda_err(launch_transpose16(src, rows, cols, ld_src, dst, ld_dst, sms, reinterpret_cast<cudaStream_t>(stream)),
                  "transpose launch");
}

sk_status sk_quantize_e4m3(const float *x, int64_t n, uint8_t *q, float *scale_out, float *amax_work,
                           sk_stream_t stream) {
  if (n < 0 || (n > 0 && (!x || !q)) || !scale_out || !amax_work) return SK_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(x) & 7u) || (reinterpret_cast<uintptr_t>(q) & 1u)) return SK_ERR_UNSUPPORTED;
  return cuda_err(launch_quant_e4m3(x, n, q, scale_out, amax_work, reinterpret_cast<cudaStream_t>(stream)),
                  "E4M3 quantise launch");
}

sk_status sk_get_status(const void *ws, size_t ws_bytes, sk_stream_t stream, int clear, sk_status *device_status) {
  if (!ws || ws_bytes < 256 || !device_status) return SK_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail_cuda("cudaStreamSynchronize", e);
  uint32_t v = 0;
  e = cudaMemcpy(&v, ws, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail_cuda("cudaMemcpy(status)", e);
  *device_status = v == 0 ? SK_OK : (sk_status)v;
  if (clear && v != 0) {
    e = cudaMemset(const_cast<void *>(ws), 0, sizeof(v));
    if (e != cudaSuccess) return fail_cuda("cudaMemset(status)", e);
  }
  return SK_OK;
}

sk_status sk_plan_query(const sk_problem *problems, int count, const sk_config *cfg, int num_sms,
                        sk_plan_info *out) {
  if (!out) return SK_ERR_INVALID_ARG;
  Cfg c;
  PlanOut pl;
  sk_status rc = plan_for_query(problems, count, cfg, num_sms, &c, &pl);
  if (rc != SK_OK) return rc;
  out->tile_m = c.BM;
  out->tile_n = c.BN;
  out->tile_k = c.BK;
  out->stages = c.stages;
  out->mode = c.mode;
  out->num_ctas = c.g;
  out->sk_units = pl.s.sk_units;
  out->tiles = pl.s.total_tiles;
  out->sk_tiles = pl.s.sk_tiles;
  out->dp_tiles = pl.s.total_tiles - pl.s.sk_tiles;
  out->sk_iters = pl.s.sk_iters;
  out->iters_per_unit = pl.s.q;
  out->extra_units = pl.s.r;
  out->workspace_bytes = ws_bytes_for(c, (size_t)pl.s.num_problems);
  out->predicted_us = pl.predicted_ns * 1e-3;
  out->fixup = c.fixup == FIXUP_SPLIT_CLUSTER ? SK_FIXUP_SPLIT_CLUSTER
               : c.fixup == FIXUP_SPLIT       ? SK_FIXUP_SPLIT
               : c.fixup == FIXUP_LAST_ARRIVER ? SK_FIXUP_LAST_ARRIVER
                                               : SK_FIXUP_OWNER;
  out->coverage_words = total_iters(pl) + pl.s.total_tiles * (int64_t)(c.BM / 32) * (c.BN / 32);
  return SK_OK;
}

sk_status sk_plan_unit_items(const sk_problem *problems, int count, const sk_config *cfg, int num_sms, int unit,
                             sk_work_item *items, int max_items, int *n_items) {
  if (!n_items || max_items < 0 || (max_items > 0 && !items)) return SK_ERR_INVALID_ARG;
  Cfg c;
  PlanOut pl;
  sk_status rc = plan_for_query(problems, count, cfg, num_sms, &c, &pl);
  if (rc != SK_OK) return rc;
  if (unit < 0 || unit >= c.g) return SK_ERR_INVALID_ARG;
  Cursor cur;
  cursor_init(pl.s, unit, cur);
  Item w;
  int n = 0;
  while (pl.s.num_problems > 0 && cursor_next(pl.s, pl.ps.data(), unit, cur, w)) {
    if (n < max_items) {
      sk_work_item &o = items[n];
      o.problem = pl.orig_index[w.problem];
      o.tile = w.tile;
      o.tile_row = w.tm;
      o.tile_col = w.tn;
      o.k0 = w.k0;
      o.k1 = w.k1;
      o.role = w.role;
      o.peer_first = w.peer_first;
      o.peer_last = w.peer_last;
      o.pad = 0;
      o.global_tile = w.gtile;
    }
    ++n;
  }
  *n_items = n;
  return SK_OK;
}

}  // extern "C"

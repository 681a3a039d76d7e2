// FP32 Stream-K GEMM on the SIMT FFMA pipes.
//
// One persistent CTA per unit walks the items the scheduler gives it
// (Stream-K segments first, then data-parallel tiles).  For each item it
// accumulates its k-block range of a 128x128 tile in registers (8x8 per
// thread), then, by role:
//   peer  : writes the FP32 partial to its workspace slot and raises its flag
//   owner : waits for its peers' flags (bounded), adds their partials in
//           ascending CTA order, then runs the epilogue
//   whole / dp : runs the epilogue
// With the last-arriver fixup, owner and peers both write their partials
// and count their arrival at the owner's counter; the CTA completing the
// count sums the partials in the same order (owner's, then peers
// ascending) and runs the epilogue.  Nobody waits.
// Epilogue: C = alpha * acc + beta * C_in, bounds-masked (no padding).
// FP32 needs FFMA: TF32 tensor-core products would miss the 5e-5 relative
// accuracy this path promises.
#include "common.cuh"
#include "ptx.cuh"

namespace sk {

namespace {

constexpr int PAD = 4;

struct F32Smem {
  float As[2][F32_BK][F32_BM + PAD];
  float Bs[2][F32_BK][F32_BN + PAD];
};

// Load the 128 x 16 slice of an operand into registers.  `rows` index the
// output dimension (M for A, N for B), `ks` the reduction dimension.
// kmajor: element (r, k) at X[r*rs + k] -> thread reads 8 consecutive k of one row.
// else  : element (r, k) at X[r + k*cs] -> thread reads 8 consecutive rows of one k.
__device__ __forceinline__ void load_slice(const float *X, int64_t rs, int64_t cs, int kmajor,
                                           int vec, int R, int Kd, int r0, int k0, float (&v)[8]) {
  const int t = threadIdx.x;
  if (kmajor) {
    const int r = r0 + (t & 127);
    const int k = k0 + (t >> 7) * 8;
    if (r < R) {
      const float *p = X + (int64_t)r * rs + k;
      if (vec && k + 8 <= Kd) {
        float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (k + e < Kd) ? __ldg(p + e) : 0.f;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = 0.f;
    }
  } else {
    const int k = k0 + (t >> 4);
    const int r = r0 + (t & 15) * 8;
    if (k < Kd) {
      const float *p = X + (int64_t)k * cs + r;
      if (vec && r + 8 <= R) {
        float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (r + e < R) ? __ldg(p + e) : 0.f;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = 0.f;
    }
  }
}

__device__ __forceinline__ void store_slice(float (*S)[F32_BM + PAD], int kmajor, const float (&v)[8]) {
  const int t = threadIdx.x;
  if (kmajor) {
    const int r = t & 127, k = (t >> 7) * 8;
#pragma unroll
    for (int e = 0; e < 8; ++e) S[k + e][r] = v[e];
  } else {
    const int k = t >> 4, r = (t & 15) * 8;
    *reinterpret_cast<float4 *>(&S[k][r]) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4 *>(&S[k][r + 4]) = make_float4(v[4], v[5], v[6], v[7]);
  }
}

template <int MAXP>
__global__ void __launch_bounds__(F32_THREADS, 1) sk_simt_f32_kernel(const __grid_constant__ SimtParams<MAXP> P) {
  __shared__ __align__(16) F32Smem sm;
  __shared__ uint32_t fix_word[2];   // last-arriver decisions, alternating
  int ndecide = 0;
  const bool last_arriver = P.fixup == FIXUP_LAST_ARRIVER;
  const bool split_reduce = P.fixup == FIXUP_SPLIT;
  const int t = threadIdx.x;
  const int ty = t >> 4, tx = t & 15;
  const int u = blockIdx.x;
  const Sched &S = P.sched;
  // Problem tables: inline in the parameter block, or, for groups larger
  // than MAXP, in global memory.
  const bool gtab = MAXP > 1 && P.gprob != nullptr;
  const SimtProblem *const probs = gtab ? P.gprob : P.prob;
  const ProbSched *const pss = gtab ? P.gps : P.ps;

  Cursor cur;
  cursor_init(S, u, cur);
  Item w;
  while (cursor_next(S, pss, u, cur, w)) {
    const SimtProblem &pr = probs[w.problem];
    const int m0 = w.tm * F32_BM, n0 = w.tn * F32_BN;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float ra[8], rb[8];
    load_slice(pr.A, pr.a_rs, pr.a_cs, pr.a_kmajor, pr.a_vec, pr.M, pr.K, m0, w.k0 * F32_BK, ra);
    load_slice(pr.B, pr.b_cs, pr.b_rs, pr.b_kmajor, pr.b_vec, pr.N, pr.K, n0, w.k0 * F32_BK, rb);
    store_slice(sm.As[0], pr.a_kmajor, ra);
    store_slice(sm.Bs[0], pr.b_kmajor, rb);
    cta_sync();

    for (int kb = w.k0; kb < w.k1; ++kb) {
      const int buf = (kb - w.k0) & 1;
      const bool more = kb + 1 < w.k1;
      if (more) {
        load_slice(pr.A, pr.a_rs, pr.a_cs, pr.a_kmajor, pr.a_vec, pr.M, pr.K, m0, (kb + 1) * F32_BK, ra);
        load_slice(pr.B, pr.b_cs, pr.b_rs, pr.b_kmajor, pr.b_vec, pr.N, pr.K, n0, (kb + 1) * F32_BK, rb);
      }
#pragma unroll
      for (int kk = 0; kk < F32_BK; ++kk) {
        float a[8], b[8];
        float4 a0 = *reinterpret_cast<const float4 *>(&sm.As[buf][kk][ty * 4]);
        float4 a1 = *reinterpret_cast<const float4 *>(&sm.As[buf][kk][64 + ty * 4]);
        float4 b0 = *reinterpret_cast<const float4 *>(&sm.Bs[buf][kk][tx * 4]);
        float4 b1 = *reinterpret_cast<const float4 *>(&sm.Bs[buf][kk][64 + tx * 4]);
        a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
        a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
        b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
        b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      if (more) {
        store_slice(sm.As[buf ^ 1], pr.a_kmajor, ra);
        store_slice(sm.Bs[buf ^ 1], pr.b_kmajor, rb);
      }
      cta_sync();
    }

    // Partial slot layout: float4 index v*256 + t, v = row_group*2 + col_half,
    // so consecutive threads touch consecutive 16-byte words.
    float4 *slot_base = reinterpret_cast<float4 *>(P.ws.partials);
    float4 *oslot_base = reinterpret_cast<float4 *>(P.ws.owner_partials);
    const int64_t slot_f4 = (int64_t)F32_BM * F32_BN / 4;
    auto spill = [&](float4 *slot) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int h = 0; h < 2; ++h)
          __stcg(slot + (i * 2 + h) * F32_THREADS + t,
                 make_float4(acc[i][h * 4 + 0], acc[i][h * 4 + 1], acc[i][h * 4 + 2], acc[i][h * 4 + 3]));
    };
    // acc = slot (assign) or acc += slot.
    auto gather = [&](const float4 *slot, bool assign) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float4 v = __ldcg(slot + (i * 2 + h) * F32_THREADS + t);
          if (assign) {
            acc[i][h * 4 + 0] = v.x;
            acc[i][h * 4 + 1] = v.y;
            acc[i][h * 4 + 2] = v.z;
            acc[i][h * 4 + 3] = v.w;
          } else {
            acc[i][h * 4 + 0] += v.x;
            acc[i][h * 4 + 1] += v.y;
            acc[i][h * 4 + 2] += v.z;
            acc[i][h * 4 + 3] += v.w;
          }
        }
    };
    auto broadcast = [&](bool mine) {
      volatile uint32_t *word = fix_word + (ndecide++ & 1);
      if (t == 0) *word = mine ? 1u : 0u;
      cta_sync();
      return *word != 0u;
    };

    if (split_reduce && (w.role == ROLE_PEER || w.role == ROLE_OWNER)) {
      // Split reduce (host-checked: every unit holds one tile-aligned
      // range): all contributors spill, count their arrival and wait for
      // the others; contributor j then sums the j-th share of the slot's
      // float4 words from all partials in the fixed order and stores it.
      int o = u, pl = w.peer_last;
      if (w.role == ROLE_PEER) {
        const ProbSched &q = pss[w.problem];
        const int64_t ts = q.iter_base + (int64_t)w.tile * q.iters;
        o = unit_of_iter(S, ts);
        pl = unit_of_iter(S, ts + q.iters - 1);
      }
      const int kc = pl - o + 1;
      const int jx = u - o;
      const int f0 = (int)(slot_f4 * jx / kc), f1 = (int)(slot_f4 * (jx + 1) / kc);
      spill(slot_base + (int64_t)u * slot_f4);
      __threadfence();
      cta_sync();
      uint32_t *cnt = P.ws.flags + o;
      // test-only injection: peers never count their arrival
      const bool withhold = (P.debug_flags & DEBUG_SKIP_PEER_FLAG) && w.role == ROLE_PEER;
      if (f0 == f1) {
        if (t == 0 && !withhold && (atom_add_acq_rel_gpu(cnt, 1u + SPLIT_DEPART) >> 16) == (uint32_t)(kc - 1))
          *cnt = 0u;
        continue;
      }
      if (t == 0) {
        if (!withhold) atom_add_acq_rel_gpu(cnt, 1u);
        const uint64_t t0 = globaltimer();
        while ((ld_relaxed_gpu(cnt) & 0xffffu) < (uint32_t)kc) {
          if (globaltimer() - t0 > P.timeout_ns) {
            atomicExch(P.ws.status, STATUS_TIMEOUT);
            break;
          }
        }
        fence_acq_rel_gpu();
      }
      cta_sync();
      for (int idx = f0 + t; idx < f1; idx += F32_THREADS) {
        float4 acc4 = __ldcg(slot_base + (int64_t)o * slot_f4 + idx);
        for (int p = o + 1; p <= pl; ++p) {
          const float4 q = __ldcg(slot_base + (int64_t)p * slot_f4 + idx);
          acc4.x += q.x;
          acc4.y += q.y;
          acc4.z += q.z;
          acc4.w += q.w;
        }
        // word idx = (row group i * 2 + column half h) * 256 + thread
        const int vv = idx / F32_THREADS, tt = idx - vv * F32_THREADS;
        const int i = vv >> 1, h = vv & 1, sty = tt >> 4, stx = tt & 15;
        const int row = m0 + (i < 4 ? sty * 4 + i : 64 + sty * 4 + (i - 4));
        const int col = n0 + h * 64 + stx * 4;
        if (row < pr.M) {
          const float o4[4] = {acc4.x, acc4.y, acc4.z, acc4.w};
          float *cp = pr.C + (int64_t)row * pr.ldc + col;
          const float *cin = pr.C_in ? pr.C_in + (int64_t)row * pr.ldc + col : nullptr;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (col + e < pr.N) {
              float r = pr.alpha * o4[e];
              if (pr.beta != 0.f) r += pr.beta * cin[e];
              cp[e] = r;
            }
          }
        }
      }
      cta_sync();
      if (t == 0 && (atom_add_acq_rel_gpu(cnt, SPLIT_DEPART) >> 16) == (uint32_t)(kc - 1)) *cnt = 0u;
      continue;
    } else if (w.role == ROLE_PEER) {
      spill(slot_base + (int64_t)u * slot_f4);
      __threadfence();
      cta_sync();
      if (!last_arriver) {
        if (t == 0 && !(P.debug_flags & DEBUG_SKIP_PEER_FLAG)) st_release_gpu(P.ws.flags + u, 1u);
        continue;
      }
      // Count this arrival at the tile's owner o; the CTA completing the
      // count (pl - o earlier arrivals) sums the tile in the fixed order.
      const ProbSched &q = pss[w.problem];
      const int64_t ts = q.iter_base + (int64_t)w.tile * q.iters;
      const int o = unit_of_iter(S, ts);
      const int pl = unit_of_iter(S, ts + q.iters - 1);
      bool mine = false;
      if (t == 0) mine = atom_add_acq_rel_gpu(P.ws.flags + o, 1u) == (uint32_t)(pl - o);
      if (!broadcast(mine)) continue;
      gather(oslot_base + (int64_t)o * slot_f4, true);
      for (int p = o + 1; p <= pl; ++p) gather(slot_base + (int64_t)p * slot_f4, false);
      if (t == 0) P.ws.flags[o] = 0u;
    } else if (w.role == ROLE_OWNER && last_arriver) {
      // If every peer has already arrived, sum now; otherwise write this
      // partial to the owner slot and count this arrival too.
      const uint32_t npeers = (uint32_t)(w.peer_last - w.peer_first + 1);
      bool mine = false;
      if (t == 0) {
        mine = ld_relaxed_gpu(P.ws.flags + u) == npeers;
        if (mine) fence_acq_rel_gpu();
      }
      if (!broadcast(mine)) {
        spill(oslot_base + (int64_t)u * slot_f4);
        __threadfence();
        cta_sync();
        if (t == 0) mine = atom_add_acq_rel_gpu(P.ws.flags + u, 1u) == npeers;
        if (!broadcast(mine)) continue;
      }
      for (int p = w.peer_first; p <= w.peer_last; ++p) gather(slot_base + (int64_t)p * slot_f4, false);
      if (t == 0) P.ws.flags[u] = 0u;
    } else if (w.role == ROLE_OWNER) {
      if (t == 0) {
        // Relaxed polls of every peer flag overlap; one acquire fence then
        // orders the partial reads after the peers' release stores.
        const uint64_t t0 = globaltimer();
        for (;;) {
          bool all = true;
          for (int p = w.peer_first; p <= w.peer_last; ++p) all &= ld_relaxed_gpu(P.ws.flags + p) != 0u;
          if (all) break;
          if (globaltimer() - t0 > P.timeout_ns) {
            atomicExch(P.ws.status, STATUS_TIMEOUT);
            break;
          }
        }
        fence_acq_rel_gpu();
      }
      cta_sync();
      // Fixed summation order: own partial, then peers in ascending CTA index.
      for (int p = w.peer_first; p <= w.peer_last; ++p) gather(slot_base + (int64_t)p * slot_f4, false);
      cta_sync();
      if (t == 0)
        for (int p = w.peer_first; p <= w.peer_last; ++p) P.ws.flags[p] = 0u;
    }

    // Epilogue.
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
      if (row >= pr.M) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int col = n0 + h * 64 + tx * 4;
        float o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) o[e] = pr.alpha * acc[i][h * 4 + e];
        float *cp = pr.C + (int64_t)row * pr.ldc + col;
        const float *cin = pr.C_in ? pr.C_in + (int64_t)row * pr.ldc + col : nullptr;
        if (pr.c_vec && col + 4 <= pr.N) {
          if (pr.beta != 0.f) {
            float4 c = *reinterpret_cast<const float4 *>(cin);
            o[0] += pr.beta * c.x; o[1] += pr.beta * c.y; o[2] += pr.beta * c.z; o[3] += pr.beta * c.w;
          }
          *reinterpret_cast<float4 *>(cp) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (col + e < pr.N) {
              float r = o[e];
              if (pr.beta != 0.f) r += pr.beta * cin[e];
              cp[e] = r;
            }
          }
        }
      }
    }
  }
}

}  // namespace

template <int MAXP>
cudaError_t launch_simt_f32(const SimtParams<MAXP> &p, int grid, cudaStream_t st) {
  (void)cudaGetLastError();   // drop a stale error left by an earlier call on this thread
  sk_simt_f32_kernel<MAXP><<<grid, F32_THREADS, 0, st>>>(p);
  return cudaGetLastError();
}

template cudaError_t launch_simt_f32<1>(const SimtParams<1> &, int, cudaStream_t);
template cudaError_t launch_simt_f32<MAXP_GROUPED>(const SimtParams<MAXP_GROUPED> &, int, cudaStream_t);

}  // namespace sk

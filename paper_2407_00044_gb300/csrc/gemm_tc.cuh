// Stream-K GEMM on the 5th-generation tensor cores (tcgen05), sm_103a.
//
// One persistent CTA per unit (192 threads, 1 CTA per SM):
//   warp 0 (lane 0) : TMA producer.  For every k-block of every item it waits
//                     for a free ring slot, then loads the 128 x BK slice of A
//                     and the BN x BK slice of B (128-byte swizzled rows) into
//                     shared memory, completing on the slot's `full` mbarrier.
//   warp 1          : allocates TMEM (2 accumulators of BN fp32 columns);
//                     lane 0 issues tcgen05.mma (M=128, N=BN) per k-block into
//                     the current accumulator, frees ring slots with
//                     tcgen05.commit, and signals `tmem_full` per item.
//   warps 2-5       : epilogue.  Each thread owns one accumulator row (TMEM
//                     lane).  By role: peer -> FP32 partial to the workspace
//                     + release flag; owner -> bounded acquire-wait on the
//                     peers' flags, add their partials in ascending CTA order;
//                     then C = alpha*acc + beta*C_in, rounded to the output
//                     type and stored with bounds masks (no padding).
// Two accumulators let the epilogue of item i overlap the MMAs of item i+1.
// All three roles walk the same item sequence from the shared scheduler.
//
// Every wait is bounded (timeout_ns of %globaltimer).  On expiry the kernel
// records STATUS_TIMEOUT in the workspace status word, raises a CTA-wide
// abort flag so the other roles stop issuing work, drains what it issued,
// frees TMEM and returns.
#pragma once
#include <cuda_bf16.h>

#include <type_traits>
#include "common.cuh"
#include "ptx.cuh"

namespace sk {

template <int IN>
struct InTraits;
template <>
struct InTraits<IN_BF16> {
  static constexpr int BK = 64;       // elements per k-block (128 bytes)
  static constexpr int UMMA_K = 16;   // K of one tcgen05.mma kind::f16
  // D f32 (bit 4), A bf16 (bits 7-9 = 1), B bf16 (bits 10-12 = 1)
  static constexpr uint32_t IDESC_TYPES = (1u << 4) | (1u << 7) | (1u << 10);
};
template <>
struct InTraits<IN_E4M3> {
  static constexpr int BK = 128;
  static constexpr int UMMA_K = 32;   // K of one tcgen05.mma kind::f8f6f4
  // D f32, A e4m3 (0), B e4m3 (0)
  static constexpr uint32_t IDESC_TYPES = (1u << 4);
};

template <>
struct InTraits<IN_TF32X3> {
  static constexpr int BK = 32;       // 128 bytes of FP32
  static constexpr int UMMA_K = 8;    // K of one tcgen05.mma kind::tf32
  // D f32 (bit 4), A tf32 (bits 7-9 = 2), B tf32 (bits 10-12 = 2)
  static constexpr uint32_t IDESC_TYPES = (1u << 4) | (2u << 7) | (2u << 10);
};

template <typename OutT>
struct OutStore;

template <>
struct OutStore<float> {
  // 32 consecutive outputs of one row.
  __device__ static __forceinline__ void run(const TcProblem &pr, int row, int col, const float (&v)[32],
                                             float alpha) {
    float *cp = static_cast<float *>(pr.C) + (int64_t)row * pr.ldc + col;
    const float *ci = pr.beta != 0.f ? static_cast<const float *>(pr.C_in) + (int64_t)row * pr.ldc + col : nullptr;
    if (pr.c_vec && col + 32 <= pr.N) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float4 o = make_float4(alpha * v[4 * j], alpha * v[4 * j + 1], alpha * v[4 * j + 2], alpha * v[4 * j + 3]);
        if (ci) {
          float4 c = *reinterpret_cast<const float4 *>(ci + 4 * j);
          o.x += pr.beta * c.x; o.y += pr.beta * c.y; o.z += pr.beta * c.z; o.w += pr.beta * c.w;
        }
        *reinterpret_cast<float4 *>(cp + 4 * j) = o;
      }
    } else {
      for (int j = 0; j < 32 && col + j < pr.N; ++j) {
        float o = alpha * v[j];
        if (ci) o += pr.beta * ci[j];
        cp[j] = o;
      }
    }
  }
};

template <>
struct OutStore<__nv_bfloat16> {
  __device__ static __forceinline__ void run(const TcProblem &pr, int row, int col, const float (&v)[32],
                                             float alpha) {
    __nv_bfloat16 *cp = static_cast<__nv_bfloat16 *>(pr.C) + (int64_t)row * pr.ldc + col;
    const __nv_bfloat16 *ci =
        pr.beta != 0.f ? static_cast<const __nv_bfloat16 *>(pr.C_in) + (int64_t)row * pr.ldc + col : nullptr;
    if (pr.c_vec && col + 32 <= pr.N) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float o[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) o[e] = alpha * v[8 * j + e];
        if (ci) {
          uint4 raw = *reinterpret_cast<const uint4 *>(ci + 8 * j);
          const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&raw);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float2 f = __bfloat1622float2(h[e]);
            o[2 * e] += pr.beta * f.x;
            o[2 * e + 1] += pr.beta * f.y;
          }
        }
        uint4 packed;
        __nv_bfloat162 *ph = reinterpret_cast<__nv_bfloat162 *>(&packed);
#pragma unroll
        for (int e = 0; e < 4; ++e) ph[e] = __floats2bfloat162_rn(o[2 * e], o[2 * e + 1]);
        *reinterpret_cast<uint4 *>(cp + 8 * j) = packed;
      }
    } else {
      for (int j = 0; j < 32 && col + j < pr.N; ++j) {
        float o = alpha * v[j];
        if (ci) o += pr.beta * __bfloat162float(ci[j]);
        cp[j] = __float2bfloat16_rn(o);
      }
    }
  }
};

// PAIR = false: one CTA per unit, 128 x BN tile, tcgen05 cta_group::1.
// BN = 512 (pairs, BF16 / E4M3): two N = 256 MMAs per k-step into one
//   512-column accumulator -- all of TMEM, so the epilogue of a tile is not
//   overlapped by the next tile's MMAs -- loading a quarter fewer operand
//   bytes per MAC than a 256 x 256 pair (12.5 % fewer shared-memory bytes,
//   TMA writes plus MMA operand reads, as both MMAs read A).  Each CTA
//   holds B rows [r*128, r*128+128) of either MMA's 256 columns.
// PAIR = true : a cluster of two CTAs per unit, 256 x BN tile.  Each CTA
//   TMA-loads its own 128 rows of A and its half (BN/2 rows) of B (either
//   operand K-major or MN-major) into its
//   own shared memory; both loads complete on the leader CTA's `full`
//   barrier; the leader's MMA warp issues tcgen05.mma.cta_group::2 (M=256),
//   which reads both CTAs' operands and writes rows 0-127 of the tile into
//   the leader's TMEM and rows 128-255 into the peer's; its commits arrive
//   on both CTAs' barriers (multicast).  Each CTA's epilogue handles its own
//   128 rows; both CTAs' epilogues release the leader's `tmem_empty`.  Each
//   CTA of a pair has its own partial slot and flag (index 2*unit + rank).
// XS = true (split tiles of exactly two contributors, FIXUP_SPLIT_CLUSTER):
//   a tile's two units run as one cluster -- two CTAs, or two CTA pairs
//   (cluster ranks 0-1 and 2-3, each pair its own cta_group::2 pair) -- and
//   each CTA writes the half of its accumulator rows that the other sums
//   straight into that CTA's shared memory (st.async, counted on its
//   mbarrier): no workspace, no flags.
template <int IN, typename OutT, int BN, int MAXP, bool PAIR, bool DBG, bool XS>
__global__ void __launch_bounds__(192, 1) sk_tc_kernel(const __grid_constant__ TcParams<MAXP> P) {
  using Tr = InTraits<IN>;
  constexpr int BM = PAIR ? 256 : 128;          // tile rows per unit
  constexpr int BK = Tr::BK;
  constexpr int UMMA_K = Tr::UMMA_K;
  constexpr int B_ROWS = PAIR ? BN / 2 : BN;    // rows of B (N direction) this CTA loads
  constexpr int A_BYTES = 128 * 128;
  constexpr int B_BYTES = B_ROWS * 128;
  // 3xTF32: each stage holds the loaded operands (read by the MMA as
  // their TF32 high parts) followed by their low parts.
  constexpr bool X3 = IN == IN_TF32X3;
  constexpr int OP_BYTES = A_BYTES + B_BYTES;
  constexpr int STAGE_BYTES = X3 ? 2 * OP_BYTES : OP_BYTES;
  // Where a CTA's operand loads complete: on its own `full` barrier (single
  // CTAs, and 3xTF32 pairs, whose splitting warps wait for their own CTA's
  // operands), or on the pair leader's (the leader's MMA issuer waits for
  // both halves there).
  constexpr bool OWN_FULL = !PAIR || X3;
  constexpr int TX_BYTES = OWN_FULL ? OP_BYTES : 2 * OP_BYTES;
  constexpr int MMA_N = BN > 256 ? 256 : BN;   // columns per MMA
  constexpr int NMMA = BN / MMA_N;               // MMAs per k-step (BN = 512: 2)
  constexpr int NACC = BN > 256 ? 1 : 2;         // TMEM accumulators (double-buffered up to BN = 256)
  constexpr int B_BLOCK = B_ROWS / NMMA;         // B rows of one MMA in this CTA
  constexpr uint32_t TMEM_COLS = NACC * BN;
  constexpr int MN_CHUNK_BYTES = BK * 128;   // one 64-wide MN chunk of an MN-major slice
  constexpr uint32_t IDESC = Tr::IDESC_TYPES | ((uint32_t)(MMA_N >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  static_assert(BN % 32 == 0 && BN >= 32 && (BN <= 256 || (BN == 512 && PAIR && !XS)), "tile N");
  static_assert(BN <= 256 || IN != IN_TF32X3, "512-column tiles: BF16 and E4M3 pairs");
  static_assert(!PAIR || BN % 64 == 0, "pair tile N");
  static_assert(!X3 || !PAIR || BN == 256, "3xTF32 pairs use 256 x 256 tiles");

  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  uint8_t *smem = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
  const int stages = P.stages;
  // [operand ring: stages x STAGE_BYTES][epilogue staging][barriers, TMEM slot]
  uint8_t *epi_stage = smem + stages * STAGE_BYTES;
  uint64_t *bars = reinterpret_cast<uint64_t *>(epi_stage + EPI_STAGE_BYTES);
  uint64_t *full_bar = bars;
  uint64_t *empty_bar = bars + stages;
  uint64_t *tfull_bar = bars + 2 * stages;
  uint64_t *tempty_bar = tfull_bar + 2;
  uint64_t *done_bar = tempty_bar + 2;
  uint64_t *fix_bar = done_bar + 1;   // FIX_SMEM_UNITS barriers of the staged fixup
  uint64_t *conv_bar = fix_bar + FIX_SMEM_UNITS;   // 3xTF32: stage split (one per stage; the leader's in a pair)
  uint64_t *xr_bar = conv_bar + (X3 ? stages : 0);   // XS: the partner's ring is free to write
  uint64_t *xd_bar = xr_bar + 1;                      // XS: per own unit, every partner's block has arrived
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(xd_bar + (XS ? XS_MAX_UNITS : 0));
  volatile uint32_t *abort_flag = tmem_slot + 1;
  volatile uint32_t *fix_word = tmem_slot + 2;   // two words: last-arriver decisions
  volatile uint32_t *fix_fail = tmem_slot + 4;   // two words: a staged-sum group failed
  const uint32_t tiles_addr = smem_u32(smem);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // clusters: a CTA pair, or, XS, the P.xs_k units of a tile (CTAs or pairs)
  constexpr bool CLUSTER = XS || PAIR;
  const uint32_t crank = CLUSTER ? cluster_ctarank() : 0u;
  const uint32_t rank = PAIR ? (XS ? (crank & 1u) : crank) : 0u;   // this CTA within its pair
  const uint32_t pbase = (PAIR && XS) ? (crank & ~1u) : 0u;        // cluster rank of its pair's leader
  const bool leader = rank == 0;
  const int u = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int slot_id = PAIR ? 2 * u + (int)rank : u;   // workspace slot / flag of this CTA
  const Sched &S = P.sched;
  const uint64_t tmo = P.timeout_ns;
  // Problem tables: inline in the parameter block, or, for groups larger
  // than MAXP, in global memory.
  const bool gtab = MAXP > 1 && P.gprob != nullptr;
  const TcProblem *const probs = gtab ? P.gprob : P.prob;
  const ProbSched *const pss = gtab ? P.gps : P.ps;

  // (debug variant) the moment this CTA entered the kernel, before any set-up
  if (DBG && threadIdx.x == 0) trace_put(P.trace, TRACE_ENTRY, 9, 0, globaltimer_ordered());
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(smem_u32(full_bar + s), 1);
      mbar_init(smem_u32(empty_bar + s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(tfull_bar + a), 1);
      mbar_init(smem_u32(tempty_bar + a), PAIR ? 8 : 4);
    }
    mbar_init(smem_u32(done_bar), 1);
    for (int b = 0; b < FIX_SMEM_UNITS; ++b) mbar_init(smem_u32(fix_bar + b), 1);
    if constexpr (XS) {
      mbar_init(smem_u32(xr_bar), (uint32_t)(P.xs_k - 1));   // one remote arrival per partner
      for (int l = 0; l < XS_MAX_UNITS; ++l) mbar_init(smem_u32(xd_bar + l), 1);   // this CTA's arrive.expect_tx
    }
    if constexpr (X3)   // the 4 epilogue warps of this CTA (of both CTAs in a pair)
      for (int s = 0; s < stages; ++s) mbar_init(smem_u32(conv_bar + s), PAIR ? 8 : 4);
    *abort_flag = 0;
    fix_fail[0] = fix_fail[1] = 0;
    fence_barrier_init();
    fence_proxy_async_smem();
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      tmem_alloc_pair(smem_u32(tmem_slot), TMEM_COLS);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  cta_sync();
  if constexpr (CLUSTER) cluster_sync();   // the other CTAs' barriers exist before anyone signals them
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // Timeline tracing and coverage counting are compiled only into the DBG
  // instantiations (launched when a trace or coverage buffer is given).
  uint64_t *const trace = DBG ? P.trace : nullptr;
  uint32_t *const cover = DBG ? P.cover : nullptr;
  if (DBG && threadIdx.x == 0) trace_put(trace, TRACE_CTA_BASE, 1, 0, globaltimer_ordered());

  auto fail = [&]() {
    *abort_flag = 1;
    atomicExch(P.ws.status, STATUS_TIMEOUT);
  };

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      if (!gtab) {
        const int np = S.num_problems < MAXP ? S.num_problems : MAXP;
        for (int p = 0; p < np && p < 4; ++p) {
          tma_prefetch_desc(&P.prob[p].tmap_a);
          tma_prefetch_desc(&P.prob[p].tmap_b);
        }
      }
      int acquired = -1;   // global-table problem whose tensor maps this thread has acquired
      int stage = 0;
      uint32_t phase = 0;
      int64_t loads = 0;
      Cursor c;
      cursor_init(S, u, c);
      Item w;
      bool ok = true;
      while (ok && !*abort_flag && cursor_next(S, pss, u, c, w)) {
        const TcProblem &pr = probs[w.problem];
        if (gtab && w.problem != acquired) {
          tensormap_acquire(&pr.tmap_a);
          tensormap_acquire(&pr.tmap_b);
          acquired = w.problem;
        }
        const int m0 = w.tm * BM + (int)rank * 128;
        // B rows of MMA j: n0 + j * MMA_N (+ 64 * chunk for MN-major loads)
        const int n0 = w.tn * BN + (int)rank * B_BLOCK;
        // Both operands K-major is the common case: one load per operand,
        // decided once per item (a per-load layout test in the pair loop
        // measured 16 % slower on 8192^3).
        const bool kmaj = !(pr.a_mn | pr.b_mn);
        for (int kb = w.k0; kb < w.k1; ++kb) {
          if (!mbar_wait(smem_u32(empty_bar + stage), phase ^ 1u, tmo) || *abort_flag) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(full_bar + stage);
          if (OWN_FULL || leader) mbar_arrive_expect_tx(fb, TX_BYTES);
          const uint32_t sa = tiles_addr + stage * STAGE_BYTES;
          const uint32_t sb = sa + A_BYTES;
          const int kx = kb * BK;
          if constexpr (!OWN_FULL) {
            const uint32_t fbl = mapa_shared(fb, pbase);   // the leader's barrier
            if (kmaj) {
              tma_load_2d_pair(sa, &pr.tmap_a, fbl, kx, m0);
#pragma unroll
              for (int j = 0; j < NMMA; ++j)
                tma_load_2d_pair(sb + j * B_BLOCK * 128, &pr.tmap_b, fbl, kx, n0 + j * MMA_N);
            } else {
              if (!pr.a_mn) {
                tma_load_2d_pair(sa, &pr.tmap_a, fbl, kx, m0);
              } else {
#pragma unroll
                for (int ch = 0; ch < 128 / 64; ++ch)
                  tma_load_2d_pair(sa + ch * MN_CHUNK_BYTES, &pr.tmap_a, fbl, m0 + 64 * ch, kx);
              }
              if (!pr.b_mn) {
#pragma unroll
                for (int j = 0; j < NMMA; ++j)
                  tma_load_2d_pair(sb + j * B_BLOCK * 128, &pr.tmap_b, fbl, kx, n0 + j * MMA_N);
              } else {
                constexpr int CPM = B_BLOCK / 64;   // 64-wide chunks per MMA block
#pragma unroll
                for (int ch = 0; ch < B_ROWS / 64; ++ch)
                  tma_load_2d_pair(sb + ch * MN_CHUNK_BYTES, &pr.tmap_b, fbl, n0 + (ch / CPM) * MMA_N + 64 * (ch % CPM),
                                   kx);
              }
            }
          } else {
            if (kmaj) {
              tma_load_2d(sa, &pr.tmap_a, fb, kx, m0);
              tma_load_2d(sb, &pr.tmap_b, fb, kx, n0);
            } else {
              if (!pr.a_mn) {
                tma_load_2d(sa, &pr.tmap_a, fb, kx, m0);
              } else {
#pragma unroll
                for (int ch = 0; ch < 128 / 64; ++ch)
                  tma_load_2d(sa + ch * MN_CHUNK_BYTES, &pr.tmap_a, fb, m0 + 64 * ch, kx);
              }
              if (!pr.b_mn) {
                tma_load_2d(sb, &pr.tmap_b, fb, kx, n0);
              } else {
#pragma unroll
                for (int ch = 0; ch < B_ROWS / 64; ++ch)
                  tma_load_2d(sb + ch * MN_CHUNK_BYTES, &pr.tmap_b, fb, n0 + 64 * ch, kx);
              }
            }
          }
          ++loads;
          if (++stage == stages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) fail();
      // Drain (bounded): every issued TMA load must land before the CTA may
      // exit -- slot s last completed phase `phase` if s < stage, else the
      // phase before (in a BF16/E4M3 pair, the leader's barrier sees both
      // CTAs' loads) -- and, on the normal path, every slot must have been
      // released by the MMA's commits.
      if (OWN_FULL || leader) {
        for (int s = 0; s < stages && s < loads; ++s) {
          const uint32_t par = s < stage ? phase : (phase ^ 1u);
          if (!mbar_wait(smem_u32(full_bar + s), par, tmo)) {
            fail();
            break;
          }
        }
      }
      for (int i = 0; i < stages && !*abort_flag; ++i) {
        if (!mbar_wait(smem_u32(empty_bar + stage), phase ^ 1u, tmo)) {
          fail();
          break;
        }
        if (++stage == stages) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0 && leader) {
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      Cursor c;
      cursor_init(S, u, c);
      Item w;
      bool ok = true;
      int nitem = 0;
      while (ok && !*abort_flag && cursor_next(S, pss, u, c, w)) {
        const TcProblem &pr = probs[w.problem];
        const uint32_t idesc = IDESC | ((uint32_t)pr.a_mn << 15) | ((uint32_t)pr.b_mn << 16);
        // Operand descriptors of stage 0, k-step 0; a stage / k-step offset is
        // added to the 14-bit start-address field (addresses < 256 KB, so the
        // field cannot carry).  K-major: UMMA_K advances 32 bytes along the
        // swizzled row; MN-major: UMMA_K rows of 128 bytes.
        const uint64_t a_desc0 = smem_desc_sw128(tiles_addr, pr.a_mn ? MN_CHUNK_BYTES : 16, 1024);
        const uint64_t b_desc0 = smem_desc_sw128(tiles_addr + A_BYTES, pr.b_mn ? MN_CHUNK_BYTES : 16, 1024);
        const uint32_t a_kstep = pr.a_mn ? (UMMA_K * 128) >> 4 : 32 >> 4;
        const uint32_t b_kstep = pr.b_mn ? (UMMA_K * 128) >> 4 : 32 >> 4;
        const int tr = TRACE_MMA_BASE + 3 * nitem;
        const bool got = PAIR ? mbar_wait_cluster(smem_u32(tempty_bar + acc), acc_phase ^ 1u, tmo)
                              : mbar_wait(smem_u32(tempty_bar + acc), acc_phase ^ 1u, tmo);
        if (!got) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (DBG && nitem < 16) trace_put(trace, tr, 2, nitem, globaltimer());
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
        for (int kb = w.k0; kb < w.k1; ++kb) {
          // 3xTF32 waits for the epilogue warps' conversion of the stage
          // (in a pair: of both CTAs' halves, arriving on the leader's barrier)
          const bool got_stage = (X3 && PAIR) ? mbar_wait_cluster(smem_u32(conv_bar + stage), phase, tmo)
                                              : mbar_wait(smem_u32((X3 ? conv_bar : full_bar) + stage), phase, tmo);
          if (!got_stage) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t soff = (uint64_t)((stage * STAGE_BYTES) >> 4);
#pragma unroll
          for (int kk = 0; kk < BK / UMMA_K; ++kk) {
            const uint64_t ad = a_desc0 + soff + (uint64_t)(kk * a_kstep);
            const uint64_t bd = b_desc0 + soff + (uint64_t)(kk * b_kstep);
            const uint32_t accum = (kb > w.k0 || kk > 0) ? 1u : 0u;
            if constexpr (X3) {
              // a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (the low parts
              // sit OP_BYTES after the high parts)
              constexpr uint64_t LO = (uint64_t)(OP_BYTES >> 4);
              if constexpr (PAIR) {
                mma_tf32_pair(d_tmem, ad, bd, idesc, accum);
                mma_tf32_pair(d_tmem, ad, bd + LO, idesc, 1u);
                mma_tf32_pair(d_tmem, ad + LO, bd, idesc, 1u);
              } else {
                mma_tf32(d_tmem, ad, bd, idesc, accum);
                mma_tf32(d_tmem, ad, bd + LO, idesc, 1u);
                mma_tf32(d_tmem, ad + LO, bd, idesc, 1u);
              }
            } else if constexpr (PAIR) {
              // (BN = 512: MMA j reads this CTA's B block j, B_BLOCK rows on,
              // and writes accumulator columns [j * 256, j * 256 + 256))
#pragma unroll
              for (int j = 0; j < NMMA; ++j) {
                const uint64_t bdj = bd + (uint64_t)((j * B_BLOCK * 128) >> 4);
                if constexpr (IN == IN_BF16)
                  mma_f16_pair(d_tmem + j * MMA_N, ad, bdj, idesc, accum);
                else
                  mma_f8_pair(d_tmem + j * MMA_N, ad, bdj, idesc, accum);
              }
            } else {
              if constexpr (IN == IN_BF16)
                mma_f16(d_tmem, ad, bd, idesc, accum);
              else
                mma_f8(d_tmem, ad, bd, idesc, accum);
            }
          }
          if constexpr (PAIR)
            mma_commit_pair_mc(smem_u32(empty_bar + stage), (uint16_t)(3u << pbase));
          else
            mma_commit(smem_u32(empty_bar + stage));
          if (DBG && cover) {
            // this unit issued MAC-loop iteration (tile, kb)
            const ProbSched &q = pss[w.problem];
            atomicAdd(cover + q.iter_base + (int64_t)w.tile * q.iters + kb, cover_visit(u));
          }
          if (++stage == stages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        if constexpr (PAIR)
          mma_commit_pair_mc(smem_u32(tfull_bar + acc), (uint16_t)(3u << pbase));
        else
          mma_commit(smem_u32(tfull_bar + acc));
        if (DBG && nitem < 16) trace_put(trace, tr + 2, 4, nitem, globaltimer());
        ++nitem;
        if (++acc == NACC) {
          acc = 0;
          acc_phase ^= 1u;
        }
      }
      if (!ok) fail();
      // All MMAs issued by this thread are complete once done_bar flips.
      if constexpr (PAIR)
        mma_commit_pair_mc(smem_u32(done_bar), (uint16_t)(1u << pbase));
      else
        mma_commit(smem_u32(done_bar));
      if (!mbar_wait(smem_u32(done_bar), 0u, tmo)) fail();
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q4 = warp & 3;                 // TMEM lane quarter this warp may access
    const int row = q4 * 32 + lane;          // accumulator row of this thread
    const int et = threadIdx.x - 64;         // 0..127
    // TMA-store staging of this warp: two 4 KB buffers of 32 rows x 128 B,
    // 128-byte swizzled (16-byte chunk c of row r at chunk c ^ (r % 8)).
    uint8_t *const my_stage = epi_stage + (warp - 2) * 8192;
    int sbuf = 0;
    float4 *const slots = reinterpret_cast<float4 *>(P.ws.partials);         // peer segments
    float4 *const oslots = reinterpret_cast<float4 *>(P.ws.owner_partials);  // owner segments (last arriver)
    constexpr int64_t SLOT_F4 = (int64_t)128 * BN / 4;
    const bool last_arriver = P.fixup == FIXUP_LAST_ARRIVER;
    const bool split_reduce = P.fixup == FIXUP_SPLIT;
    int ndecide = 0;   // last-arriver decisions so far; its parity picks the smem word
    int acc = 0;
    uint32_t acc_phase = 0;
    Cursor c;
    cursor_init(S, u, c);
    Item w;
    // Releases accumulator `a` to the MMA issuer (the leader's barrier).
    auto release_acc = [&](int a) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if constexpr (PAIR)
          mbar_arrive_cluster(mapa_shared(smem_u32(tempty_bar + a), pbase));
        else
          mbar_arrive(smem_u32(tempty_bar + a));
      }
    };
    // Slot / flag / counter index of unit p's CTA holding these rows.
    auto cslot = [&](int p) { return PAIR ? 2 * p + (int)rank : p; };
    int nitem = 0;
    const bool tr_lead = DBG && et == 0;
    // Loop exit and wait results are made uniform over the 128 epilogue
    // threads: the lanes of a warp must stay converged for the
    // warp-collective tcgen05.ld, and all four warps must reach the same
    // named barriers.
    int cstage = 0;          // 3xTF32: next stage to convert and its phase
    uint32_t cphase = 0;
    while (cursor_next(S, pss, u, c, w)) {
      const TcProblem &pr = probs[w.problem];
      if constexpr (X3) {
        // Split every loaded FP32 value x of the item's stages: the MMA
        // reads the FP32 container itself as x_hi (kind::tf32 drops the low
        // 13 mantissa bits: x_hi = x truncated to TF32), and x_lo =
        // tf32_rn(x - x_hi) (the difference is exact in FP32) is written
        // OP_BYTES further on; then the stage goes to the MMA issuer.  The
        // operation is elementwise, so the swizzled layout is kept as TMA
        // wrote it.  (Measured: with x_lo taken against truncation the
        // worst error is 3.3e-7 of S at K = 16384; had the MMA rounded the
        // container instead, it would be of order 2^-11.)
        for (int kb = w.k0; kb < w.k1; ++kb) {
          if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(full_bar + cstage), cphase, tmo)) || *abort_flag) {
            if (lane == 0) fail();
            break;
          }
          float4 *x = reinterpret_cast<float4 *>(smem + cstage * STAGE_BYTES);
          float4 *lo = x + OP_BYTES / 16;
          // fully unrolled (16 words a thread): the loads of a stage are in
          // flight together (measured 16 % faster at 4096^3 than 4-deep)
#pragma unroll
          for (int i = et; i < OP_BYTES / 16; i += 128) {
            const float4 v = x[i];
            const float4 h = make_float4(trunc_tf32(v.x), trunc_tf32(v.y), trunc_tf32(v.z), trunc_tf32(v.w));
            lo[i] = make_float4(round_tf32(v.x - h.x), round_tf32(v.y - h.y), round_tf32(v.z - h.z),
                                round_tf32(v.w - h.w));
          }
          fence_proxy_async_smem_cta();   // the generic writes, to the tensor cores' reads
          __syncwarp();
          if (lane == 0) {
            if constexpr (PAIR)   // the leader's MMAs read both CTAs' halves
              mbar_arrive_cluster(mapa_shared(smem_u32(conv_bar + cstage), pbase));
            else
              mbar_arrive(smem_u32(conv_bar + cstage));
          }
          if (++cstage == stages) {
            cstage = 0;
            cphase ^= 1u;
          }
        }
      }
      const bool got = mbar_wait(smem_u32(tfull_bar + acc), acc_phase, tmo);
      if (named_bar_or(1, 128, !got || *abort_flag != 0u)) {
        if (!got) fail();
        break;
      }
      tc_fence_after();
      const int tr = TRACE_EPI_BASE + 3 * nitem;
      if (tr_lead && nitem < 21) trace_put(trace, tr, 5, nitem, globaltimer_ordered());
      const uint32_t tbase = tmem_base + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(acc * BN);
      // The item is this CTA's last: every MMA has completed, so the operand
      // ring in shared memory is free for staging partials.
      const bool ring_free = c.it >= c.end && c.dp >= S.total_tiles;

      auto get_alpha = [&]() {
        float alpha = pr.alpha;
        if (IN == IN_E4M3) {
          if (pr.scale_a) alpha *= *pr.scale_a;
          if (pr.scale_b) alpha *= *pr.scale_b;
        }
        return alpha;
      };
      const int grow = w.tm * BM + (int)rank * 128 + row;
      const int row0 = w.tm * BM + (int)rank * 128 + q4 * 32;   // first row of this warp
      auto store_chunk = [&](int ch, const float (&v)[32], float alpha) {
        if (DBG && cover && lane == 0) {
          // this unit stores the 32 x 32 block (rows of this warp, chunk ch)
          constexpr int BLK_N = BN / 32;
          const int64_t blk = w.gtile * (int64_t)(BM / 32) * BLK_N + ((int)rank * 4 + q4) * BLK_N + ch;
          atomicAdd(cover + P.cover_iters + blk, cover_visit(u));
        }
        if (pr.c_tma) {
          // Stage the chunk in shared memory and write it with one TMA
          // store per 128-byte-wide box (BF16: 64 columns = two chunks;
          // FP32: 32 columns); TMA clips rows/columns outside C.
          constexpr bool F32OUT = sizeof(OutT) == 4;
          const int part = F32OUT ? 0 : (ch & 1);
          uint8_t *buf = my_stage + sbuf * 4096;
          if (part == 0) {
            if (lane == 0) bulk_wait_group_read<1>();   // this buffer's previous store has read it
            __syncwarp();
          }
          uint8_t *rowp = buf + lane * 128;
          if constexpr (F32OUT) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
              *reinterpret_cast<float4 *>(rowp + ((q ^ (lane & 7)) * 16)) =
                  make_float4(alpha * v[4 * q], alpha * v[4 * q + 1], alpha * v[4 * q + 2], alpha * v[4 * q + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              uint4 pk;
              __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&pk);
#pragma unroll
              for (int e = 0; e < 4; ++e)
                h[e] = __floats2bfloat162_rn(alpha * v[8 * q + 2 * e], alpha * v[8 * q + 2 * e + 1]);
              *reinterpret_cast<uint4 *>(rowp + (((part * 4 + q) ^ (lane & 7)) * 16)) = pk;
            }
          }
          if (F32OUT || part == 1) {
            fence_proxy_async_smem_cta();
            __syncwarp();
            if (lane == 0) {
              tma_store_2d(&P.tmap_c[0], smem_u32(buf), w.tn * BN + (ch - part) * 32, row0);
              bulk_commit_group();
            }
            sbuf ^= 1;
          }
        } else if (grow < pr.M) {
          const int gcol = w.tn * BN + ch * 32;
          if (gcol < pr.N) OutStore<OutT>::run(pr, grow, gcol, v, alpha);
        }
      };
      // Writes this CTA's accumulator rows to a workspace slot in TMEM
      // fragment order: float4 ((chunk*4 + q4)*8 + j)*32 + lane, so a warp
      // writes 512 contiguous bytes per store, a 32-column chunk of all
      // rows is one 16 KB block and a warp's 32 rows of it one 4 KB block.
      // Leaves out the chunks for which skip(ch) holds.
      auto spill = [&](float4 *slot, auto skip) {
        // two chunks per TMEM load where both leave
#pragma unroll 1
        for (int ch = 0; ch < BN / 32; ch += 2) {
          const bool s0 = skip(ch), s1 = skip(ch + 1);
          if (s0 && s1) continue;
          if (!s0 && !s1) {
            float v[64];
            tmem_ld64(tbase + ch * 32, v);
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
              for (int j = 0; j < 8; ++j)
                __stcg(slot + (((ch + h) * 4 + q4) * 8 + j) * 32 + lane,
                       make_float4(v[32 * h + 4 * j], v[32 * h + 4 * j + 1], v[32 * h + 4 * j + 2],
                                   v[32 * h + 4 * j + 3]));
          } else {
            const int c1 = s0 ? ch + 1 : ch;
            float v[32];
            tmem_ld32(tbase + c1 * 32, v);
#pragma unroll
            for (int j = 0; j < 8; ++j)
              __stcg(slot + ((c1 * 4 + q4) * 8 + j) * 32 + lane,
                     make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
          }
        }
      };
      auto no_skip = [](int) { return false; };
      // Sums the partials of a tile whose k-blocks units o..pl computed, in
      // the fixed order: unit o's partial (k-block 0; from this CTA's TMEM
      // if own_in_tmem, else from o's owner slot), then units o+1..pl
      // ascending (their peer slots), and stores C.  Every partial has been
      // acquired by the caller.  own_in_tmem is a compile-time constant: a
      // run-time flag here measured 2 us slower on 128 x 8192 x 16384.
      auto fixup_sum = [&](auto own_c, int o, int pl) {
        constexpr bool own_in_tmem = decltype(own_c)::value;
        const float alpha = get_alpha();
        constexpr int NCH = BN / 32;
        auto src_of = [&](int ch, int ti) -> const float4 * {
          // ti-th staged term: own_in_tmem ? peer o+1+ti : (ti == 0 ? owner o : peer o+ti)
          const float4 *base = own_in_tmem ? slots + (int64_t)cslot(o + 1 + ti) * SLOT_F4
                               : ti == 0   ? oslots + (int64_t)cslot(o) * SLOT_F4
                                           : slots + (int64_t)cslot(o + ti) * SLOT_F4;
          return base + (ch * 8) * 128;
        };
        const int nst = (pl - o) + (own_in_tmem ? 0 : 1);   // terms read from the workspace
        if (ring_free) {
          // Stage the partials in the idle ring with bulk copies, 16 KB units
          // (chunk, term) in chunk-major order, up to FIX_SMEM_UNITS in flight.
          const int nunits = NCH * nst;
          int nb = (stages * STAGE_BYTES) / FIX_UNIT_BYTES;
          if (nb > FIX_SMEM_UNITS) nb = FIX_SMEM_UNITS;
          float v[32];
          int group = 0;
          for (int g0 = 0; g0 < nunits; g0 += nb, ++group) {
            const int gn = nunits - g0 < nb ? nunits - g0 : nb;
            if (tr_lead && group == 0) trace_put(trace, TRACE_FIX_BASE, 11, nitem, globaltimer_ordered());
            if (et < gn) {
              // one copy per thread (gn <= FIX_SMEM_UNITS): address
              // arithmetic and issue in parallel
              const int i = g0 + et;
              const int ch = i / nst;
              const uint32_t fb = smem_u32(fix_bar + et);
              fence_proxy_async_global();   // the acquired partials, to the copy engine
              mbar_arrive_expect_tx(fb, FIX_UNIT_BYTES);
              bulk_copy_g2s(tiles_addr + et * FIX_UNIT_BYTES, src_of(ch, i - ch * nst), FIX_UNIT_BYTES, fb);
            }
            for (int b = 0; b < gn; ++b) {
              const int i = g0 + b;
              const int ch = i / nst;
              const int ti = i - ch * nst;
              if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(fix_bar + b), (uint32_t)(group & 1), tmo))) {
                fail();
                if (lane == 0) fix_fail[group & 1] = 1u;
                break;
              }
              if (tr_lead && group == 0 && b == 0) trace_put(trace, TRACE_FIX_BASE + 1, 12, nitem, globaltimer_ordered());
              if (tr_lead && group == 0 && b == gn - 1) trace_put(trace, TRACE_FIX_BASE + 2, 13, nitem, globaltimer_ordered());
              const float4 *sb = reinterpret_cast<const float4 *>(smem + b * FIX_UNIT_BYTES);
              if (ti == 0 && !own_in_tmem) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  const float4 q = sb[(q4 * 8 + j) * 32 + lane];
                  v[4 * j] = q.x;
                  v[4 * j + 1] = q.y;
                  v[4 * j + 2] = q.z;
                  v[4 * j + 3] = q.w;
                }
              } else {
                if (ti == 0) tmem_ld32(tbase + ch * 32, v);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  const float4 q = sb[(q4 * 8 + j) * 32 + lane];
                  v[4 * j] += q.x;
                  v[4 * j + 1] += q.y;
                  v[4 * j + 2] += q.z;
                  v[4 * j + 3] += q.w;
                }
              }
              if (ti == nst - 1) store_chunk(ch, v, alpha);
            }
            // Every thread is done with the group's buffers; a failed wait
            // in any warp ends the sum in all of them.  (A group's failure
            // word is written only before its barrier and, alternating by
            // parity, not again before every thread has read it; a plain
            // barrier here measured faster than a reducing one.)
            named_bar_sync(1, 128);
            if (fix_fail[group & 1] != 0u) break;
          }
        } else {
          // More work follows on this CTA: the sum overlaps the next item's
          // MMAs, so plain loads suffice.
#pragma unroll 1
          for (int ch = 0; ch < NCH; ++ch) {
            float v[32];
            if (own_in_tmem) {
              tmem_ld32(tbase + ch * 32, v);
            } else {
              const float4 *src = src_of(ch, 0) + q4 * 256 + lane;
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float4 q = __ldcg(src + j * 32);
                v[4 * j] = q.x;
                v[4 * j + 1] = q.y;
                v[4 * j + 2] = q.z;
                v[4 * j + 3] = q.w;
              }
            }
            for (int ti = own_in_tmem ? 0 : 1; ti < nst; ++ti) {
              const float4 *src = src_of(ch, ti) + q4 * 256 + lane;
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float4 q = __ldcg(src + j * 32);
                v[4 * j] += q.x;
                v[4 * j + 1] += q.y;
                v[4 * j + 2] += q.z;
                v[4 * j + 3] += q.w;
              }
            }
            store_chunk(ch, v, alpha);
          }
        }
      };
      // Last-arriver fixup: one thread's decision, broadcast to the 128
      // epilogue threads through one of two shared words (alternating, so
      // a word is rewritten only after every thread has read it).
      auto broadcast = [&](bool mine) {
        volatile uint32_t *word = fix_word + (ndecide++ & 1);
        if (et == 0) *word = mine ? 1u : 0u;
        named_bar_sync(1, 128);
        return *word != 0u;
      };

      // Which sum, if any, this CTA does for the item: units o..pl's
      // partials, the first from TMEM (own_tmem) or from o's owner slot.
      bool do_sum = false, own_tmem = true;
      int o = u, pl = w.peer_last;
      if (XS && (w.role == ROLE_PEER || w.role == ROLE_OWNER)) {
        // Cluster split (the host launches it only when every tile has
        // exactly kc = P.xs_k contributors (2, 4 or 8), they are the
        // cluster's kc units in unit order (contributor jx = u - o holds
        // k-range jx; jx = 0 is the owner), and the operand ring holds the
        // exchanged blocks).  The tile's (column group x warp) units are
        // dealt out as in the split reduce: unit s is 32-column chunk group
        // s / 4 (UW chunks) of warp s % 4, contributor j sums units
        // [j NS / kc, (j+1) NS / kc).  Each warp sends the blocks of its
        // units that other contributors sum -- TMEM -> registers -> a
        // staging block in its own idle ring (TMEM-fragment order, 4 KB per
        // chunk) -> one bulk copy into the receiver's ring, counted on the
        // receiver's data barrier -- once every partner has signalled that
        // its MMAs are done (its ring is free).  Then each warp sums its own
        // units from the kc partials in ascending contributor order (its
        // own from TMEM at its place), the order every other protocol uses,
        // so C is bit-identical to them.
        constexpr int UW = sizeof(OutT) == 4 ? 1 : 2;   // 32-column chunks per unit
        constexpr int NS = 4 * (BN / 32) / UW;          // units of the tile
        constexpr uint32_t BLK = UW * 4096;             // one unit of one partial
        const int kc = P.xs_k;
        const int jx = (int)(PAIR ? (crank >> 1) : crank);
        auto s_lo = [&](int j) { return j * NS / kc; };
        auto cta_of = [&](int j) { return (uint32_t)(PAIR ? 2 * j + (int)rank : j); };
        const int s0 = s_lo(jx), s1 = s_lo(jx + 1), own_n = s1 - s0;
        // ring: [incoming: (kc - 1) sources x own_n units][outgoing staging:
        // the other contributors' units in unit order]
        const uint32_t out_base = (uint32_t)((kc - 1) * own_n) * BLK;
        if (et == 0) {
          // one barrier per own unit: its kc - 1 incoming blocks
          for (int l = 0; l < own_n; ++l) mbar_arrive_expect_tx(smem_u32(xd_bar + l), (uint32_t)(kc - 1) * BLK);
          for (int i = 0; i < kc; ++i)
            if (i != jx) mbar_arrive_cluster(mapa_shared(smem_u32(xr_bar), cta_of(i)));   // this ring is free
        }
        // (cluster-scope acquires: the arrivals and the data come from the partners)
        bool okx = mbar_wait_cluster(smem_u32(xr_bar), 0u, tmo);
        if (named_bar_or(1, 128, !okx)) {
          if (et == 0) fail();
        } else {
#pragma unroll 1
          for (int s = q4; s < NS; s += 4) {
            if (s >= s0 && s < s1) continue;
            int i = s * kc / NS;   // the contributor that sums unit s
            while (s_lo(i + 1) <= s) ++i;
            while (s_lo(i) > s) --i;
            const int own_i = s_lo(i + 1) - s_lo(i);
            const uint32_t src_slot = (uint32_t)(jx < i ? jx : jx - 1);   // this CTA among i's sources
            const uint32_t dst_off = (src_slot * (uint32_t)own_i + (uint32_t)(s - s_lo(i))) * BLK;
            const uint32_t stg_off = out_base + (uint32_t)(s - (s >= s1 ? own_n : 0)) * BLK;
            float4 *const stg = reinterpret_cast<float4 *>(smem + stg_off);
#pragma unroll
            for (int h = 0; h < UW; ++h) {
              float v[32];
              tmem_ld32(tbase + ((s / 4) * UW + h) * 32, v);
#pragma unroll
              for (int j = 0; j < 8; ++j)
                stg[(h * 8 + j) * 32 + lane] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            }
            fence_proxy_async_smem_cta();   // the generic writes, to the copy engine
            __syncwarp();
            if (lane == 0)
              bulk_copy_s2cluster(mapa_shared(tiles_addr + dst_off, cta_of(i)), tiles_addr + stg_off, BLK,
                                  mapa_shared(smem_u32(xd_bar + (s - s_lo(i))), cta_of(i)));
          }
          if (tr_lead) trace_put(trace, TRACE_FIX_BASE + 5, 15, nitem, globaltimer_ordered());   // blocks sent
          const float alpha = get_alpha();
          bool first = true;
#pragma unroll 1
          for (int s = s0 + ((q4 - s0 % 4) + 4) % 4; s < s1; s += 4) {   // this warp's own units
            // summed as soon as the unit's blocks have landed
            okx = __all_sync(0xffffffffu, mbar_wait_cluster(smem_u32(xd_bar + (s - s0)), 0u, tmo));
            if (!okx && lane == 0) fail();
            if (tr_lead && first && nitem < 21) trace_put(trace, tr + 1, 6, nitem, globaltimer_ordered());
            first = false;
#pragma unroll
            for (int h = 0; h < UW; ++h) {
              float v[32];
              for (int i = 0; i < kc; ++i) {
                if (i == jx) {
                  float t[32];
                  tmem_ld32(tbase + ((s / 4) * UW + h) * 32, t);
#pragma unroll
                  for (int e = 0; e < 32; ++e) v[e] = i == 0 ? t[e] : v[e] + t[e];
                } else {
                  const uint32_t src_slot = (uint32_t)(i < jx ? i : i - 1);
                  const float4 *blk = reinterpret_cast<const float4 *>(
                      smem + (src_slot * (uint32_t)own_n + (uint32_t)(s - s0)) * BLK);
#pragma unroll
                  for (int j = 0; j < 8; ++j) {
                    const float4 q = blk[(h * 8 + j) * 32 + lane];
                    if (i == 0) {
                      v[4 * j] = q.x;
                      v[4 * j + 1] = q.y;
                      v[4 * j + 2] = q.z;
                      v[4 * j + 3] = q.w;
                    } else {
                      v[4 * j] += q.x;
                      v[4 * j + 1] += q.y;
                      v[4 * j + 2] += q.z;
                      v[4 * j + 3] += q.w;
                    }
                  }
                }
              }
              store_chunk((s / 4) * UW + h, v, alpha);
            }
          }
        }
        release_acc(acc);
        if (tr_lead && nitem < 21) trace_put(trace, tr + 2, 7, nitem, globaltimer_ordered());
      } else if (split_reduce && (w.role == ROLE_PEER || w.role == ROLE_OWNER)) {
        // Split reduce (the host uses it only when every unit holds one
        // tile-aligned range, so a tile's units finish together): every
        // contributor spills what the others sum, counts its arrival, waits
        // (bounded) for all of them; then each of its warps sums its units
        // from all the partials in the fixed order and stores them.
        if (w.role == ROLE_PEER) {
          const ProbSched &q = pss[w.problem];
          const int64_t ts = q.iter_base + (int64_t)w.tile * q.iters;
          o = unit_of_iter(S, ts);
          pl = unit_of_iter(S, ts + q.iters - 1);
        }
        const int kc = pl - o + 1;
        const int jx = u - o;
        // A unit is UW chunks (64 columns for BF16 output, the width of its
        // TMA store box; 32 for FP32) of one warp's 32 rows; unit s covers
        // chunk group s / 4 of warp s % 4, and contributor jx takes units
        // [s0, s1), so consecutive units go to different warps.
        constexpr int UW = sizeof(OutT) == 4 ? 1 : 2;
        constexpr int NS = 4 * (BN / 32) / UW;
        const int s0 = jx * NS / kc, s1 = (jx + 1) * NS / kc;
        const int s_first = s0 + ((q4 - s0 % 4) + 4) % 4;   // this warp's first unit
        const int nunit_w = s_first < s1 ? (s1 - 1 - s_first) / 4 + 1 : 0;
        // This warp's own units stay in TMEM and enter the sum in their
        // place; the rest of its rows go to the workspace.
        spill(slots + (int64_t)slot_id * SLOT_F4, [&](int ch) {
          const int su = (ch / UW) * 4 + q4;
          return su >= s0 && su < s1;
        });
        if (nunit_w == 0) release_acc(acc);
        __threadfence();
        if (tr_lead) trace_put(trace, TRACE_FIX_BASE + 5, 15, nitem, globaltimer_ordered());   // spill visible
        named_bar_sync(1, 128);
        uint32_t *cnt = P.ws.flags + cslot(o);
        // test-only injection: peers never count their arrival, so every
        // other contributor's bounded wait expires
        const bool withhold = (P.debug_flags & DEBUG_SKIP_PEER_FLAG) && w.role == ROLE_PEER;
        // Departures are counted per warp in the counter's high half (4 kc
        // of them per tile); the last resets the counter for the next call.
        const uint32_t last_depart = (uint32_t)(4 * kc - 1);
        if (s0 == s1) {
          // nothing to sum here: arrive and depart (all four warps) at once
          if (et == 0 && !withhold &&
              (atom_add_acq_rel_gpu(cnt, 1u + 4 * SPLIT_DEPART) >> 16) == last_depart - 3u)
            *cnt = 0u;
        } else {
          if (et == 0) {
            if (!withhold) atom_add_acq_rel_gpu(cnt, 1u);
            const uint64_t t0 = globaltimer();
            while ((ld_relaxed_gpu(cnt) & 0xffffu) < (uint32_t)kc) {
              if (globaltimer() - t0 > tmo) {
                atomicExch(P.ws.status, STATUS_TIMEOUT);
                break;
              }
            }
            fence_acq_rel_gpu();
            if (tr_lead && nitem < 21) trace_put(trace, tr + 1, 6, nitem, globaltimer_ordered());
          }
          named_bar_sync(1, 128);
          // A warp departs as soon as it no longer reads the other
          // contributors' partials (its staged copies have landed), so the
          // atomic's round trip overlaps its sum.  Relaxed: within this
          // launch no slot of the tile is written again, and every warp
          // departs only after its CTA has seen all arrivals.
          uint32_t dep = 0;
          bool departed = false;
          auto depart = [&]() {
            if (lane == 0) dep = atom_add_relaxed_gpu(cnt, SPLIT_DEPART);
            departed = true;
          };
          if (nunit_w == 0) depart();
          if (nunit_w > 0) {
            const float alpha = get_alpha();
            // Adds this CTA's own partial of chunk ch (term jx of the sum)
            // to v, or starts v with it when it is the first term.
            auto add_own = [&](int ch, float (&v)[32]) {
              if (jx == 0) {
                tmem_ld32(tbase + ch * 32, v);
                return;
              }
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                float t8[8];
                tmem_ld8(tbase + ch * 32 + j * 8, t8);
#pragma unroll
                for (int e = 0; e < 8; ++e) v[8 * j + e] += t8[e];
              }
            };
            // v = q (first term) or v += q, q this warp's 4 KB block image
            auto add_block = [&](const float4 *blk, bool first, bool global, float (&v)[32]) {
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float4 q = global ? __ldcg(blk + j * 32 + lane) : blk[j * 32 + lane];
                if (first) {
                  v[4 * j] = q.x;
                  v[4 * j + 1] = q.y;
                  v[4 * j + 2] = q.z;
                  v[4 * j + 3] = q.w;
                } else {
                  v[4 * j] += q.x;
                  v[4 * j + 1] += q.y;
                  v[4 * j + 2] += q.z;
                  v[4 * j + 3] += q.w;
                }
              }
            };
            // The other kc - 1 partials: term ti (ascending unit, this
            // CTA's own unit skipped); piece i = (chunk i / nst of this
            // warp's chunks, term i % nst).
            const int nst = kc - 1;
            auto other = [&](int ti) { return o + ti + (ti >= jx ? 1 : 0); };
            auto chunk_of = [&](int k) { return ((s_first + 4 * (k / UW)) / 4) * UW + k % UW; };
            auto block_of = [&](int ch, int ti) {
              return slots + (int64_t)cslot(other(ti)) * SLOT_F4 + (ch * 4 + q4) * 256;
            };
            const int npieces = nunit_w * UW * nst;
            if (ring_free) {
              // Stage the pieces in this warp's share of the idle operand
              // ring (the ring split among the CTA's summing warps) with 4 KB
              // bulk copies, a group at a time on one barrier.
              constexpr int PIECE = 4096;
              const int nw = s1 - s0 < 4 ? s1 - s0 : 4;       // warps of this CTA that sum
              const int wq = (q4 - s0 % 4 + 4) % 4;            // this warp's place among them
              const int region = (stages * STAGE_BYTES / nw) / PIECE * PIECE;
              int nb = region / PIECE;
              if (nb > 32) nb = 32;                            // one copy per lane
              const uint32_t wbase = tiles_addr + (uint32_t)(wq * region);
              const float4 *wsmem = reinterpret_cast<const float4 *>(smem + wq * region);
              const uint32_t fb = smem_u32(fix_bar + q4);
              float v[32];
              int group = 0;
              bool okw = true;
              int kq = 0, ti = 0;   // chunk (of this warp's) and term of the next piece
              for (int g0 = 0; g0 < npieces && okw; g0 += nb, ++group) {
                const int gn = npieces - g0 < nb ? npieces - g0 : nb;
                __syncwarp();   // the previous group's images are consumed
                if (lane == 0) mbar_arrive_expect_tx(fb, (uint32_t)(gn * PIECE));
                __syncwarp();
                if (lane < gn) {
                  // one copy per lane (gn <= 32): the address arithmetic and
                  // the issue run in parallel
                  const int i = g0 + lane;
                  fence_proxy_async_global();   // the acquired partials, to the copy engine
                  bulk_copy_g2s(wbase + lane * PIECE, block_of(chunk_of(i / nst), i % nst), PIECE, fb);
                }
                if (tr_lead && group == 0) trace_put(trace, TRACE_FIX_BASE, 11, nitem, globaltimer_ordered());
                if (!__all_sync(0xffffffffu, mbar_wait(fb, (uint32_t)(group & 1), tmo))) {
                  if (lane == 0) fail();
                  okw = false;
                  break;
                }
                if (g0 + gn >= npieces) depart();   // every partial this warp needs is staged
                if (tr_lead && group == 0) trace_put(trace, TRACE_FIX_BASE + 2, 13, nitem, globaltimer_ordered());
                for (int bi = 0; bi < gn; ++bi) {
                  const int ch = chunk_of(kq);
                  if (ti == jx) add_own(ch, v);   // own term comes before this one
                  add_block(wsmem + bi * (PIECE / 16), ti == 0 && jx != 0, false, v);
                  if (ti == nst - 1) {
                    if (jx == kc - 1) add_own(ch, v);   // own term is the last
                    store_chunk(ch, v, alpha);
                    ti = 0;
                    ++kq;
                  } else {
                    ++ti;
                  }
                }
              }
            } else {
#pragma unroll 1
              for (int k = 0; k < nunit_w * UW; ++k) {
                const int ch = chunk_of(k);
                float v[32];
                for (int ti = 0; ti < nst; ++ti) {
                  if (ti == jx) add_own(ch, v);
                  add_block(block_of(ch, ti), ti == 0 && jx != 0, true, v);
                }
                if (jx == kc - 1) add_own(ch, v);
                store_chunk(ch, v, alpha);
              }
            }
            release_acc(acc);
          }
          if (tr_lead) trace_put(trace, TRACE_FIX_BASE + 3, 16, nitem, globaltimer_ordered());
          if (!departed) depart();   // plain-load sum done, or a staging wait failed
          if (lane == 0 && (dep >> 16) == last_depart) *cnt = 0u;
        }
        if (tr_lead && nitem < 21) trace_put(trace, tr + 2, 7, nitem, globaltimer_ordered());
      } else if (w.role == ROLE_PEER) {
        spill(slots + (int64_t)slot_id * SLOT_F4, no_skip);
        release_acc(acc);
        if (tr_lead) trace_put(trace, TRACE_FIX_BASE + 4, 14, nitem, globaltimer_ordered());   // spill issued
        __threadfence();
        if (tr_lead) trace_put(trace, TRACE_FIX_BASE + 5, 15, nitem, globaltimer_ordered());   // spill visible
        named_bar_sync(1, 128);
        if (!last_arriver) {
          if (et == 0 && !(P.debug_flags & DEBUG_SKIP_PEER_FLAG)) st_release_gpu(P.ws.flags + slot_id, 1u);
        } else {
          // Count this arrival at the tile's owner o; the contributor that
          // completes the count (pl - o earlier arrivals) sums the tile.
          const ProbSched &q = pss[w.problem];
          const int64_t ts = q.iter_base + (int64_t)w.tile * q.iters;
          o = unit_of_iter(S, ts);
          pl = unit_of_iter(S, ts + q.iters - 1);
          bool mine = false;
          if (et == 0) mine = atom_add_acq_rel_gpu(P.ws.flags + cslot(o), 1u) == (uint32_t)(pl - o);
          do_sum = broadcast(mine);
          own_tmem = false;
        }
      } else if (w.role == ROLE_OWNER) {
        if (!last_arriver) {
          // Poll every peer's flag with relaxed loads (they overlap), then
          // one acquire fence orders the partial reads after the peers'
          // release stores.
          if (et == 0) {
            const uint64_t t0 = globaltimer();
            for (;;) {
              bool all = true;
              for (int p = w.peer_first; p <= w.peer_last; ++p) all &= ld_relaxed_gpu(P.ws.flags + cslot(p)) != 0u;
              if (all) break;
              if (globaltimer() - t0 > tmo) {
                atomicExch(P.ws.status, STATUS_TIMEOUT);
                break;
              }
            }
            fence_acq_rel_gpu();
            if (tr_lead && nitem < 21) trace_put(trace, tr + 1, 6, nitem, globaltimer_ordered());
          }
          named_bar_sync(1, 128);
          do_sum = true;
        } else {
          // If every peer has already arrived, sum now from TMEM; otherwise
          // spill to the owner slot and count this arrival too.
          const uint32_t npeers = (uint32_t)(w.peer_last - w.peer_first + 1);
          bool mine = false;
          if (et == 0) {
            mine = ld_relaxed_gpu(P.ws.flags + slot_id) == npeers;
            if (mine) fence_acq_rel_gpu();
          }
          do_sum = broadcast(mine);
          if (!do_sum) {
            spill(oslots + (int64_t)slot_id * SLOT_F4, no_skip);
            __threadfence();
            named_bar_sync(1, 128);
            if (et == 0) mine = atom_add_acq_rel_gpu(P.ws.flags + slot_id, 1u) == npeers;
            do_sum = broadcast(mine);
          }
        }
      } else {
        const float alpha = get_alpha();
#pragma unroll 1
        for (int ch = 0; ch < BN / 32; ch += 2) {
          float v[64];
          tmem_ld64(tbase + ch * 32, v);
          store_chunk(ch, *reinterpret_cast<const float(*)[32]>(v), alpha);
          store_chunk(ch + 1, *reinterpret_cast<const float(*)[32]>(v + 32), alpha);
        }
      }
      if (do_sum) {
        if (own_tmem)
          fixup_sum(std::true_type{}, o, pl);
        else
          fixup_sum(std::false_type{}, o, pl);
        // Self-cleaning: the owner protocol clears the peers' flags, the
        // last-arriver protocol the tile's counter.
        if (et == 0) {
          if (!last_arriver)
            for (int p = w.peer_first; p <= w.peer_last; ++p) P.ws.flags[cslot(p)] = 0u;
          else
            P.ws.flags[cslot(o)] = 0u;
        }
      }
      if (!((XS || split_reduce) && (w.role == ROLE_PEER || w.role == ROLE_OWNER))) {
        if (w.role != ROLE_PEER) release_acc(acc);
        if (tr_lead && nitem < 21) trace_put(trace, tr + 2, 7, nitem, globaltimer_ordered());
      }
      ++nitem;
      if (++acc == NACC) {
        acc = 0;
        acc_phase ^= 1u;
      }
    }
    // Every TMA store of this warp must finish before the CTA exits.
    if (lane == 0) bulk_wait_group<0>();
    __syncwarp();
  }

  tc_fence_before();
  // Trace: each role's lead thread (producer 0, MMA issuer 1, epilogue 2)
  // stamps when its role is done; the CTA ends at the latest of these.
  // (A stamp taken right after a barrier can be read before the barrier
  // completes, so none is taken there.)
  if (DBG) {
    const int role_lead = threadIdx.x == 0 ? 0 : threadIdx.x == 32 ? 1 : threadIdx.x == 64 ? 2 : -1;
    if (role_lead >= 0) trace_put(trace, TRACE_CTA_BASE + 1 + role_lead, 8, role_lead, globaltimer_ordered());
  }
  cta_sync();
  // A pair's leader MMAs read the peer's shared memory and write its TMEM,
  // and XS partners write each other's shared memory: no CTA of a cluster
  // frees TMEM or exits before all are done.
  if constexpr (CLUSTER) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    if constexpr (PAIR)
      tmem_dealloc_pair(tmem_base, TMEM_COLS);
    else
      tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

template <int IN, typename OutT, int BN, int MAXP, bool PAIR, bool DBG, bool XS>
cudaError_t launch_tc_variant(const TcParams<MAXP> &p, int grid, cudaStream_t st) {
  auto kern = sk_tc_kernel<IN, OutT, BN, MAXP, PAIR, DBG, XS>;
  // CTAs per cluster: a pair, or, XS, the xs_k units of a tile
  const int cl = XS ? (PAIR ? 2 : 1) * p.xs_k : (PAIR ? 2 : 1);
  const int smem = tc_smem_bytes(PAIR ? BN / 2 : BN, p.stages, IN == IN_TF32X3);
  (void)cudaGetLastError();   // drop a stale error left by an earlier call on this thread
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (cl == 1) {
    kern<<<grid, 192, smem, st>>>(p);
    return cudaGetLastError();
  } else {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 0);
    (void)e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
  }
}

// Debug variants (timeline trace, coverage counts) exist for single-problem
// BF16 and 3xTF32 launches and for grouped BF16 launches with BF16 output;
// elsewhere both buffers are ignored.
template <int IN, typename OutT, int BN, int MAXP, bool PAIR>
constexpr bool has_debug_variant() {
  return (IN == IN_BF16 && (MAXP == 1 || std::is_same<OutT, __nv_bfloat16>::value)) ||
         (IN == IN_TF32X3 && MAXP == 1);
}

// Cluster-split variants (FIXUP_SPLIT_CLUSTER) exist for single-problem
// BF16 launches on 128 x 128 / 128 x 256 tiles and 256 x 256 pairs, and
// for single-problem 3xTF32 launches (128 x 128 tiles, 256 x 256 pairs).
template <int IN, typename OutT, int BN, int MAXP, bool PAIR>
constexpr bool has_xs_variant() {
  return (IN == IN_BF16 || IN == IN_TF32X3) && MAXP == 1 && (!PAIR || BN == 256);
}

template <int IN, typename OutT, int BN, int MAXP, bool PAIR>
cudaError_t launch_tc(const TcParams<MAXP> &p, int grid, cudaStream_t st) {
  if constexpr (has_xs_variant<IN, OutT, BN, MAXP, PAIR>()) {
    if (p.fixup == FIXUP_SPLIT_CLUSTER)
      return (p.trace || p.cover) ? launch_tc_variant<IN, OutT, BN, MAXP, PAIR, true, true>(p, grid, st)
                                  : launch_tc_variant<IN, OutT, BN, MAXP, PAIR, false, true>(p, grid, st);
  }
  if (p.fixup == FIXUP_SPLIT_CLUSTER) return cudaErrorNotSupported;
  if constexpr (has_debug_variant<IN, OutT, BN, MAXP, PAIR>()) {
    if (p.trace || p.cover) return launch_tc_variant<IN, OutT, BN, MAXP, PAIR, true, false>(p, grid, st);
  }
  return launch_tc_variant<IN, OutT, BN, MAXP, PAIR, false, false>(p, grid, st);
}

// Co-resident clusters of the kernel (0 if it cannot launch): CTA pairs
// (xs = false), or, for the cluster split (xs = true), clusters of two
// units -- four CTAs for pairs, two single CTAs otherwise.
template <int IN, typename OutT, int BN, int MAXP, bool PAIR>
int tc_max_clusters(int stages, bool xs, int xs_k = 2) {
  constexpr bool XS_OK = has_xs_variant<IN, OutT, BN, MAXP, PAIR>();
  if (xs && !XS_OK) return 0;
  if (!xs && !PAIR) return 0;
  auto kern = xs ? sk_tc_kernel<IN, OutT, BN, MAXP, PAIR, false, XS_OK>
                 : sk_tc_kernel<IN, OutT, BN, MAXP, PAIR, false, false>;
  const int cl = xs ? (PAIR ? 2 : 1) * xs_k : 2;
  const int smem = tc_smem_bytes(PAIR ? BN / 2 : BN, stages, IN == IN_TF32X3);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cl, 1, 1);
  cfg.blockDim = dim3(192, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return n;
}

template <int IN, typename OutT, int BN, int MAXP>
int pair_max_clusters(int stages) {
  return tc_max_clusters<IN, OutT, BN, MAXP, true>(stages, false);
}

template <int IN, typename OutT, int BN, bool PAIR>
int xs_max_clusters(int stages, int xs_k) {
  return tc_max_clusters<IN, OutT, BN, 1, PAIR>(stages, true, xs_k);
}

}  // namespace sk

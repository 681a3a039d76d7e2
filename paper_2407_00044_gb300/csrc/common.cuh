// Kernel parameter blocks and launch declarations shared by the C-ABI layer
// and the kernel translation units.
#pragma once
#include <cuda.h>          // CUtensorMap (type only; the driver is reached at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include "sched.cuh"

namespace sk {

// Problems a grouped launch carries inline in its kernel parameter block;
// larger groups (up to MAX_PROBLEMS) keep their problem table in the
// caller's workspace (TcParams::gprob / SimtParams::gprob).
constexpr int MAXP_GROUPED = 64;
constexpr int MAX_PROBLEMS = 1 << 16;
constexpr uint32_t STATUS_TIMEOUT = 4;  // == SK_ERR_TIMEOUT

// Device views of the caller's workspace.
struct Workspace {
  float *partials;        // g slots of tile_m * tile_n floats (a unit's peer segment)
  uint32_t *flags;        // g flags (owner fixup) or arrival counters (last-arriver
                          // fixup, indexed by the owner's slot), zero between calls
  uint32_t *status;       // 0, or STATUS_TIMEOUT after an expired wait
  float *owner_partials;  // last-arriver fixup: g more slots (a unit's owner segment)
};

// Workspace layout: [status word, padded to 256 B][WS_MAX_CTAS flag words]
// [per-CTA partial slots].  The flag region has a fixed size so that calls
// with different CTA counts sharing one workspace never find another call's
// partials where their flags are (flags must read zero between calls).
constexpr int WS_MAX_CTAS = 1024;
constexpr size_t WS_FLAG_OFFSET = 256;
constexpr size_t WS_FLAG_BYTES = (size_t)WS_MAX_CTAS * 4;

// Fixup protocols (sk_fixup).
constexpr int32_t FIXUP_OWNER = 0, FIXUP_LAST_ARRIVER = 1, FIXUP_SPLIT = 2, FIXUP_SPLIT_CLUSTER = 3;
// Split reduce: one counter word per tile (at the owner's flag) counts
// arrivals in its low half and departures in its high half.
constexpr uint32_t SPLIT_DEPART = 1u << 16;

// ----------------------------------------------------------- FP32 SIMT path
constexpr int F32_BM = 128, F32_BN = 128, F32_BK = 16, F32_THREADS = 256;

struct SimtProblem {
  const float *A, *B, *C_in;
  float *C;
  int64_t a_rs, a_cs;   // A(i,k) = A[i*a_rs + k*a_cs]
  int64_t b_rs, b_cs;   // B(k,j) = B[k*b_rs + j*b_cs]
  int64_t ldc;          // C row-major (C_in shares it)
  int32_t M, N, K;
  float alpha, beta;
  int32_t a_kmajor;     // a_cs == 1
  int32_t b_kmajor;     // b_rs == 1
  int32_t a_vec, b_vec, c_vec;   // 16-byte vector access legal
};

// debug_flags bit 0: peers do not raise their flags (test-only; makes every
// owner's bounded wait expire).
constexpr int32_t DEBUG_SKIP_PEER_FLAG = 1;

template <int MAXP>
struct SimtParams {
  Sched sched;
  ProbSched ps[MAXP];
  SimtProblem prob[MAXP];
  // Groups of more than MAXP problems: the tables in global memory (the
  // inline arrays are then unused); null otherwise.
  const SimtProblem *gprob;
  const ProbSched *gps;
  Workspace ws;
  uint64_t timeout_ns;
  int32_t debug_flags;
  int32_t fixup;
};

// --------------------------------------------------------- tcgen05 path
// IN_TF32X3: FP32 operands on the tensor cores as three TF32 products
// (a_hi b_hi + a_hi b_lo + a_lo b_hi, x = x_hi + x_lo split in the kernel).
enum InKind : int { IN_BF16 = 0, IN_E4M3 = 1, IN_TF32X3 = 2 };

struct TcProblem {
  CUtensorMap tmap_a;   // K-major: box {BK, 128}; MN-major: box {64, BK}
  CUtensorMap tmap_b;   // K-major: box {BK, BN};  MN-major: box {64, BK}
  int32_t c_tma;        // epilogue writes C with TMA stores via TcParams::tmap_c
  int32_t pad_;
  void *C;
  const void *C_in;
  int64_t ldc;          // C row-major
  int32_t M, N, K;
  float alpha, beta;
  int32_t a_mn, b_mn;   // operand stored MN-major (transposed) in memory
  int32_t c_vec;        // 16-byte vector stores legal for C / C_in
  const float *scale_a, *scale_b;   // E4M3 per-tensor scales (may be null)
};

// The C tensor map serves single-problem launches only (c_tma is never set
// in grouped ones): 64 more maps would exceed the 32 KB parameter limit.
template <int MAXP>
struct TcParams {
  TcProblem prob[MAXP];
  CUtensorMap tmap_c[1];   // C of problem 0 (row-major, box {128 B of columns, 32 rows}, 128B swizzle)
  ProbSched ps[MAXP];
  // Groups of more than MAXP problems: the tables in global memory (the
  // inline arrays are then unused; the tensor maps were written there by
  // launch_upload and are acquired by the tensormap proxy before use).
  const TcProblem *gprob;
  const ProbSched *gps;
  Sched sched;
  Workspace ws;
  uint64_t timeout_ns;
  int32_t stages;
  int32_t debug_flags;
  uint64_t *trace;      // optional per-CTA timeline (SK_TRACE_* in skgemm.h)
  uint32_t *cover;      // optional coverage counts (SK_COVERAGE in skgemm.h)
  int64_t cover_iters;  // MAC-loop iterations of all problems: the first block-store word
  int32_t fixup;
  int32_t xs_k;         // FIXUP_SPLIT_CLUSTER: units per tile (= per cluster), 2, 4 or 8
};

// Cluster split: most units a contributor sums (NS / k with NS <= 32 and
// k >= 2), one data barrier each.
constexpr int XS_MAX_UNITS = 16;

// Coverage word increment of one visit by unit u (SK_COVERAGE_VISIT).
__host__ __device__ __forceinline__ uint32_t cover_visit(int u) { return 1u + ((uint32_t)(u + 1) << 8); }

constexpr int TRACE_ENTRIES = 128;
constexpr int TRACE_MMA_BASE = 0, TRACE_EPI_BASE = 48, TRACE_CTA_BASE = 112, TRACE_FIX_BASE = 116,
              TRACE_ENTRY = 122;

__device__ __forceinline__ void trace_put(uint64_t *trace, int entry, uint32_t ev, uint32_t item, uint64_t t) {
  if (trace && entry >= 0 && entry < TRACE_ENTRIES) {
    uint64_t *e = trace + ((uint64_t)blockIdx.x * TRACE_ENTRIES + entry) * 2;
    e[0] = ((uint64_t)ev << 32) | item;
    e[1] = t;
  }
}

// Bytes of dynamic shared memory of a tcgen05 launch.  Never less than
// 120 KB, so two CTAs can never share an SM: each CTA holds up to all 512
// TMEM columns, and an owner CTA waits on peer CTAs, so a peer stuck in
// tcgen05.alloc behind its owner on the same SM would stall until timeout.
// Epilogue staging for TMA stores of C: per epilogue warp two 4 KB buffers
// (32 rows x 128 bytes, 128-byte swizzled).
constexpr int EPI_STAGE_BYTES = 4 * 2 * 4096;

// (split_in: the 3xTF32 kernel keeps a low-part copy of every stage)
inline int tc_smem_bytes(int bn, int stages, bool split_in = false) {
  const int stage = (128 * 128 + bn * 128) * (split_in ? 2 : 1);
  const int need = 1024 /*alignment slack*/ + stages * stage + EPI_STAGE_BYTES + 512 /*barriers, TMEM slot*/;
  return need < 120 * 1024 ? 120 * 1024 : need;
}

// Owner fixup staged in shared memory: 16 KB units (one 32-column chunk of
// one peer's partial), at most FIX_SMEM_UNITS in flight.
constexpr int FIX_UNIT_BYTES = 128 * 32 * 4;
constexpr int FIX_SMEM_UNITS = 12;

template <int MAXP>
cudaError_t launch_simt_f32(const SimtParams<MAXP> &p, int grid, cudaStream_t st);

template <int IN, typename OutT, int BN, int MAXP, bool PAIR>
cudaError_t launch_tc(const TcParams<MAXP> &p, int grid, cudaStream_t st);

template <int IN, typename OutT, int BN, int MAXP>
int pair_max_clusters(int stages);

// Co-resident clusters of the cluster-split kernel (FIXUP_SPLIT_CLUSTER,
// single problem): xs_k units (CTAs or CTA pairs) per cluster.
template <int IN, typename OutT, int BN, bool PAIR>
int xs_max_clusters(int stages, int xs_k);

cudaError_t launch_scale(void *C, const void *C_in, int64_t ldc, int64_t M, int64_t N,
                         float beta, int c_is_f32, cudaStream_t st);

// Copies `bytes` (a multiple of 16) of host memory to the device address
// `dst` (16-byte aligned) with kernels that carry the bytes in their
// parameter blocks (UPLOAD_CHUNK_BYTES per launch): ordered on the stream,
// nothing allocated, and a captured CUDA graph keeps its own copy of the
// bytes.  Tensor maps among them are released to the tensormap proxy.
constexpr int UPLOAD_CHUNK_BYTES = 30720;
cudaError_t launch_upload(void *dst, const void *src, size_t bytes, cudaStream_t st);

cudaError_t launch_quant_e4m3(const float *x, int64_t n, uint8_t *q, float *scale_out,
                              float *amax_work, cudaStream_t st);

}  // namespace sk

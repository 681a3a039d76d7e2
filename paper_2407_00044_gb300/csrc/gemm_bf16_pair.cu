// BF16-input instantiations of the CTA-pair (256-row tile) Stream-K kernel
// (single problem; the grouped ones are in gemm_bf16_pair_grouped.cu).
#include "gemm_tc.cuh"

namespace sk {
template cudaError_t launch_tc<IN_BF16, __nv_bfloat16, 256, 1, true>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_BF16, float, 256, 1, true>(const TcParams<1> &, int, cudaStream_t);
template int pair_max_clusters<IN_BF16, __nv_bfloat16, 256, 1>(int);
template int pair_max_clusters<IN_BF16, float, 256, 1>(int);
// 256 x 128 pair tiles (each CTA loads 128 rows of A and 64 rows of B)
template cudaError_t launch_tc<IN_BF16, __nv_bfloat16, 128, 1, true>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_BF16, float, 128, 1, true>(const TcParams<1> &, int, cudaStream_t);
template int pair_max_clusters<IN_BF16, __nv_bfloat16, 128, 1>(int);
template int pair_max_clusters<IN_BF16, float, 128, 1>(int);
}  // namespace sk

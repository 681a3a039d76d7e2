// BF16-input instantiations of the CTA-pair Stream-K kernel with 256 x 256
// tiles (single problem; the grouped ones are in gemm_bf16_pair_grouped.cu,
// the 256 x 128 pairs in gemm_bf16_pair128.cu).
#include "gemm_tc.cuh"

namespace sk {
template cudaError_t launch_tc<IN_BF16, __nv_bfloat16, 256, 1, true>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_BF16, float, 256, 1, true>(const TcParams<1> &, int, cudaStream_t);
template int pair_max_clusters<IN_BF16, __nv_bfloat16, 256, 1>(int);
template int pair_max_clusters<IN_BF16, float, 256, 1>(int);
template int xs_max_clusters<IN_BF16, __nv_bfloat16, 256, true>(int, int);
template int xs_max_clusters<IN_BF16, float, 256, true>(int, int);
}  // namespace sk

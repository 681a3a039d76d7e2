// BF16-input instantiations of the CTA-pair Stream-K kernel with 256 x 512
// tiles (two N = 256 MMAs per k-step into one 512-column accumulator;
// single problem).
#include "gemm_tc.cuh"

namespace sk {
template cudaError_t launch_tc<IN_BF16, __nv_bfloat16, 512, 1, true>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_BF16, float, 512, 1, true>(const TcParams<1> &, int, cudaStream_t);
template int pair_max_clusters<IN_BF16, __nv_bfloat16, 512, 1>(int);
template int pair_max_clusters<IN_BF16, float, 512, 1>(int);
}  // namespace sk

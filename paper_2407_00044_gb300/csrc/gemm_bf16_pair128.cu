// BF16-input instantiations of the CTA-pair Stream-K kernel with 256 x 128
// tiles (each CTA loads 128 rows of A and 64 rows of B; single problem).
#include "gemm_tc.cuh"

namespace sk {
template cudaError_t launch_tc<IN_BF16, __nv_bfloat16, 128, 1, true>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_BF16, float, 128, 1, true>(const TcParams<1> &, int, cudaStream_t);
template int pair_max_clusters<IN_BF16, __nv_bfloat16, 128, 1>(int);
template int pair_max_clusters<IN_BF16, float, 128, 1>(int);
}  // namespace sk

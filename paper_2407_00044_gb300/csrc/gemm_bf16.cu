// BF16-input, BF16-output instantiations of the tcgen05 Stream-K kernel
// (single problem, one CTA per unit).
#include "gemm_tc.cuh"

namespace sk {
template cudaError_t launch_tc<IN_BF16, __nv_bfloat16, 256, 1, false>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_BF16, __nv_bfloat16, 128, 1, false>(const TcParams<1> &, int, cudaStream_t);
template int xs_max_clusters<IN_BF16, __nv_bfloat16, 256, false>(int, int);
template int xs_max_clusters<IN_BF16, __nv_bfloat16, 128, false>(int, int);
}  // namespace sk

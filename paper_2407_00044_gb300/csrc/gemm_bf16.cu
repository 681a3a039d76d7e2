// BF16-input instantiations of the tcgen05 Stream-K kernel (single problem).
#include "gemm_tc.cuh"

namespace sk {
template cudaError_t launch_tc<IN_BF16, __nv_bfloat16, 256, 1, false>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_BF16, __nv_bfloat16, 128, 1, false>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_BF16, float, 256, 1, false>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_BF16, float, 128, 1, false>(const TcParams<1> &, int, cudaStream_t);
}  // namespace sk

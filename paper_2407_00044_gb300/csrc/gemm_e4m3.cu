// FP8 E4M3-input instantiations of the tcgen05 Stream-K kernel.
#include "gemm_tc.cuh"

namespace sk {
template cudaError_t launch_tc<IN_E4M3, __nv_bfloat16, 256, 1, false>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_E4M3, __nv_bfloat16, 128, 1, false>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_E4M3, float, 256, 1, false>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_E4M3, float, 128, 1, false>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_E4M3, __nv_bfloat16, 256, 1, true>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_E4M3, float, 256, 1, true>(const TcParams<1> &, int, cudaStream_t);
template int pair_max_clusters<IN_E4M3, __nv_bfloat16, 256, 1>(int);
template int pair_max_clusters<IN_E4M3, float, 256, 1>(int);
}  // namespace sk

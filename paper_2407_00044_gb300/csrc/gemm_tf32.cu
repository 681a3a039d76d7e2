// FP32-input instantiations of the tcgen05 Stream-K kernel (3xTF32).
#include "gemm_tc.cuh"

namespace sk {
template cudaError_t launch_tc<IN_TF32X3, float, 128, 1, false>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_TF32X3, float, 128, MAXP_GROUPED, false>(const TcParams<MAXP_GROUPED> &, int,
                                                                           cudaStream_t);
// 256 x 256 tiles on CTA pairs
template cudaError_t launch_tc<IN_TF32X3, float, 256, 1, true>(const TcParams<1> &, int, cudaStream_t);
template cudaError_t launch_tc<IN_TF32X3, float, 256, MAXP_GROUPED, true>(const TcParams<MAXP_GROUPED> &, int,
                                                                          cudaStream_t);
template int pair_max_clusters<IN_TF32X3, float, 256, 1>(int);
template int xs_max_clusters<IN_TF32X3, float, 256, true>(int, int);
template int xs_max_clusters<IN_TF32X3, float, 128, false>(int, int);
template int pair_max_clusters<IN_TF32X3, float, 256, MAXP_GROUPED>(int);
}  // namespace sk

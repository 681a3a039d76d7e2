// BF16-input instantiations of the tcgen05 Stream-K kernel for grouped
// launches (up to MAXP_GROUPED problems; also used by the backward pass).
#include "gemm_tc.cuh"

namespace sk {
template cudaError_t launch_tc<IN_BF16, __nv_bfloat16, 256, MAXP_GROUPED, false>(const TcParams<MAXP_GROUPED> &, int,
                                                                                cudaStream_t);
template cudaError_t launch_tc<IN_BF16, __nv_bfloat16, 128, MAXP_GROUPED, false>(const TcParams<MAXP_GROUPED> &, int,
                                                                                cudaStream_t);
template cudaError_t launch_tc<IN_BF16, float, 256, MAXP_GROUPED, false>(const TcParams<MAXP_GROUPED> &, int,
                                                                        cudaStream_t);
template cudaError_t launch_tc<IN_BF16, float, 128, MAXP_GROUPED, false>(const TcParams<MAXP_GROUPED> &, int,
                                                                        cudaStream_t);
}  // namespace sk

// BF16-input instantiations of the CTA-pair (256-row tile) Stream-K kernel
// for grouped launches (up to MAXP_GROUPED problems inline; also used by the
// backward pass).
#include "gemm_tc.cuh"

namespace sk {
template cudaError_t launch_tc<IN_BF16, __nv_bfloat16, 256, MAXP_GROUPED, true>(const TcParams<MAXP_GROUPED> &, int,
                                                                               cudaStream_t);
template cudaError_t launch_tc<IN_BF16, float, 256, MAXP_GROUPED, true>(const TcParams<MAXP_GROUPED> &, int,
                                                                       cudaStream_t);
template int pair_max_clusters<IN_BF16, __nv_bfloat16, 256, MAXP_GROUPED>(int);
template int pair_max_clusters<IN_BF16, float, 256, MAXP_GROUPED>(int);
// 256 x 128 pair tiles
template cudaError_t launch_tc<IN_BF16, __nv_bfloat16, 128, MAXP_GROUPED, true>(const TcParams<MAXP_GROUPED> &, int,
                                                                               cudaStream_t);
template cudaError_t launch_tc<IN_BF16, float, 128, MAXP_GROUPED, true>(const TcParams<MAXP_GROUPED> &, int,
                                                                       cudaStream_t);
template int pair_max_clusters<IN_BF16, __nv_bfloat16, 128, MAXP_GROUPED>(int);
template int pair_max_clusters<IN_BF16, float, 128, MAXP_GROUPED>(int);
}  // namespace sk

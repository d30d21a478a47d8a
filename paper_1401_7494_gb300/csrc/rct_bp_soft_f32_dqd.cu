// Software-bilinear backprojection kernels: F32 projections, dqd route (difference quads) (see rct_bp_kernel.cuh).
#include "rct_bp_kernel.cuh"

namespace rct {

cudaError_t launch_bp_soft_f32_dqd(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    return dispatch_xv<G_SOFT, DT_F32, ROUTE_DQD>(c, p, s);
}

}  // namespace rct

// Software-bilinear backprojection kernels: F32 projections, qld route (see rct_bp_kernel.cuh).
#include "rct_bp_kernel.cuh"

namespace rct {

cudaError_t launch_bp_soft_f32_qld(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    return dispatch_xv<G_SOFT, DT_F32, ROUTE_QLD>(c, p, s);
}

}  // namespace rct

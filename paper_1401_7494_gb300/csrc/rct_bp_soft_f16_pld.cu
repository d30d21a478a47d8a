// Software-bilinear backprojection kernels: F16 projections, pld route (see rct_bp_kernel.cuh).
#include "rct_bp_kernel.cuh"

namespace rct {

cudaError_t launch_bp_soft_f16_pld(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    return dispatch_xv<G_SOFT, DT_F16, ROUTE_PLD>(c, p, s);
}

}  // namespace rct

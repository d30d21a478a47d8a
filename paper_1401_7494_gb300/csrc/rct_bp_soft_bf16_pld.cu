// Software-bilinear backprojection kernels: BF16 projections, pld route (see rct_bp_kernel.cuh).
#include "rct_bp_kernel.cuh"

namespace rct {

cudaError_t launch_bp_soft_bf16_pld(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    return dispatch_xv<G_SOFT, DT_BF16, ROUTE_PLD>(c, p, s);
}

}  // namespace rct

// Software-bilinear backprojection kernels: BF16 projections, qld route (see rct_bp_kernel.cuh).
#include "rct_bp_kernel.cuh"

namespace rct {

cudaError_t launch_bp_soft_bf16_qld(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    return dispatch_xv<G_SOFT, DT_BF16, ROUTE_QLD>(c, p, s);
}

}  // namespace rct

// Software-bilinear backprojection kernels with Listing 1's truncating cell index: F32 projections,
// ldg route (see rct_bp_kernel.cuh).
#include "rct_bp_kernel.cuh"

namespace rct {

cudaError_t launch_bp_soft_f32_trunc(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    return dispatch_trunc(c, p, s);
}

}  // namespace rct

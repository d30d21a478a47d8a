// Backprojection kernels that gather the four taps with predicated read-only loads
// straight from the caller's linear projection images (no staging copy).
#include "rct_bp_kernel.cuh"

namespace rct {

cudaError_t launch_bp_ldg(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    switch (c.dtype) {
        case DT_F32: return dispatch_xv<G_LDG, DT_F32>(c, p, s);
        case DT_F16: return dispatch_xv<G_LDG, DT_F16>(c, p, s);
        case DT_BF16: return dispatch_xv<G_LDG, DT_BF16>(c, p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rct

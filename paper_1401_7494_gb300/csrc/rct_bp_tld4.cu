// Backprojection kernels that fetch the 2x2 cell with one texture gather (tld4) from
// projections staged into gather-capable 2D CUDA arrays with a zero border.
#include "rct_bp_kernel.cuh"

namespace rct {

cudaError_t launch_bp_tld4(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    switch (c.dtype) {
        case DT_F32: return dispatch_xv<G_TLD4, DT_F32>(c, p, s);
        case DT_F16: return dispatch_xv<G_TLD4, DT_F16>(c, p, s);
        case DT_BF16: return dispatch_xv<G_TLD4, DT_BF16>(c, p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rct

// Backprojection kernels that let the texture unit interpolate (hardware bilinear,
// fixed-point weights).  The texture holds FP32 or FP16 values; the element type of
// the staged array does not change the kernel.
#include "rct_bp_kernel.cuh"

namespace rct {

cudaError_t launch_bp_texlin(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    return dispatch_xv<G_TEXLIN, DT_F32, ROUTE_TEX>(c, p, s);
}

}  // namespace rct

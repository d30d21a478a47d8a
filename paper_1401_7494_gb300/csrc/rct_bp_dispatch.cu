// Route selection for the software-bilinear kernels: the run-time split tex_zrun and the quad flag
// pick a kernel compiled for that route (all texture, all plain loads, all quad loads, or texture
// mixed with quad loads), so the single-route kernels carry no branch on the route.
#include "rct_internal.h"

namespace rct {

#define RCT_DECLARE_ROUTES(dt)                                                               \
    cudaError_t launch_bp_soft_##dt##_tex(const LaunchConfig &, const BpParams &, cudaStream_t); \
    cudaError_t launch_bp_soft_##dt##_ldg(const LaunchConfig &, const BpParams &, cudaStream_t); \
    cudaError_t launch_bp_soft_##dt##_qld(const LaunchConfig &, const BpParams &, cudaStream_t); \
    cudaError_t launch_bp_soft_##dt##_pld(const LaunchConfig &, const BpParams &, cudaStream_t); \
    cudaError_t launch_bp_soft_##dt##_mix(const LaunchConfig &, const BpParams &, cudaStream_t);
RCT_DECLARE_ROUTES(f32)
cudaError_t launch_bp_soft_f32_dqd(const LaunchConfig &, const BpParams &, cudaStream_t);
RCT_DECLARE_ROUTES(f16)
RCT_DECLARE_ROUTES(bf16)
#undef RCT_DECLARE_ROUTES

#define RCT_ROUTE_SWITCH(dt)                                                                      \
    if (p.tex_zrun <= 0) {                                                                        \
        if (p.quad == 2) return launch_bp_soft_##dt##_pld(c, p, s);                               \
        return p.quad ? launch_bp_soft_##dt##_qld(c, p, s) : launch_bp_soft_##dt##_ldg(c, p, s);  \
    }                                                                                             \
    if (p.tex_zrun < c.zrun) return launch_bp_soft_##dt##_mix(c, p, s);                           \
    return launch_bp_soft_##dt##_tex(c, p, s);

cudaError_t launch_bp_soft_f32(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    if (p.tex_zrun <= 0 && p.quad == 3) return launch_bp_soft_f32_dqd(c, p, s);
    RCT_ROUTE_SWITCH(f32)
}
cudaError_t launch_bp_soft_f16(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    if (p.quad == 3) return cudaErrorInvalidValue;   // difference quads hold FP32 values
    RCT_ROUTE_SWITCH(f16)
}
cudaError_t launch_bp_soft_bf16(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    if (p.quad == 3) return cudaErrorInvalidValue;
    RCT_ROUTE_SWITCH(bf16)
}

}  // namespace rct

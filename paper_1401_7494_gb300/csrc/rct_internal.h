// Internal interface between the C-ABI layer (rct_api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/rct.h"

namespace rct {

constexpr int KMAX = 32;  // views per pass held in the launch parameters

// G_SOFT: software bilinear; per z position of a run the 2x2 cell comes from a texture gather or
// from predicated global loads (BpParams::tex_zrun).  G_TEXLIN: texture-unit bilinear.
enum Gather : int { G_SOFT = 1, G_TEXLIN = 3 };
enum DType : int { DT_F32 = 0, DT_F16 = 1, DT_BF16 = 2 };

// One view as the kernel sees it.  The host folds the voxel origin, spacing
// and the volume centre into the matrix in FP64 (the paper's O and MM), so
// that for centred voxel coordinates (xc, yc, zc) = (x, y, z) - (L-1)/2
//     (u', v', w) = m * (xc, yc, zc, 1)
// and the detector position is (cu + u'/w, cv + v'/w).  Subtracting the
// integer pixel shift (cu, cv) -- the pixel nearest to where the volume
// centre projects -- keeps u' and v' small, so FP32 rounding of the
// coordinates stays close to one rounding of the final pixel position.
struct ViewParams {
    float m[12];               // row-major rows u', v', w
    int cu, cv;                // integer detector shift (0 for texture-filtered sampling)
    unsigned long long tex;    // cudaTextureObject_t (TLD4, TEXLIN)
    const void *img;           // linear image, H x W, row-major (LDG)
};

struct BpParams {
    float *vol;      // L^3, z-major, x fastest
    int L, W, H;
    int K;           // views in this pass, 1..KMAX
    float cen;       // (L - 1) / 2
    int accumulate;  // 0: the volume is logically zero, overwrite instead of adding
    int tex_zrun;    // G_SOFT: z positions [0, tex_zrun) of each run use the texture gather
    ViewParams view[KMAX];
};

struct LaunchConfig {
    int gather;  // Gather
    int dtype;   // DType of the stored projections
    int xv;      // voxels per thread along x: 1, 2, 4
    int zrun;    // voxels per thread along z: 1, 2, 4, 8
    int bx, by;  // block shape
};

// Kernel launchers (one translation unit per gather kind).
cudaError_t launch_bp_soft_f32(const LaunchConfig &c, const BpParams &p, cudaStream_t s);
cudaError_t launch_bp_soft_f16(const LaunchConfig &c, const BpParams &p, cudaStream_t s);
cudaError_t launch_bp_soft_bf16(const LaunchConfig &c, const BpParams &p, cudaStream_t s);
cudaError_t launch_bp_texlin(const LaunchConfig &c, const BpParams &p, cudaStream_t s);

cudaError_t launch_convert(const float *src, void *dst, size_t n, int dtype, cudaStream_t s);

// Record a message for rct_last_error() on the calling thread and return `code`.
rct_status rct_internal_fail(rct_status code, const char *fmt, ...);
cudaError_t launch_widen_bf16(const uint16_t *src, float *dst, size_t n, cudaStream_t s);

}  // namespace rct

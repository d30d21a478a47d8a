// Internal interface between the C-ABI layer (rct_api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/rct.h"

namespace rct {

constexpr int KMAX = 32;  // views per pass held in the launch parameters

// G_SOFT: software bilinear; per z position of a run the 2x2 cell comes from a texture gather
// (z positions [0, tex_zrun)) or from loads (the rest): four predicated loads from the caller's
// linear image, or, when BpParams::quad is set, one load of a staged quad element holding the
// whole cell.  G_TEXLIN: texture-unit bilinear.
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
//
// ViewGeo (device memory, one per view of the context, uploaded by rct_set_geometry) holds the
// same matrix split into FP32 high parts and the FP32 rounding of the remainders (low parts).
// With it, the first warp of a block evaluates the block corner's (u', v', w) for each view of
// the pass in double-float arithmetic, picks a block-local integer shift, and the block's
// threads then work with short local offsets, so the FP32 pixel coordinate is accurate to a
// few units in the last place of a short local distance wherever the block sits on the detector.
struct ViewParams {
    float muv[8];              // rows u', v' interleaved: (m0, m4), (m1, m5), (m2, m6), (m3, m7)
    float mw[4];               // row w
    int cu, cv;                // integer detector shift of the fold (0 for texture-filtered sampling)
    unsigned long long tex;    // cudaTextureObject_t (gather or filtered texture)
    const void *img;           // linear image, H x W, row-major (plain loads)
    const void *quad;          // staged quad or pair image, zero padded (quad / pair loads)
};

struct __align__(16) ViewGeo {
    float hu[8], lu[8];        // rows u', v' interleaved as in ViewParams: high and low parts
    float hw[4], lw[4];        // row w: high and low parts
    int cu, cv;
    int pad_[2];
};

// A quad element at padded (row jy, column ix) holds the cell with corner (i0, j0) =
// (ix - 1, jy - 1) in the order (I[j0][i0], I[j0+1][i0], I[j0][i0+1], I[j0+1][i0+1]), zero where
// a tap lies off the image; the quad image has H + 1 rows of W + 1 elements (16 bytes FP32,
// 8 bytes FP16/BF16).  A pair element at padded (row jy, column ix) holds the vertical pair
// (I[jy-1][ix-1], I[jy][ix-1]); the pair image has H + 1 rows of W + 2 pairs (8 bytes FP32,
// 4 bytes FP16/BF16), and the cell with corner (i0, j0) is the two consecutive pairs at
// (j0 + 1, i0 + 1) and (j0 + 1, i0 + 2).  A difference quad (FP32 only) is laid out as a quad
// element, H + 1 rows of W + 1 elements of 16 bytes, but holds (I[j0][i0], I[j0+1][i0],
// I[j0][i0+1] - I[j0][i0], I[j0+1][i0+1] - I[j0+1][i0]), the differences rounded to FP32: the
// horizontal lerps of both rows are then one packed FMA, with the very roundings the quad and pair
// routes perform in the kernel.  A cell with a tap on the image has its padded index in
// [0, W] x [0, H]; a kernel tests that and sends every other lane to element 0.

struct BpParams {
    float *vol;      // L^3, z-major, x fastest: the address of plane 0 (for a slab context, which holds
                     // planes [z_first, z_first + z_count) only, an address z_first planes before its buffer;
                     // no plane outside the slab is touched)
    int L, W, H;
    int K;           // views in this pass, 1..KMAX
    float cen;       // (L - 1) / 2
    int accumulate;  // 0: the volume is logically zero, overwrite instead of adding
    int tex_zrun;    // G_SOFT: z positions [0, tex_zrun) of each run use the texture gather
    int quad;        // G_SOFT load route: 0 = linear image, 1 = staged quads, 2 = staged pairs,
                     // 3 = staged difference quads
    const ViewGeo *geo;  // G_SOFT: the context's per-view geometry for block frames (null: global frame)
    int first_view;      // view index of view[0] in geo
    int z_base;          // first z plane of this launch (0: the whole volume)
    int z_count;         // z planes from z_base (0: all L); a multiple of the z-run unless it ends at L
    long long qelems;    // elements of one staged quad / pair image (bounds-checking build only)
#ifdef RCT_CHECK_BOUNDS
    int vol_z0;          // bounds-checking build: first plane the volume buffer holds
    long long vol_elems; // bounds-checking build: floats the volume buffer holds
#endif
    unsigned long long *viol;  // bounds-checking build: violation counter on the device (null: not counted)
    ViewParams view[KMAX];
    // View split (kernels compiled with SPLIT only): the pass's views are dealt out in contiguous groups of
    // split_views to `splits` groups of blocks; group 0 adds into vol, group s > 0 into the partial volume
    // part + (s - 1) * part_stride (addressed like vol), written when accumulate_part is 0.  blockIdx.z =
    // group * split_runs + z-run.  The partials are added into vol after the call's last pass.
    float *part;
    long long part_stride;
    int split_runs;
    int split_views;
    int accumulate_part;
};

struct LaunchConfig {
    int gather;  // Gather
    int dtype;   // DType of the stored projections
    int xv;      // voxels per thread along x: 1, 2, 4
    int zrun;    // voxels per thread along z: 1, 2, 4, 8
    int bx, by;  // block shape
    int frame;   // 1: block frames (FP32 software gathers only; BpParams::geo set)
    int trunc;   // 1: Listing 1's truncating cell index (FP32, plain loads, global frame)
    int split;   // groups of the view split (1: none; global frame, floor rule, software gathers only)
};

// Kernel launchers (one translation unit per gather kind).
cudaError_t launch_bp_soft_f32(const LaunchConfig &c, const BpParams &p, cudaStream_t s);
cudaError_t launch_bp_soft_f16(const LaunchConfig &c, const BpParams &p, cudaStream_t s);
cudaError_t launch_bp_soft_bf16(const LaunchConfig &c, const BpParams &p, cudaStream_t s);
cudaError_t launch_bp_texlin(const LaunchConfig &c, const BpParams &p, cudaStream_t s);
cudaError_t launch_bp_soft_f32_trunc(const LaunchConfig &c, const BpParams &p, cudaStream_t s);

// Cosine weighting + row-wise ramp filter of raw projections (rct_filter.cu).
struct FilterParams {
    int W, H;
    int log2n;                 // transform length N = 2^log2n >= 2W - 1
    float sdd, pitch;          // source-detector distance, pixel pitch (mm)
    const float2 *twiddle;     // N entries exp(-2 pi i k / N)
    const float *spectrum;     // N entries: the kernel's DFT times pitch / N (real)
    const float2 *principal;   // (u0, v0) of the first view filtered, then one per view
};
cudaError_t launch_ramp_filter(const FilterParams &f, const float *raw, void *out, int out_dtype, int n,
                               cudaStream_t s);

cudaError_t launch_convert(const float *src, void *dst, size_t n, int dtype, cudaStream_t s);
// Build the zero-padded quad images of n views (see ViewParams) from their linear images: view k reads
// src + k * W * H elements and writes the staged image k images after dst (one launch per batch).
cudaError_t launch_stage_quads(const void *src, void *dst, int W, int H, int dtype, int n, cudaStream_t s);
size_t quad_bytes(int W, int H, int dtype);
// Build the zero-padded vertical-pair images of n views (see ViewParams), laid out as above.
cudaError_t launch_stage_pairs(const void *src, void *dst, int W, int H, int dtype, int n, cudaStream_t s);
// Build the zero-padded difference-quad images of n FP32 views (see ViewParams; quad_bytes(W, H, DT_F32)
// each), laid out as above.
cudaError_t launch_stage_dquads(const float *src, void *dst, int W, int H, int n, cudaStream_t s);
size_t pair_bytes(int W, int H, int dtype);

// Fill the matrix of a view (FP32) from its FP64 fold (rows u', v', w over centred voxel
// coordinates) and integer detector shift; and the high/low split used for block frames.
void set_view_geometry(ViewParams *vp, const double fold[12], int cu, int cv);
void set_view_geo(ViewGeo *vg, const double fold[12], int cu, int cv);

// Record a message for rct_last_error() on the calling thread and return `code`.
rct_status rct_internal_fail(rct_status code, const char *fmt, ...);
cudaError_t launch_widen_bf16(const uint16_t *src, float *dst, size_t n, cudaStream_t s);
// vol[i] += part[i] + part[stride + i] + ... (parts terms, in that order) for i < n.
cudaError_t launch_add_partials(float *vol, const float *part, size_t n, size_t stride, int parts, cudaStream_t s);

}  // namespace rct

// Voxel-driven backprojection kernel (the paper's Listing 1, Parts 1-3), sm_103a.
//
// Thread -> voxel mapping: a thread owns XV consecutive voxels along x
// (one 128-bit access for XV = 4) times a run of R voxels along z at a fixed
// y.  It keeps their XV*R partial sums in registers while it walks the K
// views of one pass, so the volume is read and written once per K views
// (8/K bytes of HBM traffic per voxel update instead of the listing's 8).
//
// Per voxel update (Part 1): three FMAs give (u', v', w) from the folded
// matrix, one approximate reciprocal r = 1/w (as the paper's kernels use a
// reciprocal instead of a divide, Section "SIMD Vectorization"), two
// multiplies give q = (u' r, v' r).  floor(q) and frac(q) come from one
// directed-rounding add of 1.5 * 2^23 (the integer part lands in the low
// mantissa bits), which keeps the conversion off the quarter-rate pipe.
// Part 2 fetches the 2x2 cell, Part 3 does three lerps and adds val * r^2.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "rct_internal.h"

namespace rct {

// 1.5 * 2^23: adding it to |q| < 2^22 with rounding toward -inf leaves floor(q) in the low bits.
constexpr float kMagic = 12582912.0f;
constexpr int kMagicBits = 0x4B400000;

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int DT>
__device__ __forceinline__ float load_px(const void *img, ptrdiff_t off) {
    if constexpr (DT == DT_F32) {
        return __ldg(static_cast<const float *>(img) + off);
    } else if constexpr (DT == DT_F16) {
        return __half2float(__ldg(static_cast<const __half *>(img) + off));
    } else {
        const unsigned short b = __ldg(static_cast<const unsigned short *>(img) + off);
        return __uint_as_float(static_cast<unsigned>(b) << 16);
    }
}

// Part 2 + 3 for one voxel and one view: returns the bilinear value at
// detector position (cu + qx, cv + qy), zero outside the W x H image.
template <int G, int DT>
__device__ __forceinline__ float sample(const ViewParams &v, float qx, float qy, int W, int H) {
    if constexpr (G == G_TEXLIN) {
        // Texture-unit bilinear; the matrix already carries the +0.5 texel-centre shift.
        return tex2D<float>(static_cast<cudaTextureObject_t>(v.tex), qx, qy);
    } else {
        const float tx = __fadd_rd(qx, kMagic);   // kMagic + floor(qx)
        const float ty = __fadd_rd(qy, kMagic);
        const float flx = tx - kMagic;            // floor(qx), exact
        const float fly = ty - kMagic;
        const float fx = qx - flx;                // interpolation weights in [0, 1)
        const float fy = qy - fly;
        float a, b, c, d;                          // (i0,j0) (i0+1,j0) (i0,j0+1) (i0+1,j0+1)
        if constexpr (G == G_TLD4) {
            // The gather footprint of coordinate (i0 + 1, j0 + 1) is exactly texels i0..i0+1,
            // j0..j0+1 (texel centres at +0.5), independent of the unit's coordinate rounding.
            const float gx = tx - (kMagic - static_cast<float>(v.cu + 1));
            const float gy = ty - (kMagic - static_cast<float>(v.cv + 1));
            const cudaTextureObject_t t = static_cast<cudaTextureObject_t>(v.tex);
            if constexpr (DT == DT_BF16) {
                const uint4 g = tex2Dgather<uint4>(t, gx, gy, 0);
                a = __uint_as_float(g.w << 16);
                b = __uint_as_float(g.z << 16);
                c = __uint_as_float(g.x << 16);
                d = __uint_as_float(g.y << 16);
            } else {
                const float4 g = tex2Dgather<float4>(t, gx, gy, 0);
                a = g.w; b = g.z; c = g.x; d = g.y;
            }
        } else {
            const int i0 = __float_as_int(tx) - kMagicBits + v.cu;
            const int j0 = __float_as_int(ty) - kMagicBits + v.cv;
            const bool x0 = static_cast<unsigned>(i0) < static_cast<unsigned>(W);
            const bool x1 = static_cast<unsigned>(i0 + 1) < static_cast<unsigned>(W);
            const bool y0 = static_cast<unsigned>(j0) < static_cast<unsigned>(H);
            const bool y1 = static_cast<unsigned>(j0 + 1) < static_cast<unsigned>(H);
            const ptrdiff_t o = static_cast<ptrdiff_t>(j0) * W + i0;
            a = (y0 && x0) ? load_px<DT>(v.img, o) : 0.0f;
            b = (y0 && x1) ? load_px<DT>(v.img, o + 1) : 0.0f;
            c = (y1 && x0) ? load_px<DT>(v.img, o + W) : 0.0f;
            d = (y1 && x1) ? load_px<DT>(v.img, o + W + 1) : 0.0f;
        }
        const float t0 = fmaf(fx, b - a, a);
        const float t1 = fmaf(fx, d - c, c);
        return fmaf(fy, t1 - t0, t0);
    }
}

template <int G, int DT, int XV, int R>
__global__ void __launch_bounds__(512) bp_kernel(const __grid_constant__ BpParams p) {
    const int L = p.L;
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * XV;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z0 = blockIdx.z * R;
    if (x0 >= L || y >= L) return;
    const size_t plane = static_cast<size_t>(L) * L;
    float *vb = p.vol + static_cast<size_t>(z0) * plane + static_cast<size_t>(y) * L + x0;

    float acc[R][XV];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool live = p.accumulate && (z0 + r < L);
        if constexpr (XV == 4) {
            float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
            if (live) t = *reinterpret_cast<const float4 *>(vb + r * plane);
            acc[r][0] = t.x; acc[r][1] = t.y; acc[r][2] = t.z; acc[r][3] = t.w;
        } else if constexpr (XV == 2) {
            float2 t = make_float2(0.f, 0.f);
            if (live) t = *reinterpret_cast<const float2 *>(vb + r * plane);
            acc[r][0] = t.x; acc[r][1] = t.y;
        } else {
            acc[r][0] = live ? vb[r * plane] : 0.0f;
        }
    }

    const float xc0 = static_cast<float>(x0) - p.cen;
    const float yc = static_cast<float>(y) - p.cen;
    const float zc0 = static_cast<float>(z0) - p.cen;

#pragma unroll 1
    for (int k = 0; k < p.K; ++k) {
        const ViewParams &v = p.view[k];
        const float *m = v.m;
        // Part 1 at the thread's first voxel, then steps along z and x.
        const float bu = fmaf(m[0], xc0, fmaf(m[1], yc, fmaf(m[2], zc0, m[3])));
        const float bv = fmaf(m[4], xc0, fmaf(m[5], yc, fmaf(m[6], zc0, m[7])));
        const float bw = fmaf(m[8], xc0, fmaf(m[9], yc, fmaf(m[10], zc0, m[11])));
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float ur = fmaf(static_cast<float>(r), m[2], bu);
            const float vr = fmaf(static_cast<float>(r), m[6], bv);
            const float wr = fmaf(static_cast<float>(r), m[10], bw);
#pragma unroll
            for (int j = 0; j < XV; ++j) {
                const float u = fmaf(static_cast<float>(j), m[0], ur);
                const float vv = fmaf(static_cast<float>(j), m[4], vr);
                const float w = fmaf(static_cast<float>(j), m[8], wr);
                const float rw = rcp_approx(w);
                const float val = sample<G, DT>(v, u * rw, vv * rw, p.W, p.H);
                acc[r][j] = fmaf(val, rw * rw, acc[r][j]);
            }
        }
    }

#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (z0 + r >= L) break;
        if constexpr (XV == 4) {
            *reinterpret_cast<float4 *>(vb + r * plane) =
                make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
        } else if constexpr (XV == 2) {
            *reinterpret_cast<float2 *>(vb + r * plane) = make_float2(acc[r][0], acc[r][1]);
        } else {
            vb[r * plane] = acc[r][0];
        }
    }
}

template <int G, int DT, int XV, int R>
cudaError_t launch_one(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    const int gx = (p.L / XV + c.bx - 1) / c.bx;
    const dim3 grid(gx, (p.L + c.by - 1) / c.by, (p.L + R - 1) / R);
    bp_kernel<G, DT, XV, R><<<grid, dim3(c.bx, c.by, 1), 0, s>>>(p);
    return cudaGetLastError();
}

template <int G, int DT, int XV>
cudaError_t dispatch_r(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    switch (c.zrun) {
        case 1: return launch_one<G, DT, XV, 1>(c, p, s);
        case 2: return launch_one<G, DT, XV, 2>(c, p, s);
        case 4: return launch_one<G, DT, XV, 4>(c, p, s);
        case 8: return launch_one<G, DT, XV, 8>(c, p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int G, int DT>
cudaError_t dispatch_xv(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    switch (c.xv) {
        case 1: return dispatch_r<G, DT, 1>(c, p, s);
        case 2: return dispatch_r<G, DT, 2>(c, p, s);
        case 4: return dispatch_r<G, DT, 4>(c, p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rct

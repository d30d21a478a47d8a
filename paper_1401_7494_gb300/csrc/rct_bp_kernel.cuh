// Voxel-driven backprojection kernel (the paper's Listing 1, Parts 1-3), sm_103a.
//
// Thread -> voxel mapping: a thread owns XV consecutive voxels along x
// (one 128-bit access for XV = 4) times a run of R voxels along z at a fixed
// y.  It keeps their XV*R partial sums in registers while it walks the K
// views of one pass, so the volume is read and written once per K views
// (8/K bytes of HBM traffic per voxel update instead of the listing's 8).
//
// Part 1 per voxel update: the (u', v') pair comes from one packed FMA
// (f32x2) and w from one FMA of the folded matrix; one approximate
// reciprocal r = 1/w (the paper's kernels also use a reciprocal instead of a
// divide, Section "SIMD Vectorization"); one packed multiply gives
// q = (u' r, v' r).  floor(q) and frac(q) come from a packed add of
// 1.5 * 2^23 rounded toward -inf (the integer part lands in the low mantissa
// bits), so no conversion instruction is needed.  The coordinates are either
// global (the folded matrix over centred voxel coordinates, its rows read from
// kernel parameters into uniform registers) or block frames (FRAME: per block
// and view, the block corner's coordinates in double-float and a block-local
// integer shift, held in shared memory: smaller rounding error, more
// registers per thread).
//
// Part 2 fetches the 2x2 cell by one of these routes (ROUTE below):
//   * texture gather (tld4) from a staged gather-capable array with a zero
//     border -- the texture pipe;
//   * one 128-bit (64-bit for 16-bit data) load of a staged "quad" element
//     that holds the whole cell, from a zero-padded copy of the image (the
//     paper's zero-padded projection buffer, Section "SIMD Vectorization",
//     taken one step further) -- the load/store pipe;
//   * two 64-bit (32-bit) loads of staged vertical pairs: the same cell in
//     half the staged bytes, and neighbouring lanes share cache sectors;
//   * one 128-bit load of a staged "difference quad" (FP32): the cell's left
//     column and the two horizontal differences, so that both rows are
//     interpolated along x by one packed FMA;
//   * four predicated loads straight from the caller's linear image (no
//     staging at all);
//   * mixed: each z-run split between the texture gather and the quad load.
// A view is skipped for a warp whose voxel runs all project off the detector.
// Part 3: three lerps (two of them as one packed f32x2 pair) and
// acc += val * r^2.
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

// Double-float accumulation: adds (h + l) * d to the unevaluated sum s + e, with the exact
// product error (FMA) and the exact addition error (two-sum) kept in e.
__device__ __forceinline__ void df_add_term(float h, float l, float d, float &s, float &e) {
    const float p = h * d;
    const float pe = fmaf(h, d, -p);
    const float t = s + p;
    const float bb = t - s;
    const float se = (s - (t - bb)) + (p - bb);
    s = t;
    e += se + fmaf(l, d, pe);
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

// Bounds-checking build (-DRCT_CHECK_BOUNDS): every computed index of a staged image, of a plain-load
// tap and of the volume is checked against its buffer before the access; a violation is counted on
// the device (BpParams::viol) and the access is skipped -- never a trap.
#ifdef RCT_CHECK_BOUNDS
__device__ __forceinline__ bool rct_in_bounds(bool ok, unsigned long long *viol) {
    if (!ok && viol) atomicAdd(viol, 1ull);
    return ok;
}
#endif

// Per-view constants the inner loop needs, hoisted out of the z-run.
struct ViewConsts {
    float2 m_z;      // (m[2], m[6]): step of (u', v') per z voxel
    float w_z;       // m[10]
    float2 gofs;     // t + gofs = gather corner (i0 + 1, j0 + 1)
    int cu, cv;
    int qcx, qcy;    // bits(t) - qc = padded quad index (i0 + 1, j0 + 1)
    cudaTextureObject_t tex;
    const void *img;
    const void *quad;
#ifdef RCT_CHECK_BOUNDS
    long long qelems;
    unsigned long long *viol;
#endif
};

// Route of the load part of a z-run (G_SOFT only).
//   ROUTE_TEX: every z position by texture gather;  ROUTE_LDG: every z position by four
//   predicated loads from the linear image;  ROUTE_QLD: every z position by one quad load;
//   ROUTE_MIX: z positions [0, tex_zrun) by texture gather, the rest by quad loads.
//   ROUTE_PLD: every z position by two loads of staged vertical pairs.
//   ROUTE_DQD: every z position by one load of a staged difference quad (FP32).
enum Route : int { ROUTE_TEX = 0, ROUTE_LDG = 1, ROUTE_QLD = 2, ROUTE_MIX = 3, ROUTE_PLD = 4, ROUTE_DQD = 5 };

// Floor and fraction of q = uv * r (r = 1 / w): the packed add of 1.5 * 2^23 rounded toward -inf
// gives t = kMagic + floor(q), whose low bits are floor(q) as an integer; f = q - floor(q), formed by one
// FMA: exact except for q in (-0.5, 0) -- the half pixel before the integer shift (cu, cv) -- where the
// fraction needs a bit below q's last one and is rounded to nearest (error <= 2^-25, below the rounding
// that q itself carries).
// (Folding the multiply into a directed-rounding FMA saves an instruction but measured slower:
// the compiler's schedule of the z-run changes with it.)
__device__ __forceinline__ void floor_frac(float2 uv, float rw, float2 &t, float2 &f) {
    const float2 q = __fmul2_rn(uv, make_float2(rw, rw));
    t = __fadd2_rd(q, make_float2(kMagic, kMagic));
    f = __ffma2_rn(__fadd2_rn(t, make_float2(-kMagic, -kMagic)), make_float2(-1.0f, -1.0f), q);
}

// Part 2 + 3 by texture gather: adds the bilinear value at detector (cu + q.x, cv + q.y), times
// w2, to acc.  Taps off the detector read the texture's zero border.
template <int DT>
__device__ __forceinline__ void accumulate_tex(const ViewConsts &c, float2 t, float2 f, float w2, float &acc) {
    // The gather footprint of coordinate (i0 + 1, j0 + 1) is exactly texels i0..i0+1 x
    // j0..j0+1 (texel centres at +0.5), independent of the unit's coordinate rounding.
    const float2 g = __fadd2_rn(t, c.gofs);
    float a, b, cc, d;                                                      // (i0,j0) (i0+1,j0) (i0,j0+1) (i0+1,j0+1)
    if constexpr (DT == DT_BF16) {
        const uint4 v = tex2Dgather<uint4>(c.tex, g.x, g.y, 0);
        a = __uint_as_float(v.w << 16);
        b = __uint_as_float(v.z << 16);
        cc = __uint_as_float(v.x << 16);
        d = __uint_as_float(v.y << 16);
    } else {
        const float4 v = tex2Dgather<float4>(c.tex, g.x, g.y, 0);
        a = v.w; b = v.z; cc = v.x; d = v.y;
    }
    const float t0 = fmaf(f.x, b - a, a);
    const float t1 = fmaf(f.x, d - cc, cc);
    acc = fmaf(fmaf(f.y, t1 - t0, t0), w2, acc);
}

// Part 2 + 3 by one load of the staged quad element (see ViewParams).  A cell with no tap on the
// image has no element: such a lane loads element 0, which every off-image lane of the warp
// shares (one cached sector), and adds it with weight 0.
template <int DT>
__device__ __forceinline__ void accumulate_quad(const ViewConsts &c, float2 t, float2 f, float w2, int W, int H,
                                                float &acc) {
    const int ix = __float_as_int(t.x) - c.qcx;                             // padded index (i0 + 1, j0 + 1)
    const int jy = __float_as_int(t.y) - c.qcy;
    const bool on = static_cast<unsigned>(ix) <= static_cast<unsigned>(W) &&
                    static_cast<unsigned>(jy) <= static_cast<unsigned>(H);
    const unsigned e = on ? static_cast<unsigned>(jy) * static_cast<unsigned>(W + 1) + static_cast<unsigned>(ix) : 0u;
    w2 = on ? w2 : 0.0f;
#ifdef RCT_CHECK_BOUNDS
    if (!rct_in_bounds(static_cast<long long>(e) < c.qelems, c.viol)) return;
#endif
    float2 ac, bd;                                                          // (I[j0][i0], I[j0+1][i0]), (I[j0][i0+1], I[j0+1][i0+1])
    if constexpr (DT == DT_F32) {
        const float4 v = __ldg(static_cast<const float4 *>(c.quad) + e);
        ac = make_float2(v.x, v.y);
        bd = make_float2(v.z, v.w);
    } else {
        const uint2 v = __ldg(static_cast<const uint2 *>(c.quad) + e);
        if constexpr (DT == DT_F16) {
            ac = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
            bd = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
        } else {
            ac = make_float2(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u));
            bd = make_float2(__uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
        }
    }
    // both rows lerped along x at once: (t0, t1) = ac + f.x * (bd - ac)
    const float2 rows = __ffma2_rn(make_float2(f.x, f.x), __ffma2_rn(ac, make_float2(-1.0f, -1.0f), bd), ac);
    acc = fmaf(fmaf(f.y, rows.y - rows.x, rows.x), w2, acc);
}

// Part 2 + 3 by two loads of consecutive staged vertical pairs (see ViewParams): neighbouring
// lanes share cache sectors, so less data moves from L2 than with quads.  Same off-image rule.
template <int DT>
__device__ __forceinline__ void accumulate_pair(const ViewConsts &c, float2 t, float2 f, float w2, int W, int H,
                                                float &acc) {
    const int ix = __float_as_int(t.x) - c.qcx;                             // padded index (i0 + 1, j0 + 1)
    const int jy = __float_as_int(t.y) - c.qcy;
    const bool on = static_cast<unsigned>(ix) <= static_cast<unsigned>(W) &&
                    static_cast<unsigned>(jy) <= static_cast<unsigned>(H);
    const unsigned e = on ? static_cast<unsigned>(jy) * static_cast<unsigned>(W + 2) + static_cast<unsigned>(ix) : 0u;
    w2 = on ? w2 : 0.0f;
#ifdef RCT_CHECK_BOUNDS
    if (!rct_in_bounds(static_cast<long long>(e) + 1 < c.qelems, c.viol)) return;
#endif
    float2 ac, bd;                                                          // (I[j0][i0], I[j0+1][i0]), (I[j0][i0+1], I[j0+1][i0+1])
    if constexpr (DT == DT_F32) {
        const float2 *pp = static_cast<const float2 *>(c.quad) + e;
        ac = __ldg(pp);
        bd = __ldg(pp + 1);
    } else {
        const unsigned *pp = static_cast<const unsigned *>(c.quad) + e;
        const unsigned v0 = __ldg(pp), v1 = __ldg(pp + 1);
        if constexpr (DT == DT_F16) {
            ac = __half22float2(*reinterpret_cast<const __half2 *>(&v0));
            bd = __half22float2(*reinterpret_cast<const __half2 *>(&v1));
        } else {
            ac = make_float2(__uint_as_float(v0 << 16), __uint_as_float(v0 & 0xffff0000u));
            bd = make_float2(__uint_as_float(v1 << 16), __uint_as_float(v1 & 0xffff0000u));
        }
    }
    const float2 rows = __ffma2_rn(make_float2(f.x, f.x), __ffma2_rn(ac, make_float2(-1.0f, -1.0f), bd), ac);
    acc = fmaf(fmaf(f.y, rows.y - rows.x, rows.x), w2, acc);
}

// Part 2 + 3 by one load of a staged difference quad (FP32; see ViewParams): both rows' lerps along x
// in one packed FMA, with the roundings the quad and pair routes perform (bitwise the same sums).
// Same off-image rule as the quads.
__device__ __forceinline__ void accumulate_dquad(const ViewConsts &c, float2 t, float2 f, float w2, int W, int H,
                                                 float &acc) {
    const int ix = __float_as_int(t.x) - c.qcx;                             // padded index (i0 + 1, j0 + 1)
    const int jy = __float_as_int(t.y) - c.qcy;
    const bool on = static_cast<unsigned>(ix) <= static_cast<unsigned>(W) &&
                    static_cast<unsigned>(jy) <= static_cast<unsigned>(H);
    const unsigned e = on ? static_cast<unsigned>(jy) * static_cast<unsigned>(W + 1) + static_cast<unsigned>(ix) : 0u;
    w2 = on ? w2 : 0.0f;
#ifdef RCT_CHECK_BOUNDS
    if (!rct_in_bounds(static_cast<long long>(e) < c.qelems, c.viol)) return;
#endif
    const float4 v = __ldg(static_cast<const float4 *>(c.quad) + e);      // (a, c, b - a, d - c)
    const float2 rows = __ffma2_rn(make_float2(f.x, f.x), make_float2(v.z, v.w), make_float2(v.x, v.y));
    acc = fmaf(fmaf(f.y, rows.y - rows.x, rows.x), w2, acc);
}

// Part 2 + 3 by four predicated loads from the caller's linear image (no staging).
template <int DT>
__device__ __forceinline__ void accumulate_ldg(const ViewConsts &c, float2 t, float2 f, float w2, int W, int H, float &acc) {
    const int i0 = __float_as_int(t.x) - kMagicBits + c.cu;
    const int j0 = __float_as_int(t.y) - kMagicBits + c.cv;
    const bool x0 = static_cast<unsigned>(i0) < static_cast<unsigned>(W);
    const bool x1 = static_cast<unsigned>(i0 + 1) < static_cast<unsigned>(W);
    const bool y0 = static_cast<unsigned>(j0) < static_cast<unsigned>(H);
    const bool y1 = static_cast<unsigned>(j0 + 1) < static_cast<unsigned>(H);
    const ptrdiff_t o = static_cast<ptrdiff_t>(j0) * W + i0;
#ifdef RCT_CHECK_BOUNDS
    {
        const ptrdiff_t px = static_cast<ptrdiff_t>(W) * H;
        const auto in = [px](ptrdiff_t q) { return q >= 0 && q < px; };
        if (!rct_in_bounds(!(y0 && x0) || in(o), c.viol) || !rct_in_bounds(!(y0 && x1) || in(o + 1), c.viol) ||
            !rct_in_bounds(!(y1 && x0) || in(o + W), c.viol) || !rct_in_bounds(!(y1 && x1) || in(o + W + 1), c.viol))
            return;
    }
#endif
    const float a = (y0 && x0) ? load_px<DT>(c.img, o) : 0.0f;
    const float b = (y0 && x1) ? load_px<DT>(c.img, o + 1) : 0.0f;
    const float cc = (y1 && x0) ? load_px<DT>(c.img, o + W) : 0.0f;
    const float d = (y1 && x1) ? load_px<DT>(c.img, o + W + 1) : 0.0f;
    const float t0 = fmaf(f.x, b - a, a);
    const float t1 = fmaf(f.x, d - cc, cc);
    acc = fmaf(fmaf(f.y, t1 - t0, t0), w2, acc);
}

// Padded cell index (i0 + 1, j0 + 1) of the voxel at (u', v', w); a cell with a tap on the
// image has it in [0, W] x [0, H].
__device__ __forceinline__ int2 cell_index(const ViewConsts &c, float2 uv, float w) {
    const float rw = rcp_approx(w);
    const float2 t = __ffma2_rd(uv, make_float2(rw, rw), make_float2(kMagic, kMagic));   // kMagic + floor(uv r)
    return make_int2(__float_as_int(t.x) - c.qcx, __float_as_int(t.y) - c.qcy);
}

// Block frame of one view (see ViewGeo): the block corner's (u', v', w) in double-float, a
// block-local integer pixel shift (cub, cvb), and the rows with the shift applied.  Stored as three
// float4: (tu, tv, wb, bits(cu)), (mx.u, mx.v, my.u, my.v), (mz.u, mz.v, bits(cv), 0).
__device__ __forceinline__ void block_frame(const ViewGeo *vg, float bX, float bY, float bZ, float4 out[3]) {
    const float4 *g4 = reinterpret_cast<const float4 *>(vg);
    const float4 h0 = g4[0], h1 = g4[1], l0 = g4[2], l1 = g4[3], hw = g4[4], lw = g4[5];
    const int4 sh = reinterpret_cast<const int4 *>(vg)[6];
    // hu = (u0, v0, u1, v1 | u2, v2, u3, v3): columns x, y, z, translation
    float su = h1.z, eu = l1.z, sv = h1.w, ev = l1.w, sw = hw.w, ew = lw.w;
    df_add_term(h0.x, l0.x, bX, su, eu);
    df_add_term(h0.z, l0.z, bY, su, eu);
    df_add_term(h1.x, l1.x, bZ, su, eu);
    df_add_term(h0.y, l0.y, bX, sv, ev);
    df_add_term(h0.w, l0.w, bY, sv, ev);
    df_add_term(h1.y, l1.y, bZ, sv, ev);
    df_add_term(hw.x, lw.x, bX, sw, ew);
    df_add_term(hw.y, lw.y, bY, sw, ew);
    df_add_term(hw.z, lw.z, bZ, sw, ew);
    const float wb = sw + ew;
    const float rb = rcp_approx(wb);
    const float cub = rintf((su + eu) * rb);                                // any nearby integer will do
    const float cvb = rintf((sv + ev) * rb);
    const float pu = cub * sw, pv = cvb * sw;
    const float tu = (su - pu) + ((eu - fmaf(cub, sw, -pu)) - cub * ew);   // u'(corner) - cub w(corner)
    const float tv = (sv - pv) + ((ev - fmaf(cvb, sw, -pv)) - cvb * ew);
    // the shift scales with each voxel's own w: the local rows are (u' - cub w, v' - cvb w)
    out[0] = make_float4(tu, tv, wb, __int_as_float(sh.x + static_cast<int>(cub)));
    out[1] = make_float4(fmaf(-cub, hw.x, h0.x), fmaf(-cvb, hw.x, h0.y), fmaf(-cub, hw.y, h0.z), fmaf(-cvb, hw.y, h0.w));
    out[2] = make_float4(fmaf(-cub, hw.z, h1.x), fmaf(-cvb, hw.z, h1.y), __int_as_float(sh.y + static_cast<int>(cvb)), 0.f);
}

// FRAME: block frames (needs p.geo) instead of the global frame; the texture-filtered kernel
// always takes the global frame (the texture unit needs absolute coordinates).
// TRUNC: the cell index of Listing 1's (int) cast, which truncates toward zero, instead of floor
// (RabbitCT compatibility; plain loads only).
// SPLIT: the view split (see BpParams): this block handles one group of the pass's views and adds into
// vol (group 0) or into its group's partial volume.
template <int G, int DT, int XV, int R, int ROUTE, bool FRAME, bool TRUNC, bool SPLIT = false>
__device__ __forceinline__ void bp_body(const BpParams &p) {
    static_assert(!FRAME || G == G_SOFT, "block frames are for the software gathers");
    static_assert(!TRUNC || (G == G_SOFT && ROUTE == ROUTE_LDG && !FRAME), "truncation: global frame, plain loads");
    static_assert(ROUTE != ROUTE_DQD || DT == DT_F32, "difference quads hold FP32 values");
    static_assert(!SPLIT || (G == G_SOFT && !FRAME && !TRUNC), "view split: global frame, floor rule");
    const int L = p.L;
    // Lane map.  With 8-thread-wide blocks a warp covers 8 x 4 voxel columns.  The L1 data pipe serves an
    // 8-byte load half a warp (16 lanes) at a time, and a half warp's cost grows with the number of
    // cache lines its lanes touch; rows 0-1 and 2-3 of the warp (8 x 2 each) project onto strips about
    // 20 pixels long, while its left and right 4 x 4 halves project onto more compact patches.  So lanes
    // 0-15 take x 0-3 and lanes 16-31 take x 4-7 (ncu: 3.97 instead of 4.52 data-pipe wavefronts per pair
    // load).  Every voxel's arithmetic is unchanged: the result is bitwise the same.
    int tx = threadIdx.x, ty = threadIdx.y;
    if (blockDim.x == 8 && (blockDim.y & 3) == 0) {
        const int t = threadIdx.y * 8 + threadIdx.x;
        const int ln = t & 31, wp = t >> 5;
        tx = (ln & 3) | ((ln >> 4) << 2);
        ty = (wp << 2) | ((ln >> 2) & 3);
    }
    const int x0 = (blockIdx.x * blockDim.x + tx) * XV;
    const int y = blockIdx.y * blockDim.y + ty;
    int group = 0, zblock = blockIdx.z;
    if constexpr (SPLIT) {
        group = blockIdx.z / p.split_runs;
        zblock = blockIdx.z - group * p.split_runs;
    }
    const int z0 = p.z_base + zblock * R;
    float *const vol = (SPLIT && group > 0) ? p.part + (group - 1) * p.part_stride : p.vol;
    const int accumulate = (SPLIT && group > 0) ? p.accumulate_part : p.accumulate;
    const int k_begin = SPLIT ? group * p.split_views : 0;
    const int k_end = SPLIT ? min(k_begin + p.split_views, p.K) : p.K;
    // the block's first voxel (centred coordinates, exact) and this thread's offset from it
    const float bX = static_cast<float>(blockIdx.x * blockDim.x * XV) - p.cen;
    const float bY = static_cast<float>(blockIdx.y * blockDim.y) - p.cen;
    const float bZ = static_cast<float>(z0) - p.cen;
    const float lx = static_cast<float>(tx * XV);
    const float ly = static_cast<float>(ty);

    const bool inside = x0 < L && y < L;
    const size_t plane = static_cast<size_t>(L) * L;
    float *vb = vol + (inside ? static_cast<size_t>(z0) * plane + static_cast<size_t>(y) * L + x0 : 0);
    // The volume rows of the run are requested into L2 first (without holding registers), so the
    // DRAM latency overlaps the set-up below.
    if (inside && accumulate) {
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (z0 + r < L) asm volatile("prefetch.global.L2 [%0];" :: "l"(vb + r * plane));
    }

    // Block frames of the pass's views: lane k of the first warp evaluates view k once for the
    // whole block (K <= 32); every thread reaches the barrier before any of them leaves.
    __shared__ float4 s_frame[FRAME ? KMAX : 1][3];
    if constexpr (FRAME) {
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        if (tid < p.K) block_frame(p.geo + p.first_view + tid, bX, bY, bZ, s_frame[tid]);
        __syncthreads();
    }
    if (!inside) return;

    // The volume is touched once per pass: streaming (evict-first) loads and stores keep it from
    // displacing the projection data the gathers reuse in L1 and L2.
    float acc[R][XV];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        bool live = accumulate && (z0 + r < L);
#ifdef RCT_CHECK_BOUNDS
        {
            const long long at = static_cast<long long>(z0 + r - p.vol_z0) * L * L + static_cast<long long>(y) * L + x0;
            if (live) live = rct_in_bounds(at >= 0 && at + XV <= p.vol_elems, p.viol);
        }
#endif
        if constexpr (XV == 4) {
            float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
            if (live) t = __ldcs(reinterpret_cast<const float4 *>(vb + r * plane));
            acc[r][0] = t.x; acc[r][1] = t.y; acc[r][2] = t.z; acc[r][3] = t.w;
        } else if constexpr (XV == 2) {
            float2 t = make_float2(0.f, 0.f);
            if (live) t = __ldcs(reinterpret_cast<const float2 *>(vb + r * plane));
            acc[r][0] = t.x; acc[r][1] = t.y;
        } else {
            acc[r][0] = live ? __ldcs(vb + r * plane) : 0.0f;
        }
    }

    const float xc0 = static_cast<float>(x0) - p.cen;
    const float yc = static_cast<float>(y) - p.cen;
    const int tex_zrun = p.tex_zrun;   // z positions [0, tex_zrun) use the texture route

#pragma unroll 1
    for (int k = k_begin; k < k_end; ++k) {
        const ViewParams &v = p.view[k];
        const float2 *muv = reinterpret_cast<const float2 *>(v.muv);
        const float *mw = v.mw;
        ViewConsts c;
        c.w_z = mw[2];
        c.tex = static_cast<cudaTextureObject_t>(v.tex);
        c.img = v.img;
        c.quad = v.quad;
#ifdef RCT_CHECK_BOUNDS
        c.qelems = p.qelems;
        c.viol = p.viol;
#endif
        float2 m_x, buv;
        float bw;
        if constexpr (FRAME) {
            const float4 f0 = s_frame[k][0], f1 = s_frame[k][1], f2 = s_frame[k][2];
            m_x = make_float2(f1.x, f1.y);
            c.m_z = make_float2(f2.x, f2.y);
            c.cu = __float_as_int(f0.w);
            c.cv = __float_as_int(f2.z);
            buv = __ffma2_rn(make_float2(lx, lx), m_x,
                             __ffma2_rn(make_float2(ly, ly), make_float2(f1.z, f1.w), make_float2(f0.x, f0.y)));
            bw = fmaf(mw[0], lx, fmaf(mw[1], ly, f0.z));
        } else {
            // Global frame: the matrix rows stay in kernel parameters, read into uniform registers.
            m_x = muv[0];
            c.m_z = muv[2];
            buv = __ffma2_rn(make_float2(xc0, xc0), muv[0],
                             __ffma2_rn(make_float2(yc, yc), muv[1], __ffma2_rn(make_float2(bZ, bZ), muv[2], muv[3])));
            bw = fmaf(mw[0], xc0, fmaf(mw[1], yc, fmaf(mw[2], bZ, mw[3])));
            c.cu = v.cu;
            c.cv = v.cv;
        }
        c.gofs = make_float2(-(kMagic - static_cast<float>(c.cu + 1)), -(kMagic - static_cast<float>(c.cv + 1)));
        c.qcx = kMagicBits - c.cu - 1;
        c.qcy = kMagicBits - c.cv - 1;
        if constexpr (G == G_SOFT) {
            // Clipping per run (the paper's clipping mask, Section "Implementation"): the
            // thread's voxels form a segment (XV = 1) or parallelogram in (x, z); its projection
            // is the convex hull of the corners' projections.  If every corner's cell lies on the
            // same outer side of the detector, no voxel of the run touches the image.  When that
            // holds for the whole warp, the view is skipped.
            bool left = true, right = true, top = true, bottom = true;
#pragma unroll
            for (int cr = 0; cr < (R > 1 ? 2 : 1); ++cr) {
#pragma unroll
                for (int cj = 0; cj < (XV > 1 ? 2 : 1); ++cj) {
                    const float fr = cr ? static_cast<float>(R - 1) : 0.0f;
                    const float fj = cj ? static_cast<float>(XV - 1) : 0.0f;
                    const float2 uv = __ffma2_rn(make_float2(fj, fj), m_x, __ffma2_rn(make_float2(fr, fr), c.m_z, buv));
                    const float w = fmaf(fj, mw[0], fmaf(fr, c.w_z, bw));
                    const int2 ci = cell_index(c, uv, w);
                    // (a truncated cell of a coordinate in (-2, -1) still has its right tap on column 0)
                    left = left && ci.x < (TRUNC ? -1 : 0);
                    right = right && ci.x > p.W;
                    top = top && ci.y < (TRUNC ? -1 : 0);
                    bottom = bottom && ci.y > p.H;
                }
            }
            if (__all_sync(0xffffffffu, left || right || top || bottom)) continue;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float fr = static_cast<float>(r);
            const float2 uvr = __ffma2_rn(make_float2(fr, fr), c.m_z, buv);
            const float wr = fmaf(fr, c.w_z, bw);
#pragma unroll
            for (int j = 0; j < XV; ++j) {
                const float fj = static_cast<float>(j);
                const float2 uv = (j == 0) ? uvr : __ffma2_rn(make_float2(fj, fj), m_x, uvr);
                const float w = (j == 0) ? wr : fmaf(fj, mw[0], wr);
                const float rw = rcp_approx(w);
                const float w2 = rw * rw;
                if constexpr (G == G_TEXLIN) {
                    // Texture-unit bilinear; the matrix already carries the +0.5 texel-centre shift.
                    const float2 q = __fmul2_rn(uv, make_float2(rw, rw));
                    acc[r][j] = fmaf(tex2D<float>(c.tex, q.x, q.y), w2, acc[r][j]);
                } else {
                    float2 t, f;
                    floor_frac(uv, rw, t, f);
                    if constexpr (TRUNC) {
                        // (int) of a negative coordinate with a fraction is floor + 1: the cell moves one
                        // pixel right and its fraction becomes f - 1 (the listing then extrapolates).
                        const float ax = (__float_as_int(t.x) <= c.qcx && f.x != 0.0f) ? 1.0f : 0.0f;
                        const float ay = (__float_as_int(t.y) <= c.qcy && f.y != 0.0f) ? 1.0f : 0.0f;
                        t = __fadd2_rn(t, make_float2(ax, ay));
                        f = __fadd2_rn(f, make_float2(-ax, -ay));
                    }
                    if constexpr (ROUTE == ROUTE_TEX) {
                        accumulate_tex<DT>(c, t, f, w2, acc[r][j]);
                    } else if constexpr (ROUTE == ROUTE_LDG) {
                        accumulate_ldg<DT>(c, t, f, w2, p.W, p.H, acc[r][j]);
                    } else if constexpr (ROUTE == ROUTE_QLD) {
                        accumulate_quad<DT>(c, t, f, w2, p.W, p.H, acc[r][j]);
                    } else if constexpr (ROUTE == ROUTE_PLD) {
                        accumulate_pair<DT>(c, t, f, w2, p.W, p.H, acc[r][j]);
                    } else if constexpr (ROUTE == ROUTE_DQD) {
                        accumulate_dquad(c, t, f, w2, p.W, p.H, acc[r][j]);
                    } else if (r < tex_zrun) {
                        accumulate_tex<DT>(c, t, f, w2, acc[r][j]);
                    } else {
                        accumulate_quad<DT>(c, t, f, w2, p.W, p.H, acc[r][j]);
                    }
                }
            }
        }
    }

#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (z0 + r >= L) break;
#ifdef RCT_CHECK_BOUNDS
        {
            const long long at = static_cast<long long>(z0 + r - p.vol_z0) * L * L + static_cast<long long>(y) * L + x0;
            if (!rct_in_bounds(at >= 0 && at + XV <= p.vol_elems, p.viol)) continue;
        }
#endif
        if constexpr (XV == 4) {
            __stcs(reinterpret_cast<float4 *>(vb + r * plane), make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]));
        } else if constexpr (XV == 2) {
            __stcs(reinterpret_cast<float2 *>(vb + r * plane), make_float2(acc[r][0], acc[r][1]));
        } else {
            __stcs(vb + r * plane, acc[r][0]);
        }
    }
}

template <int G, int DT, int XV, int R, int ROUTE, bool FRAME, bool TRUNC = false, bool SPLIT = false>
__global__ void __launch_bounds__(512) bp_kernel(const __grid_constant__ BpParams p) {
    bp_body<G, DT, XV, R, ROUTE, FRAME, TRUNC, SPLIT>(p);
}

// Register caps (measured): the block-frame kernels keep the frame's rows and shift in per-thread
// registers through the z-run, and the z-runs of 16 keep 16 partial sums; capped, both keep more warps
// resident and run faster, while the global-frame kernels with shorter z-runs run slower under any cap.
// Swept at L=512 x 496 (pairs, K=32, z-run 16): global frame 40 / 48 / 56 / 64 registers gave 1224 / 1314 /
// 1304 / 1248 GUPS, block frame 1113 / 1257 / 1282 / 1236.
#ifndef RCT_CAPPED_MAXREG
#define RCT_CAPPED_MAXREG 48
#endif
#ifndef RCT_FRAME_MAXREG
#define RCT_FRAME_MAXREG 56
#endif
template <int DT, int XV, int R, int ROUTE>
__global__ void __maxnreg__(RCT_FRAME_MAXREG) bp_kernel_frame(const __grid_constant__ BpParams p) {
    bp_body<G_SOFT, DT, XV, R, ROUTE, true, false>(p);
}

template <int G, int DT, int XV, int ROUTE, bool TRUNC, bool SPLIT = false>
__global__ void __maxnreg__(RCT_CAPPED_MAXREG) bp_kernel_r16(const __grid_constant__ BpParams p) {
    bp_body<G, DT, XV, 16, ROUTE, false, TRUNC, SPLIT>(p);
}

template <int G, int DT, int XV, int R, int ROUTE, bool FRAME, bool TRUNC = false, bool SPLIT = false>
cudaError_t launch_one(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    if (FRAME && !p.geo) return cudaErrorInvalidValue;
    const int gx = (p.L / XV + c.bx - 1) / c.bx;
    const int zc = p.z_count > 0 ? p.z_count : p.L;
    const int runs = (zc + R - 1) / R;
    if constexpr (SPLIT) {
        if (c.split < 2 || !p.part) return cudaErrorInvalidValue;
        BpParams q = p;
        q.split_runs = runs;
        q.split_views = (p.K + c.split - 1) / c.split;
        const dim3 grid(gx, (p.L + c.by - 1) / c.by, runs * c.split);
        if constexpr (R == 16) bp_kernel_r16<G, DT, XV, ROUTE, false, true><<<grid, dim3(c.bx, c.by, 1), 0, s>>>(q);
        else bp_kernel<G, DT, XV, R, ROUTE, false, false, true><<<grid, dim3(c.bx, c.by, 1), 0, s>>>(q);
        return cudaGetLastError();
    }
    const dim3 grid(gx, (p.L + c.by - 1) / c.by, runs);
    if constexpr (FRAME) {
        bp_kernel_frame<DT, XV, R, ROUTE><<<grid, dim3(c.bx, c.by, 1), 0, s>>>(p);
    } else if constexpr (R == 16) {
        bp_kernel_r16<G, DT, XV, ROUTE, TRUNC><<<grid, dim3(c.bx, c.by, 1), 0, s>>>(p);
    } else {
        bp_kernel<G, DT, XV, R, ROUTE, FRAME, TRUNC><<<grid, dim3(c.bx, c.by, 1), 0, s>>>(p);
    }
    return cudaGetLastError();
}

template <int G, int DT, int XV, int ROUTE, bool FRAME, bool TRUNC = false, bool SPLIT = false>
cudaError_t dispatch_r(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    switch (c.zrun) {
        case 1: return launch_one<G, DT, XV, 1, ROUTE, FRAME, TRUNC, SPLIT>(c, p, s);
        case 2: return launch_one<G, DT, XV, 2, ROUTE, FRAME, TRUNC, SPLIT>(c, p, s);
        case 4: return launch_one<G, DT, XV, 4, ROUTE, FRAME, TRUNC, SPLIT>(c, p, s);
        case 8: return launch_one<G, DT, XV, 8, ROUTE, FRAME, TRUNC, SPLIT>(c, p, s);
        case 16:
            if constexpr (XV <= 2) return launch_one<G, DT, XV, 16, ROUTE, FRAME, TRUNC, SPLIT>(c, p, s);
            return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

// Block frames are compiled for the FP32 software gathers only (the API rejects them elsewhere).
template <int G, int DT, int ROUTE>
cudaError_t dispatch_xv(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    constexpr bool kFrames = (G == G_SOFT && DT == DT_F32);
    if ((c.frame && !kFrames) || c.trunc) return cudaErrorInvalidValue;
    if (c.split > 1) {
        if (G != G_SOFT || c.frame) return cudaErrorInvalidValue;
        if constexpr (G == G_SOFT) {
            switch (c.xv) {
                case 1: return dispatch_r<G, DT, 1, ROUTE, false, false, true>(c, p, s);
                case 2: return dispatch_r<G, DT, 2, ROUTE, false, false, true>(c, p, s);
                case 4: return dispatch_r<G, DT, 4, ROUTE, false, false, true>(c, p, s);
                default: return cudaErrorInvalidValue;
            }
        }
    }
    switch (c.xv) {
        case 1: return c.frame ? dispatch_r<G, DT, 1, ROUTE, kFrames>(c, p, s) : dispatch_r<G, DT, 1, ROUTE, false>(c, p, s);
        case 2: return c.frame ? dispatch_r<G, DT, 2, ROUTE, kFrames>(c, p, s) : dispatch_r<G, DT, 2, ROUTE, false>(c, p, s);
        case 4: return c.frame ? dispatch_r<G, DT, 4, ROUTE, kFrames>(c, p, s) : dispatch_r<G, DT, 4, ROUTE, false>(c, p, s);
        default: return cudaErrorInvalidValue;
    }
}

// RabbitCT compatibility (truncating cell index): FP32, global frame, plain loads from the caller's images.
inline cudaError_t dispatch_trunc(const LaunchConfig &c, const BpParams &p, cudaStream_t s) {
    switch (c.xv) {
        case 1: return dispatch_r<G_SOFT, DT_F32, 1, ROUTE_LDG, false, true>(c, p, s);
        case 2: return dispatch_r<G_SOFT, DT_F32, 2, ROUTE_LDG, false, true>(c, p, s);
        case 4: return dispatch_r<G_SOFT, DT_F32, 4, ROUTE_LDG, false, true>(c, p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rct

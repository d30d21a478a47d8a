// Allocation-free backprojection entry point.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework which owns the device memory pool and forbids allocations made
// behind its back, latency-critical loops where cudaMalloc / cudaFree would
// synchronise the whole device and stall every other stream, and embedded or
// certified pipelines that fix their memory budget at start-up.  For them
// this file offers one entry point that needs no context and allocates
// nothing: the caller passes FP32 projections and an FP32 volume; the views
// are narrowed to FP16 into a fixed scratch array that is part of the loaded
// library, and the FP16 predicated-load backprojection kernel reads them
// from there.
//
// The scratch is a file-scope __device__ array of kScratchValues 16-bit
// values (32 MiB).  Every GPU that loads the library holds it until the
// process exits.  Host code must not use the array's name as an address (on
// the host it is only a stand-in); its device address is looked up with
// cudaGetSymbolAddress on the first call made while that device is current,
// and only a successful lookup is kept (a failed one is tried again by the
// next call).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/rct.h"
#include "rct_bp_kernel.cuh"
#include "rct_internal.h"

namespace {

constexpr size_t kScratchValues = size_t(16) << 20;   // 16 Mi FP16 values = 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned short g_f16_scratch[kScratchValues];

std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices];

// Device address of the scratch array on the current device.  A successful lookup is kept for the
// device; a failed one (for instance a first call made while a stream is being captured) is not, so a
// later call looks again.
cudaError_t scratch_address(int dev, unsigned short **out) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *a = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&a, g_f16_scratch);
        if (e != cudaSuccess || !a) {
            (void)cudaGetLastError();
            *out = nullptr;
            return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
        }
        g_scratch_addr[dev] = a;
    }
    *out = static_cast<unsigned short *>(g_scratch_addr[dev]);
    return cudaSuccess;
}

// FP32 -> FP16 (round to nearest even) into the scratch, one value per thread-iteration: the
// source offset of a batch has no alignment guarantee beyond 4 bytes.
__global__ void narrow_to_scratch(const float *__restrict__ src, unsigned short *__restrict__ dst, size_t n) {
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = __half_as_ushort(__float2half_rn(src[i]));
}

}  // namespace

extern "C" rct_status rct_backproject_f16_noalloc(int L, int det_w, int det_h, const double *matrices, int n,
                                                  const double origin[3], const double spacing[3],
                                                  const float *d_proj, float *d_volume, int accumulate,
                                                  void *stream) {
    using namespace rct;
    if (L <= 0 || L > 2048 || det_w <= 0 || det_h <= 0 || n < 0)
        return rct_internal_fail(RCT_EINVAL, "rct_backproject_f16_noalloc: L=%d det=%dx%d n=%d out of range", L,
                                 det_w, det_h, n);
    if (!matrices || !origin || !spacing || !d_volume || (n > 0 && !d_proj))
        return rct_internal_fail(RCT_EINVAL, "rct_backproject_f16_noalloc: null pointer");
    const size_t px = static_cast<size_t>(det_w) * det_h;
    if (px > kScratchValues)
        return rct_internal_fail(RCT_EINVAL,
                                 "rct_backproject_f16_noalloc: a %dx%d view needs %zu scratch values; the fixed "
                                 "scratch holds %zu (32 MiB of FP16)", det_w, det_h, px, kScratchValues);
    if (n == 0) return RCT_OK;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return rct_internal_fail(RCT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return rct_internal_fail(RCT_ENOTSUP, "device %d beyond %d", dev, kMaxDevices);
    // the detector limits of rct_create (the texture-gather extents of the device)
    int max_w = 0, max_h = 0;
    cudaDeviceGetAttribute(&max_w, cudaDevAttrMaxTexture2DGatherWidth, dev);
    cudaDeviceGetAttribute(&max_h, cudaDevAttrMaxTexture2DGatherHeight, dev);
    if ((max_w > 0 && det_w > max_w) || (max_h > 0 && det_h > max_h))
        return rct_internal_fail(RCT_EINVAL, "rct_backproject_f16_noalloc: detector %dx%d exceeds %dx%d", det_w, det_h,
                                 max_w, max_h);
    unsigned short *scratch = nullptr;
    e = scratch_address(dev, &scratch);
    if (e != cudaSuccess || !scratch)
        return rct_internal_fail(RCT_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));

    for (int v = 0; v < n; ++v) {            // reject bad geometry before any work is enqueued
        double fold[12];
        int shift[2];
        rct_status st = rct_fold_geometry(L, 1, matrices + 12 * static_cast<size_t>(v), origin, spacing, fold, shift);
        if (st != RCT_OK) return st;
    }

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int per_batch = static_cast<int>(std::min<size_t>(KMAX, kScratchValues / px));
    LaunchConfig lc{};
    lc.gather = G_SOFT;
    lc.dtype = DT_F16;
    lc.xv = 1;
    lc.zrun = 4;
    lc.bx = 32;
    lc.by = 8;
    BpParams p{};
    p.vol = d_volume;
#ifdef RCT_CHECK_BOUNDS
    p.vol_elems = static_cast<long long>(L) * L * L;
#endif
    p.L = L;
    p.W = det_w;
    p.H = det_h;
    p.cen = 0.5f * (L - 1);
    p.tex_zrun = 0;                       // predicated loads from the linear FP16 scratch
    for (int b = 0; b < n; b += per_batch) {
        const int kb = std::min(per_batch, n - b);
        // The whole batch region of the scratch is rewritten before the kernel reads it; nothing
        // in the scratch needs to start at zero.
        const size_t count = static_cast<size_t>(kb) * px;
        const int blocks = static_cast<int>(std::min<size_t>((count + 255) / 256, 4096));
        narrow_to_scratch<<<blocks, 256, 0, s>>>(d_proj + static_cast<size_t>(b) * px, scratch, count);
        e = cudaGetLastError();
        if (e != cudaSuccess) return rct_internal_fail(RCT_ECUDA, "FP16 narrowing into scratch: %s", cudaGetErrorString(e));
        p.K = kb;
        p.accumulate = (b == 0) ? (accumulate ? 1 : 0) : 1;
        for (int k = 0; k < kb; ++k) {
            double fold[12];
            int shift[2];
            rct_status st = rct_fold_geometry(L, 1, matrices + 12 * static_cast<size_t>(b + k), origin, spacing,
                                              fold, shift);
            if (st != RCT_OK) return st;
            ViewParams &vp = p.view[k];
            set_view_geometry(&vp, fold, shift[0], shift[1]);
            vp.tex = 0;
            vp.img = scratch + static_cast<size_t>(k) * px;
        }
        // global frame: this entry point keeps no per-view geometry table on the device
        e = launch_one<G_SOFT, DT_F16, 1, 4, ROUTE_LDG, false>(lc, p, s);
        if (e != cudaSuccess) return rct_internal_fail(RCT_ECUDA, "backprojection launch: %s", cudaGetErrorString(e));
    }
    return RCT_OK;
}

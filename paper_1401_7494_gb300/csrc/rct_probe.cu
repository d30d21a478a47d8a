// Throughput probes that give the measured peaks the backprojection is compared against
// (the role of likwid-bench's gather microbenchmarks in the paper, Section "Gather performance").
//
// rct_probe_texture: every thread issues `iters` texture fetches of one kind (tld4 gather,
// point fetch, or filtered bilinear fetch) from a small 2D texture that stays resident in the
// texture cache, with a configurable lane-to-lane coordinate stride, and as little arithmetic
// as the fetch results need to stay live.  Result: fetches per second over the whole GPU.
// rct_probe_update_stream: a read-modify-write stream over a large buffer (the paper's
// "Node Update" benchmark, Table 1): bytes read + written per second.
// rct_probe_l1_bandwidth: coalesced 16-byte loads that hit L1: the load data path's bytes per second.
// This file builds the measurement library librct_bench.so (include/rct_bench.h), not librct.so.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "../../include/rct_bench.h"

namespace {

constexpr int kTexSide = 256;   // 256 x 256 texels: 256 KB FP32, within the 256 KB L1/texture cache

template <int MODE>
__global__ void __launch_bounds__(256) tex_probe_kernel(cudaTextureObject_t tex, int iters, float stride,
                                                        float step, float *sink) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    float x = 8.0f + lane * stride + (warp & 7) * 3.0f;
    float y = 8.0f + ((warp >> 3) & 63) * 2.0f;
    float acc = 0.0f;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        if constexpr (MODE == 0) {
            const float4 g = tex2Dgather<float4>(tex, x, y, 0);
            acc += (g.x + g.y) + (g.z + g.w);
        } else if constexpr (MODE == 1) {
            acc += tex2D<float>(tex, x, y);
        } else {
            acc += tex2D<float>(tex, x, y);
        }
        y += step;
        y = (y > kTexSide - 16.0f) ? y - (kTexSide - 32.0f) : y;
    }
    if (acc == 1.2345e-30f) sink[0] = acc;
}

// Four predicated read-only loads of a 2x2 cell from a cache-resident linear image, the
// load/store route of the backprojection kernel; same lane layout as tex_probe_kernel.
__global__ void __launch_bounds__(256) ldg4_probe_kernel(const float *__restrict__ img, int iters, float stride,
                                                         float step, float *sink) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    float x = 8.0f + lane * stride + (warp & 7) * 3.0f;
    float y = 8.0f + ((warp >> 3) & 63) * 2.0f;
    float acc = 0.0f;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        const int i0 = __float2int_rd(x), j0 = __float2int_rd(y);
        const bool ok = static_cast<unsigned>(i0) < static_cast<unsigned>(kTexSide - 1) &&
                        static_cast<unsigned>(j0) < static_cast<unsigned>(kTexSide - 1);
        const float *r0 = img + j0 * kTexSide + i0;
        const float a = ok ? __ldg(r0) : 0.f, b = ok ? __ldg(r0 + 1) : 0.f;
        const float c = ok ? __ldg(r0 + kTexSide) : 0.f, d = ok ? __ldg(r0 + kTexSide + 1) : 0.f;
        acc += (a + b) + (c + d);
        y += step;
        y = (y > kTexSide - 16.0f) ? y - (kTexSide - 32.0f) : y;
    }
    if (acc == 1.2345e-30f) sink[0] = acc;
}

// The backprojection's plain-load gather with a given warp footprint: lane l fetches the 2x2 cell at
// (x + du[l], y + dv[l]) with four 4-byte loads from a 256 x 128 FP32 image (128 KiB: L1 resident), and
// every fetch moves the warp's footprint by (step_u, step_v), as the next voxel of a z-run does.  Offsets
// come from the caller (a real warp's projected voxels), so the rate is that access pattern's ceiling.
constexpr int kPatW = 256, kPatH = 128;

__global__ void __launch_bounds__(256) pattern_probe_kernel(const float *__restrict__ img, const float2 *__restrict__ duv,
                                                            int iters, float step_u, float step_v, float *sink) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const float2 o = duv[lane];
    float x = 16.0f + o.x + (warp & 15) * 2.0f;
    float y = 8.0f + o.y + ((warp >> 4) & 15) * 1.0f;
    float acc = 0.0f;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        const int i0 = __float2int_rd(x), j0 = __float2int_rd(y);
        const bool ok = static_cast<unsigned>(i0) < static_cast<unsigned>(kPatW - 1) &&
                        static_cast<unsigned>(j0) < static_cast<unsigned>(kPatH - 1);
        const float *r0 = img + j0 * kPatW + i0;
        const float a = ok ? __ldg(r0) : 0.f, b = ok ? __ldg(r0 + 1) : 0.f;
        const float c = ok ? __ldg(r0 + kPatW) : 0.f, d = ok ? __ldg(r0 + kPatW + 1) : 0.f;
        acc += (a + b) + (c + d);
        x += step_u;
        y += step_v;
        x = (x > kPatW - 24.0f) ? x - (kPatW - 48.0f) : (x < 24.0f ? x + (kPatW - 48.0f) : x);
        y = (y > kPatH - 12.0f) ? y - (kPatH - 24.0f) : (y < 12.0f ? y + (kPatH - 24.0f) : y);
    }
    if (acc == 1.2345e-30f) sink[0] = acc;
}

// Staged-layout loads over a detector-sized buffer (larger than L1, resident in L2): one 16-byte
// quad (PAIRS = false) or two consecutive 8-byte pairs (PAIRS = true) per fetch, same lane layout.
constexpr int kLayoutW = 1280, kLayoutH = 1024;

template <bool PAIRS>
__global__ void __launch_bounds__(256) layout_probe_kernel(const float4 *__restrict__ quads, int iters, float stride,
                                                           float step, float *sink) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    float x = 8.0f + lane * stride + (warp % 11) * 100.0f;
    float y = 8.0f + ((warp / 11) % 97) * 9.0f;
    float acc = 0.0f;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        const int ix = __float2int_rd(x), jy = __float2int_rd(y);
        const unsigned e = static_cast<unsigned>(jy) * kLayoutW + static_cast<unsigned>(ix);
        if constexpr (PAIRS) {
            const float2 *pp = reinterpret_cast<const float2 *>(quads) + e;
            const float2 a = __ldg(pp), b = __ldg(pp + 1);
            acc += (a.x + a.y) + (b.x + b.y);
        } else {
            const float4 v = __ldg(quads + e);
            acc += (v.x + v.y) + (v.z + v.w);
        }
        y += step;
        y = (y > kLayoutH - 16.0f) ? y - (kLayoutH - 32.0f) : y;
    }
    if (acc == 1.2345e-30f) sink[0] = acc;
}

__global__ void update_stream_kernel(float4 *__restrict__ a, size_t n4, float s) {
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 v = a[i];
        v.x += s; v.y += s; v.z += s; v.w += s;
        a[i] = v;
    }
}

// Every block reads its own 16 KiB block of `buf` over and over with coalesced 16-byte loads (a
// warp's load covers 512 contiguous bytes; the block's eight warps start 2 KiB apart), so after
// the first pass every load hits L1 (eight resident blocks hold 128 KiB per SM).  The loaded
// words are folded with XORs (two three-input logic operations per load) into a sink.
constexpr int kL1Block = 16 * 1024;

__global__ void __launch_bounds__(256) l1_probe_kernel(const uint4 *__restrict__ buf, int iters, unsigned *sink) {
    const uint4 *base = buf + static_cast<size_t>(blockIdx.x) * (kL1Block / 16);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int at = warp * 128 + lane;                        // in 16-byte units; 1024 units per block
    unsigned x = 0;
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {
        const uint4 v = __ldg(base + at);
        x ^= v.x ^ v.y ^ v.z ^ v.w;
        at = (at + 32) & (kL1Block / 16 - 1);
    }
    if (x == 0x9e3779b9u) sink[0] = x;                 // keeps the loads live; practically never taken
}

// Scattered sector loads served by L2: every lane walks its own pseudo-random sequence of 32-byte
// sectors of a 64 MiB buffer (far larger than L1, well inside L2) and loads 16 bytes from each with an
// L1-bypassing load, so each load of a warp asks L2 for 32 distinct sectors.
constexpr size_t kL2Bytes = size_t(64) << 20;

__global__ void __launch_bounds__(256) l2_sector_probe_kernel(const uint4 *__restrict__ buf, int iters, unsigned *sink) {
    unsigned s = 2654435761u * (blockIdx.x * blockDim.x + threadIdx.x + 1);
    unsigned x = 0;
    constexpr unsigned kSectors = static_cast<unsigned>(kL2Bytes / 32);
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {
        s = s * 1664525u + 1013904223u;                     // LCG: a new sector per load
        const uint4 v = __ldcg(buf + 2 * static_cast<size_t>(s % kSectors));
        x ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (x == 0x9e3779b9u) sink[0] = x;
}

}  // namespace

extern "C" {

// mode: 0 = tld4 gather (point texture), 1 = point fetch, 2 = bilinear filtered fetch,
// 3 = four predicated global loads of the 2x2 cell (FP32 only; the load/store route),
// 4 = one 16-byte quad load, 5 = two 8-byte pair loads (FP32 layouts over a 1280 x 1024 buffer).
// dtype: RCT_PROJ_F32 or RCT_PROJ_F16 texels.  stride_px: x distance between neighbouring lanes,
// step_px: y advance per fetch.  Writes fetches per second (whole GPU) to *rate.
RCT_API rct_status rct_probe_texture(int mode, int dtype, float stride_px, float step_px, int iters,
                                     double *rate) {
    if (!rate || mode < 0 || mode > 5 || iters <= 0 || (dtype != RCT_PROJ_F32 && dtype != RCT_PROJ_F16))
        return RCT_EINVAL;
    if (mode >= 3 && dtype != RCT_PROJ_F32) return RCT_EINVAL;
    if (stride_px < 0.0f || stride_px > 10.0f || step_px < 0.0f || step_px > 8.0f) return RCT_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RCT_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaChannelFormatDesc fmt = (dtype == RCT_PROJ_F16) ? cudaCreateChannelDescHalf()
                                                        : cudaCreateChannelDesc(32, 0, 0, 0, cudaChannelFormatKindFloat);
    cudaArray_t arr = nullptr;
    cudaTextureObject_t tex = 0;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rct_status st = RCT_ECUDA;
    do {
        if (cudaMallocArray(&arr, &fmt, kTexSide, kTexSide, mode == 0 ? cudaArrayTextureGather : 0) != cudaSuccess) break;
        // sink[0]: result sink; then a 256 x 256 float image (mode 3) or a 1280 x 1024 float4 layout buffer
        const size_t floats = 4 + static_cast<size_t>(kLayoutW) * kLayoutH * 4;
        if (cudaMalloc(&sink, sizeof(float) * floats) != cudaSuccess) break;
        if (cudaMemset(sink, 0, sizeof(float) * floats) != cudaSuccess) break;
        cudaResourceDesc rd{};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = arr;
        cudaTextureDesc td{};
        td.addressMode[0] = td.addressMode[1] = cudaAddressModeBorder;
        td.filterMode = (mode == 2) ? cudaFilterModeLinear : cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        if (cudaCreateTextureObject(&tex, &rd, &td, nullptr) != cudaSuccess) break;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) break;
        const int block = 256, grid = sms * 8;
        auto run = [&]() {
            if (mode == 3) ldg4_probe_kernel<<<grid, block>>>(sink + 4, iters, stride_px, step_px, sink);
            else if (mode == 4)
                layout_probe_kernel<false><<<grid, block>>>(reinterpret_cast<const float4 *>(sink + 4), iters, stride_px, step_px, sink);
            else if (mode == 5)
                layout_probe_kernel<true><<<grid, block>>>(reinterpret_cast<const float4 *>(sink + 4), iters, stride_px, step_px, sink);
            else if (mode == 0) tex_probe_kernel<0><<<grid, block>>>(tex, iters, stride_px, step_px, sink);
            else if (mode == 1) tex_probe_kernel<1><<<grid, block>>>(tex, iters, stride_px, step_px, sink);
            else tex_probe_kernel<2><<<grid, block>>>(tex, iters, stride_px, step_px, sink);
        };
        run();
        if (cudaDeviceSynchronize() != cudaSuccess) break;
        float best = 1e30f;
        for (int r = 0; r < 3; ++r) {
            cudaEventRecord(e0);
            run();
            cudaEventRecord(e1);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = ms < best ? ms : best;
        }
        *rate = static_cast<double>(grid) * block * iters / (best * 1e-3);
        st = RCT_OK;
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (tex) cudaDestroyTextureObject(tex);
    if (arr) cudaFreeArray(arr);
    if (sink) cudaFree(sink);
    return st;
}

RCT_API rct_status rct_probe_gather_pattern(const float *lane_uv, float step_u, float step_v, int iters,
                                            double *rate) {
    if (!rate || !lane_uv || iters < 16) return RCT_EINVAL;
    for (int l = 0; l < 64; ++l)
        if (!(lane_uv[l] >= -100.0f && lane_uv[l] <= 100.0f)) return RCT_EINVAL;
    if (!(step_u >= -16.0f && step_u <= 16.0f && step_v >= -16.0f && step_v <= 16.0f)) return RCT_EINVAL;
    // the footprint (offsets, 16 warps' starts) must stay inside the image: |du| <= 100 within a width of
    // 256 leaves room; rows: |dv| <= 100 does not fit 128 rows, so narrower row spans are required
    float vmin = 0.f, vmax = 0.f;
    for (int l = 0; l < 32; ++l) {
        vmin = lane_uv[2 * l + 1] < vmin ? lane_uv[2 * l + 1] : vmin;
        vmax = lane_uv[2 * l + 1] > vmax ? lane_uv[2 * l + 1] : vmax;
    }
    if (vmax - vmin > 40.0f) return RCT_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RCT_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int block = 256, grid = sms * 8;
    float *img = nullptr;
    float2 *duv = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rct_status st = RCT_ECUDA;
    do {
        if (cudaMalloc(&img, sizeof(float) * (kPatW * kPatH + 4)) != cudaSuccess) { st = RCT_ENOMEM; break; }
        if (cudaMalloc(&duv, sizeof(float2) * 32) != cudaSuccess) { st = RCT_ENOMEM; break; }
        if (cudaMemset(img, 0, sizeof(float) * (kPatW * kPatH + 4)) != cudaSuccess) break;
        // shift the offsets so that the lowest row of the footprint is row 0 of the pattern
        float2 h[32];
        for (int l = 0; l < 32; ++l) h[l] = make_float2(lane_uv[2 * l], lane_uv[2 * l + 1] - vmin);
        if (cudaMemcpy(duv, h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess) break;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) break;
        float *sink = img + kPatW * kPatH;
        pattern_probe_kernel<<<grid, block>>>(img, duv, iters, step_u, step_v, sink);
        if (cudaDeviceSynchronize() != cudaSuccess) break;
        float best = 1e30f;
        for (int r = 0; r < 3; ++r) {
            cudaEventRecord(e0);
            pattern_probe_kernel<<<grid, block>>>(img, duv, iters, step_u, step_v, sink);
            cudaEventRecord(e1);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = ms < best ? ms : best;
        }
        if (best >= 1e29f) break;
        *rate = static_cast<double>(grid) * block * iters / (best * 1e-3);
        st = RCT_OK;
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (img) cudaFree(img);
    if (duv) cudaFree(duv);
    return st;
}

RCT_API rct_status rct_probe_l1_bandwidth(int iters, double *rate) {
    if (!rate || iters < 64) return RCT_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RCT_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int block = 256, grid = sms * 8;
    uint4 *buf = nullptr;
    unsigned *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rct_status st = RCT_ECUDA;
    do {
        if (cudaMalloc(&buf, static_cast<size_t>(grid) * kL1Block) != cudaSuccess) { st = RCT_ENOMEM; break; }
        if (cudaMalloc(&sink, sizeof(unsigned)) != cudaSuccess) { st = RCT_ENOMEM; break; }
        if (cudaMemset(buf, 1, static_cast<size_t>(grid) * kL1Block) != cudaSuccess) break;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) break;
        l1_probe_kernel<<<grid, block>>>(buf, iters, sink);
        if (cudaDeviceSynchronize() != cudaSuccess) break;
        float best = 1e30f;
        for (int r = 0; r < 5; ++r) {
            cudaEventRecord(e0);
            l1_probe_kernel<<<grid, block>>>(buf, iters, sink);
            cudaEventRecord(e1);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = ms < best ? ms : best;
        }
        if (best >= 1e29f) break;
        *rate = static_cast<double>(grid) * block * iters * 16.0 / (best * 1e-3);
        st = RCT_OK;
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    return st;
}

RCT_API rct_status rct_probe_l2_sectors(int iters, double *rate) {
    if (!rate || iters < 64) return RCT_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RCT_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int block = 256, grid = sms * 8;
    uint4 *buf = nullptr;
    unsigned *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rct_status st = RCT_ECUDA;
    do {
        if (cudaMalloc(&buf, kL2Bytes) != cudaSuccess) { st = RCT_ENOMEM; break; }
        if (cudaMalloc(&sink, sizeof(unsigned)) != cudaSuccess) { st = RCT_ENOMEM; break; }
        if (cudaMemset(buf, 1, kL2Bytes) != cudaSuccess) break;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) break;
        l2_sector_probe_kernel<<<grid, block>>>(buf, iters, sink);
        if (cudaDeviceSynchronize() != cudaSuccess) break;
        float best = 1e30f;
        for (int r = 0; r < 5; ++r) {
            cudaEventRecord(e0);
            l2_sector_probe_kernel<<<grid, block>>>(buf, iters, sink);
            cudaEventRecord(e1);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = ms < best ? ms : best;
        }
        if (best >= 1e29f) break;
        *rate = static_cast<double>(grid) * block * iters / (best * 1e-3);
        st = RCT_OK;
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    return st;
}

// Read-modify-write stream over `bytes` of device memory (allocated here); writes bytes moved per second.
RCT_API rct_status rct_probe_update_stream(size_t bytes, double *rate) {
    if (!rate || bytes < (1u << 20)) return RCT_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RCT_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float4 *a = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rct_status st = RCT_ECUDA;
    const size_t n4 = bytes / sizeof(float4);
    do {
        if (cudaMalloc(&a, n4 * sizeof(float4)) != cudaSuccess) { st = RCT_ENOMEM; break; }
        if (cudaMemset(a, 0, n4 * sizeof(float4)) != cudaSuccess) break;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) break;
        const int block = 512, grid = sms * 4;
        update_stream_kernel<<<grid, block>>>(a, n4, 1.0f);
        if (cudaDeviceSynchronize() != cudaSuccess) break;
        float best = 1e30f;
        for (int r = 0; r < 5; ++r) {
            cudaEventRecord(e0);
            update_stream_kernel<<<grid, block>>>(a, n4, 1.0f);
            cudaEventRecord(e1);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = ms < best ? ms : best;
        }
        *rate = 2.0 * static_cast<double>(n4 * sizeof(float4)) / (best * 1e-3);
        st = RCT_OK;
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (a) cudaFree(a);
    return st;
}

}  // extern "C"

// Element-type conversion of projections (staging for the reduced-precision variants).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rct_internal.h"

namespace rct {

namespace {

// Round-to-nearest-even narrowing of FP32 values; four per thread when aligned.
template <int DT>
__global__ void narrow_kernel(const float *__restrict__ src, unsigned short *__restrict__ dst, size_t n) {
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t q = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; q * 4 < n; q += stride) {
        const size_t i = q * 4;
        float v[4];
        if (i + 4 <= n) {
            const float4 t = *reinterpret_cast<const float4 *>(src + i);
            v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else {
            for (int k = 0; k < 4; ++k) v[k] = (i + k < n) ? src[i + k] : 0.0f;
        }
        unsigned short o[4];
        for (int k = 0; k < 4; ++k) {
            if constexpr (DT == DT_F16) o[k] = __half_as_ushort(__float2half_rn(v[k]));
            else o[k] = __bfloat16_as_ushort(__float2bfloat16_rn(v[k]));
        }
        if (i + 4 <= n) {
            uint2 packed;
            packed.x = static_cast<unsigned>(o[0]) | (static_cast<unsigned>(o[1]) << 16);
            packed.y = static_cast<unsigned>(o[2]) | (static_cast<unsigned>(o[3]) << 16);
            *reinterpret_cast<uint2 *>(dst + i) = packed;
        } else {
            for (int k = 0; k < 4 && i + k < n; ++k) dst[i + k] = o[k];
        }
    }
}

// vol[i] += part[i] + part[stride + i] + ... in that order (the view split's partial volumes).
__global__ void add_partials_kernel(float *__restrict__ vol, const float *__restrict__ part, size_t n, size_t stride,
                                    int parts) {
    const size_t step = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += step) {
        float v = vol[i];
        for (int k = 0; k < parts; ++k) v += part[k * stride + i];
        vol[i] = v;
    }
}

__global__ void widen_bf16_kernel(const unsigned short *__restrict__ src, float *__restrict__ dst, size_t n) {
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = __uint_as_float(static_cast<unsigned>(src[i]) << 16);
}

int grid_for(size_t work, int block) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t want = (work + block - 1) / block;
    const size_t cap = static_cast<size_t>(sms) * 8;
    return static_cast<int>(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_convert(const float *src, void *dst, size_t n, int dtype, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (dtype == DT_F32) return cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
    // 16-byte vector loads need 16-byte aligned sources, 8-byte stores 8-byte aligned destinations.
    if ((reinterpret_cast<uintptr_t>(src) & 15) || (reinterpret_cast<uintptr_t>(dst) & 7)) return cudaErrorMisalignedAddress;
    const int block = 256;
    const int grid = grid_for((n + 3) / 4, block);
    auto *d = static_cast<unsigned short *>(dst);
    if (dtype == DT_F16) narrow_kernel<DT_F16><<<grid, block, 0, s>>>(src, d, n);
    else if (dtype == DT_BF16) narrow_kernel<DT_BF16><<<grid, block, 0, s>>>(src, d, n);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_add_partials(float *vol, const float *part, size_t n, size_t stride, int parts, cudaStream_t s) {
    if (n == 0 || parts <= 0) return cudaSuccess;
    const int block = 256;
    add_partials_kernel<<<grid_for(n, block), block, 0, s>>>(vol, part, n, stride, parts);
    return cudaGetLastError();
}

cudaError_t launch_widen_bf16(const uint16_t *src, float *dst, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int block = 256;
    widen_bf16_kernel<<<grid_for(n, block), block, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace rct

namespace rct {

namespace {

template <typename T>
__device__ __forceinline__ T px_or_zero(const T *img, int W, int H, int i, int j) {
    return (static_cast<unsigned>(i) < static_cast<unsigned>(W) && static_cast<unsigned>(j) < static_cast<unsigned>(H))
               ? img[static_cast<size_t>(j) * W + i] : T(0);
}

// The staging kernels below take one view per blockIdx.z: view z reads img + z * W * H and writes its
// layout at q + z * (elements of one staged image), so a batch of views that sit next to each other in
// memory, and go to consecutive staging slots, is staged by one launch.
#define RCT_VIEW_OFFSETS(ELEMS)                                                  \
    img += static_cast<size_t>(blockIdx.z) * W * H;                             \
    q += static_cast<size_t>(blockIdx.z) * (ELEMS);

// One thread per padded element (jy, ix): gathers the 2x2 cell with corner (ix - 1, jy - 1).
__global__ void stage_quads_f32(const float *__restrict__ img, float4 *__restrict__ q, int W, int H) {
    RCT_VIEW_OFFSETS(static_cast<size_t>(W + 1) * (H + 1))
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int jy = blockIdx.y;
    if (ix > W) return;
    const int i0 = ix - 1, j0 = jy - 1;
    q[static_cast<size_t>(jy) * (W + 1) + ix] =
        make_float4(px_or_zero(img, W, H, i0, j0), px_or_zero(img, W, H, i0, j0 + 1),
                    px_or_zero(img, W, H, i0 + 1, j0), px_or_zero(img, W, H, i0 + 1, j0 + 1));
}

__global__ void stage_quads_u16(const unsigned short *__restrict__ img, uint2 *__restrict__ q, int W, int H) {
    RCT_VIEW_OFFSETS(static_cast<size_t>(W + 1) * (H + 1))
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int jy = blockIdx.y;
    if (ix > W) return;
    const int i0 = ix - 1, j0 = jy - 1;
    const unsigned a = px_or_zero(img, W, H, i0, j0), c = px_or_zero(img, W, H, i0, j0 + 1);
    const unsigned b = px_or_zero(img, W, H, i0 + 1, j0), d = px_or_zero(img, W, H, i0 + 1, j0 + 1);
    q[static_cast<size_t>(jy) * (W + 1) + ix] = make_uint2(a | (c << 16), b | (d << 16));
}

// One thread per padded pair (jy, ix): (I[jy-1][ix-1], I[jy][ix-1]), zero off the image.
__global__ void stage_pairs_f32(const float *__restrict__ img, float2 *__restrict__ q, int W, int H) {
    RCT_VIEW_OFFSETS(static_cast<size_t>(W + 2) * (H + 1))
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int jy = blockIdx.y;
    if (ix > W + 1) return;
    q[static_cast<size_t>(jy) * (W + 2) + ix] =
        make_float2(px_or_zero(img, W, H, ix - 1, jy - 1), px_or_zero(img, W, H, ix - 1, jy));
}

__global__ void stage_pairs_u16(const unsigned short *__restrict__ img, unsigned *__restrict__ q, int W, int H) {
    RCT_VIEW_OFFSETS(static_cast<size_t>(W + 2) * (H + 1))
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int jy = blockIdx.y;
    if (ix > W + 1) return;
    const unsigned a = px_or_zero(img, W, H, ix - 1, jy - 1), c = px_or_zero(img, W, H, ix - 1, jy);
    q[static_cast<size_t>(jy) * (W + 2) + ix] = a | (c << 16);
}

// One thread per padded element (jy, ix): the cell with corner (ix - 1, jy - 1) as (a, c, b - a, d - c),
// a = I[j0][i0], c = I[j0+1][i0], b = I[j0][i0+1], d = I[j0+1][i0+1], zero off the image.
__global__ void stage_dquads_f32(const float *__restrict__ img, float4 *__restrict__ q, int W, int H) {
    RCT_VIEW_OFFSETS(static_cast<size_t>(W + 1) * (H + 1))
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int jy = blockIdx.y;
    if (ix > W) return;
    const int i0 = ix - 1, j0 = jy - 1;
    const float a = px_or_zero(img, W, H, i0, j0), c = px_or_zero(img, W, H, i0, j0 + 1);
    const float b = px_or_zero(img, W, H, i0 + 1, j0), d = px_or_zero(img, W, H, i0 + 1, j0 + 1);
    q[static_cast<size_t>(jy) * (W + 1) + ix] = make_float4(a, c, __fsub_rn(b, a), __fsub_rn(d, c));
}

}  // namespace

cudaError_t launch_stage_dquads(const float *src, void *dst, int W, int H, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const dim3 block(256), grid((W + 1 + 255) / 256, H + 1, n);
    stage_dquads_f32<<<grid, block, 0, s>>>(src, static_cast<float4 *>(dst), W, H);
    return cudaGetLastError();
}

size_t pair_bytes(int W, int H, int dtype) {
    return static_cast<size_t>(W + 2) * (H + 1) * (dtype == DT_F32 ? 8 : 4);
}

cudaError_t launch_stage_pairs(const void *src, void *dst, int W, int H, int dtype, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const dim3 block(256), grid((W + 2 + 255) / 256, H + 1, n);
    if (dtype == DT_F32)
        stage_pairs_f32<<<grid, block, 0, s>>>(static_cast<const float *>(src), static_cast<float2 *>(dst), W, H);
    else
        stage_pairs_u16<<<grid, block, 0, s>>>(static_cast<const unsigned short *>(src), static_cast<unsigned *>(dst), W, H);
    return cudaGetLastError();
}

size_t quad_bytes(int W, int H, int dtype) {
    return static_cast<size_t>(W + 1) * (H + 1) * (dtype == DT_F32 ? 16 : 8);
}

cudaError_t launch_stage_quads(const void *src, void *dst, int W, int H, int dtype, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const dim3 block(256), grid((W + 1 + 255) / 256, H + 1, n);
    if (dtype == DT_F32)
        stage_quads_f32<<<grid, block, 0, s>>>(static_cast<const float *>(src), static_cast<float4 *>(dst), W, H);
    else
        stage_quads_u16<<<grid, block, 0, s>>>(static_cast<const unsigned short *>(src), static_cast<uint2 *>(dst), W, H);
    return cudaGetLastError();
}

}  // namespace rct

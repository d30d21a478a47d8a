// FDK pre-processing of raw projections on the device: cosine weighting and row-wise ramp filtering.
//
// RabbitCT ships projections that are already weighted and filtered (Section "RabbitCT
// Benchmark"); a scanner delivers raw line integrals.  For every view and pixel (i, j):
//
//   cosine weight   p'(i, j) = p(i, j) * D / sqrt(D^2 + ((i - u0) tau)^2 + ((j - v0) tau)^2)
//   ramp filter     q(i, j)  = tau * sum_k h[i - k] p'(k, j),   k in [0, W)
//                   h[n]     = -2 / (pi^2 tau^2 (4 n^2 - 1))      (Shepp-Logan kernel)
//
// with D the source-detector distance, tau the pixel pitch and (u0, v0) the view's principal
// point.  The convolution is linear (zero outside the row).
//
// One block filters two rows of one view: they are packed as the real and imaginary parts of one
// complex sequence of length N (a power of two, N >= 2W - 1, so the circular convolution of the
// zero-padded rows equals the linear one for the W outputs).  The sequence is transformed in shared
// memory by a Stockham FFT (self-sorting: natural order in and out), in passes of radix 16 (the
// last pass of radix 8, 4 or 2 when log2 N is not a multiple of 4): each thread reads 16 values,
// applies the pass's twiddles, does its small DFTs in registers and writes 16 values.  The product
// with the real, even spectrum of h (host FP64, tau / N folded in) is transformed back by the same
// forward routine through the identity IDFT(Y) = conj(DFT(conj(Y))) / N.  Because the spectrum is
// real, the real part of the result is the first row filtered and the imaginary part the second.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "rct_internal.h"

namespace rct {

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Twiddle table: tw[t] = exp(-2 pi i t / N), t in [0, N).
constexpr int kRadix = 16;          // values per thread and pass

// Shared-memory position of element i: one pad slot after every 16 elements, so that the radix-16
// pass whose threads each write 16 consecutive elements (lane stride 128 bytes) spreads its stores
// over the banks instead of hitting one.
__device__ __forceinline__ int sp(int i) { return i + (i >> 4); }

// exp(-2 pi i e / 16) for e in [0, 8): (cos, -sin) of multiples of pi / 8.
__device__ __forceinline__ float2 root16(int e) {
    constexpr float c1 = 0.923879532511286756f;   // cos(pi / 8)
    constexpr float s1 = 0.382683432365089772f;   // sin(pi / 8)
    constexpr float h = 0.707106781186547524f;    // sqrt(2) / 2
    switch (e) {
        case 0: return make_float2(1.0f, 0.0f);
        case 1: return make_float2(c1, -s1);
        case 2: return make_float2(h, -h);
        case 3: return make_float2(s1, -c1);
        case 4: return make_float2(0.0f, -1.0f);
        case 5: return make_float2(-s1, -c1);
        case 6: return make_float2(-h, -h);
        default: return make_float2(-c1, -s1);
    }
}

// In-register DFT of size R (a power of two, R <= 16) of v[0..R), natural order in and out:
// iterative radix-2 decimation in frequency, then the bit-reversal permutation (compile-time
// register renaming once unrolled).  The twiddles W_{2 half}^pos = exp(-2 pi i pos / (2 half)) are
// 16th roots of unity, constants once unrolled.
template <int R>
__device__ __forceinline__ void dft_regs(float2 (&v)[kRadix]) {
#pragma unroll
    for (int half = R / 2; half >= 1; half /= 2) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if ((i & half) == 0) {
                const int pos = i & (half - 1);
                const float2 a = v[i], b = v[i + half];
                v[i] = make_float2(a.x + b.x, a.y + b.y);
                const float2 d = make_float2(a.x - b.x, a.y - b.y);
                if (pos == 0) {
                    v[i + half] = d;
                } else {
                    v[i + half] = cmul(d, root16(pos * (8 / half)));
                }
            }
        }
    }
    float2 t[kRadix];
#pragma unroll
    for (int i = 0; i < R; ++i) t[i] = v[i];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        int r = 0;
#pragma unroll
        for (int b = 1, c = R / 2; b < R; b *= 2, c /= 2)
            if (i & b) r |= c;
        v[r] = t[i];
    }
}

// One Stockham pass of radix R over z (length N, in shared memory) with sub-transform length ns:
// each group j in [0, N / R) reads z[j + r N / R], twiddles by exp(-2 pi i r k / (ns R)) with
// k = j mod ns, takes the R-point DFT and writes to (j / ns) ns R + k + q ns.  The block's
// threads take 16 / R groups each.
template <int R>
__device__ __forceinline__ void stockham_pass(float2 *z, int log2n, int ns, const float2 *__restrict__ tw) {
    constexpr int G = kRadix / R;
    const int N = 1 << log2n;
    const int stride = N / R;
    float2 v[G][kRadix];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = threadIdx.x + g * blockDim.x;
#pragma unroll
        for (int r = 0; r < R; ++r) v[g][r] = z[sp(j + r * stride)];
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = threadIdx.x + g * blockDim.x;
        const int k = j & (ns - 1);
        const int tstep = k * (N / (ns * R));          // exp(-2 pi i r k / (ns R)) = tw[r * tstep]
        // powers-of-two r from the table, the others as products of those (at most three)
        float2 w[kRadix];
#pragma unroll
        for (int r = 1; r < R; ++r) {
            const int hb = 1 << (31 - __clz(r));       // highest set bit, a constant once unrolled
            w[r] = (r == hb) ? __ldg(&tw[r * tstep]) : cmul(w[hb], w[r - hb]);
            v[g][r] = cmul(v[g][r], w[r]);
        }
        dft_regs<R>(v[g]);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) z[sp(base + q * ns)] = v[g][q];
    }
    __syncthreads();
}

// Forward DFT of z (length N = 2^log2n, N >= 16) with N / 16 threads.
__device__ __forceinline__ void stockham_fft(float2 *z, int log2n, const float2 *__restrict__ tw) {
    int ns = 1, left = log2n;
    for (; left >= 4; left -= 4, ns *= 16) stockham_pass<16>(z, log2n, ns, tw);
    if (left == 3) stockham_pass<8>(z, log2n, ns, tw);
    else if (left == 2) stockham_pass<4>(z, log2n, ns, tw);
    else if (left == 1) stockham_pass<2>(z, log2n, ns, tw);
}

template <int OUT>
__device__ __forceinline__ void store_px(void *out, size_t at, float v) {
    if constexpr (OUT == DT_F32) {
        static_cast<float *>(out)[at] = v;
    } else if constexpr (OUT == DT_F16) {
        static_cast<__half *>(out)[at] = __float2half_rn(v);
    } else {
        static_cast<__nv_bfloat16 *>(out)[at] = __float2bfloat16_rn(v);
    }
}

template <int OUT>
__global__ void __launch_bounds__(1024) ramp_filter_kernel(const float *raw, void *out,   // may alias (in place)
                                                           int W, int H, int log2n,
                                                           const float2 *__restrict__ twiddle,
                                                           const float *__restrict__ spectrum,
                                                           const float2 *__restrict__ principal, float sdd,
                                                           float pitch) {
    extern __shared__ float2 z[];
    const int N = 1 << log2n;
    const int view = blockIdx.y;
    const int r0 = 2 * blockIdx.x, r1 = r0 + 1;
    const bool two = r1 < H;
    const size_t px = static_cast<size_t>(W) * H;
    const float *img = raw + static_cast<size_t>(view) * px;
    const float2 pp = principal[view];
    const float d2 = sdd * sdd;
    const float dv0 = (static_cast<float>(r0) - pp.y) * pitch;
    const float dv1 = (static_cast<float>(r1) - pp.y) * pitch;

    // cosine-weighted rows, zero padded
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        float a = 0.0f, b = 0.0f;
        if (k < W) {
            const float du = (static_cast<float>(k) - pp.x) * pitch;
            const float du2 = fmaf(du, du, d2);
            a = img[static_cast<size_t>(r0) * W + k] * (sdd * rsqrtf(fmaf(dv0, dv0, du2)));
            if (two) b = img[static_cast<size_t>(r1) * W + k] * (sdd * rsqrtf(fmaf(dv1, dv1, du2)));
        }
        z[sp(k)] = make_float2(a, b);
    }
    __syncthreads();
    stockham_fft(z, log2n, twiddle);
    // times the real spectrum, conjugated for the inverse
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const float hk = __ldg(&spectrum[k]);
        const float2 c = z[sp(k)];
        z[sp(k)] = make_float2(c.x * hk, -c.y * hk);
    }
    __syncthreads();
    stockham_fft(z, log2n, twiddle);
    // conj of the result: real part = first row, imaginary part = second row
    for (int k = threadIdx.x; k < W; k += blockDim.x) {
        const float2 v = z[sp(k)];
        store_px<OUT>(out, static_cast<size_t>(view) * px + static_cast<size_t>(r0) * W + k, v.x);
        if (two) store_px<OUT>(out, static_cast<size_t>(view) * px + static_cast<size_t>(r1) * W + k, -v.y);
    }
}

template <int OUT>
cudaError_t launch_filter_t(const FilterParams &f, const float *raw, void *out, int n, cudaStream_t s) {
    const size_t smem = sizeof(float2) * ((1u << f.log2n) + (1u << f.log2n) / 16);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(ramp_filter_kernel<OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    const dim3 grid((f.H + 1) / 2, n);
    ramp_filter_kernel<OUT><<<grid, (1 << f.log2n) / kRadix, smem, s>>>(raw, out, f.W, f.H, f.log2n, f.twiddle, f.spectrum, f.principal,
                                                    f.sdd, f.pitch);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ramp_filter(const FilterParams &f, const float *raw, void *out, int out_dtype, int n,
                               cudaStream_t s) {
    const size_t px = static_cast<size_t>(f.W) * f.H;
    const size_t out_size = out_dtype == DT_F32 ? 4 : 2;
    for (int b = 0; b < n; b += 65535) {                 // grid.y limit
        const int nb = n - b < 65535 ? n - b : 65535;
        FilterParams fb = f;
        fb.principal = f.principal + b;
        const float *rb = raw + static_cast<size_t>(b) * px;
        void *ob = static_cast<char *>(out) + static_cast<size_t>(b) * px * out_size;
        cudaError_t e;
        switch (out_dtype) {
            case DT_F32: e = launch_filter_t<DT_F32>(fb, rb, ob, nb, s); break;
            case DT_F16: e = launch_filter_t<DT_F16>(fb, rb, ob, nb, s); break;
            case DT_BF16: e = launch_filter_t<DT_BF16>(fb, rb, ob, nb, s); break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace rct

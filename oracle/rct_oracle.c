/*
 * rct_oracle.c -- plain, slow, FP64 reference backprojector.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes (the paper, Section "Algorithm", Listing 1 -- the
 * unoptimised RabbitCT reference backprojection, with its three parts):
 *
 *   for every view i and every voxel (x, y, z) of the L^3 volume:
 *     Part 1  world position  p = (O_x + x*MM_x, O_y + y*MM_y, O_z + z*MM_z)
 *             homogeneous detector position (u, v, w) = A_i * (p, 1)
 *             de-homogenise   ix = u / w,  iy = v / w
 *             integer cell    i0 = floor(ix), j0 = floor(iy)
 *             weights         fx = ix - i0,   fy = iy - j0
 *     Part 2  four taps g(i, j) = I_i[j * W + i] when 0 <= i < W and 0 <= j < H,
 *             otherwise 0 (the ray misses the detector)
 *     Part 3  bilinear  val = (1-fy)*((1-fx) g(i0,j0)   + fx g(i0+1,j0))
 *                           +    fy *((1-fx) g(i0,j0+1) + fx g(i0+1,j0+1))
 *             inverse-square weight and update  f[z][y][x] += val / (w*w)
 *
 * The volume is stored z-major with x fastest (index z*L*L + y*L + x), the
 * projections as n_views images of H rows by W columns, row-major.
 *
 * Readings where the listing is ambiguous (each one is also listed in the
 * design notes):
 *   - The listing truncates with an (int) cast.  That equals floor only for
 *     non-negative coordinates; for ix in (-1, 0) truncation would give
 *     i0 = 0 and a negative weight.  The oracle uses floor by default: the
 *     image is then the zero-extended grid, and the interpolant is continuous
 *     everywhere (this is also what the paper's zero-padded projection buffer,
 *     Section "SIMD Vectorization", computes).  index_rule = 1 takes the
 *     listing's truncation instead (RabbitCT compatibility): the cell is
 *     trunc(ix), and fx = ix - trunc(ix) is negative for negative ix, so the
 *     lerp extrapolates from the two taps at the image edge.
 *   - The listing's bound tests compare the row index with `width` and the
 *     column index with `height`, while it addresses rows with stride
 *     `width`.  The oracle tests the column index against W and the row
 *     index against H ("inside the projection image").
 *   - The listing reads the 3x4 matrix column-major (A[0], A[3], A[6], A[9]
 *     form u).  This oracle takes row-major matrices: A[r*4 + c].
 *   - Pixel (i, j) is the sample at detector coordinate (i, j) exactly, as
 *     the listing indexes the image with the integer cell directly.
 *   - The paper's CPU kernels use an approximate reciprocal (Section "SIMD
 *     Vectorization"); the oracle divides exactly in FP64.
 *   - w <= 0 (voxel at or behind the source) cannot occur in the scan
 *     geometries used here; the oracle reports it as an error.
 *
 * Precision of stored projections: rct_oracle_round_f16 / _bf16 give the
 * IEEE binary16 / bfloat16 value nearest to each FP32 input (ties to even),
 * so a backprojection of reduced-precision projections can be written as the
 * same FP64 backprojection of those rounded values.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_EBEHIND 2   /* larger codes win when several planes report */

#define ORACLE_INDEX_FLOOR 0
#define ORACLE_INDEX_TRUNC 1   /* the listing's (int) cast: toward zero (RabbitCT compatibility) */

/* One voxel, one view: returns the update val / w^2 of Listing 1 (Parts 1-3). */
static int oracle_update(const double *A, const float *img, int W, int H,
                         double wx, double wy, double wz, int index_rule, double *out)
{
    /* Part 1: projection and de-homogenisation */
    double u = A[0] * wx + A[1] * wy + A[2] * wz + A[3];
    double v = A[4] * wx + A[5] * wy + A[6] * wz + A[7];
    double w = A[8] * wx + A[9] * wy + A[10] * wz + A[11];
    if (!(w > 0.0)) return ORACLE_EBEHIND;
    double ix = u / w;
    double iy = v / w;
    double fi0 = floor(ix);
    double fj0 = floor(iy);
    if (index_rule == ORACLE_INDEX_TRUNC) {     /* (int) ix: toward zero, so fx < 0 for negative ix */
        fi0 = trunc(ix);
        fj0 = trunc(iy);
    }
    double fx = ix - fi0;
    double fy = iy - fj0;

    /* Part 2: four taps, zero outside the detector */
    double bl = 0.0, br = 0.0, tl = 0.0, tr = 0.0;
    if (fi0 >= -1.0 && fi0 < (double)W && fj0 >= -1.0 && fj0 < (double)H) {
        long i0 = (long)fi0;
        long j0 = (long)fj0;
        int in_i0 = (i0 >= 0 && i0 < W);
        int in_i1 = (i0 + 1 >= 0 && i0 + 1 < W);
        int in_j0 = (j0 >= 0 && j0 < H);
        int in_j1 = (j0 + 1 >= 0 && j0 + 1 < H);
        if (in_j0 && in_i0) bl = img[j0 * (long)W + i0];
        if (in_j0 && in_i1) br = img[j0 * (long)W + i0 + 1];
        if (in_j1 && in_i0) tl = img[(j0 + 1) * (long)W + i0];
        if (in_j1 && in_i1) tr = img[(j0 + 1) * (long)W + i0 + 1];
    }

    /* Part 3: bilinear interpolation and inverse-square weight */
    double valb = (1.0 - fx) * bl + fx * br;
    double valt = (1.0 - fx) * tl + fx * tr;
    double val = (1.0 - fy) * valb + fy * valt;
    *out = val / (w * w);
    return ORACLE_OK;
}

static int check_args(int L, int W, int H, int n_views, const double *A, const double *origin,
                      const double *spacing, const float *proj)
{
    if (L <= 0 || W <= 0 || H <= 0 || n_views < 0) return ORACLE_EINVAL;
    if (!A || !origin || !spacing || (!proj && n_views > 0)) return ORACLE_EINVAL;
    return ORACLE_OK;
}

/*
 * Backproject views [0, n_views) into z-planes [z_begin, z_end) of an L^3
 * volume.  `vol` holds (z_end - z_begin) planes of L*L doubles and is
 * accumulated into (the caller zeroes it for a fresh reconstruction).
 * Views are applied in order, one full pass over the planes per view, as the
 * reference module is called once per projection image.  Planes are
 * independent (Section "Implementation": one OpenMP task per voxel plane);
 * n_threads > 1 distributes them, which does not change any sum.
 */
int rct_oracle_backproject(int L, int W, int H, int n_views, const double *A,
                           const double *origin, const double *spacing, const float *proj,
                           int z_begin, int z_end, int n_threads, int index_rule, double *vol)
{
    int rc = check_args(L, W, H, n_views, A, origin, spacing, proj);
    if (rc) return rc;
    if (index_rule != ORACLE_INDEX_FLOOR && index_rule != ORACLE_INDEX_TRUNC) return ORACLE_EINVAL;
    if (z_begin < 0 || z_end > L || z_begin > z_end || !vol) return ORACLE_EINVAL;
    int status = ORACLE_OK;
    const long img_px = (long)W * H;
    const long plane = (long)L * L;
    for (int i = 0; i < n_views; ++i) {
        const double *Ai = A + 12L * i;
        const float *img = proj + img_px * i;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1) reduction(max : status)
#endif
        for (int z = z_begin; z < z_end; ++z) {
            double wz = origin[2] + z * spacing[2];
            double *vz = vol + (long)(z - z_begin) * plane;
            for (int y = 0; y < L; ++y) {
                double wy = origin[1] + y * spacing[1];
                for (int x = 0; x < L; ++x) {
                    double wx = origin[0] + x * spacing[0];
                    double upd;
                    if (oracle_update(Ai, img, W, H, wx, wy, wz, index_rule, &upd) != ORACLE_OK) {
                        status = ORACLE_EBEHIND;
                        continue;
                    }
                    vz[(long)y * L + x] += upd;
                }
            }
        }
    }
    return status;
}

/*
 * Same sums for a list of voxels given by flat index z*L*L + y*L + x.
 * out[k] (accumulated into) receives the sum over views [0, n_views) in view
 * order for voxel idx[k].  Used to check very large volumes on samples.
 */
int rct_oracle_backproject_voxels(int L, int W, int H, int n_views, const double *A,
                                  const double *origin, const double *spacing, const float *proj,
                                  const int64_t *idx, int64_t n_idx, int n_threads, int index_rule,
                                  double *out)
{
    int rc = check_args(L, W, H, n_views, A, origin, spacing, proj);
    if (rc) return rc;
    if (index_rule != ORACLE_INDEX_FLOOR && index_rule != ORACLE_INDEX_TRUNC) return ORACLE_EINVAL;
    if (n_idx < 0 || (n_idx > 0 && (!idx || !out))) return ORACLE_EINVAL;
    const long img_px = (long)W * H;
    const int64_t total = (int64_t)L * L * L;
    int status = ORACLE_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(n_threads > 0 ? n_threads : 1) reduction(max : status)
#endif
    for (int64_t k = 0; k < n_idx; ++k) {
        int64_t f = idx[k];
        if (f < 0 || f >= total) { status = ORACLE_EINVAL; continue; }
        int x = (int)(f % L);
        int y = (int)((f / L) % L);
        int z = (int)(f / ((int64_t)L * L));
        double wx = origin[0] + x * spacing[0];
        double wy = origin[1] + y * spacing[1];
        double wz = origin[2] + z * spacing[2];
        double acc = out[k];
        for (int i = 0; i < n_views; ++i) {
            double upd;
            if (oracle_update(A + 12L * i, proj + img_px * i, W, H, wx, wy, wz, index_rule, &upd) != ORACLE_OK) {
                status = ORACLE_EBEHIND;
                continue;
            }
            acc += upd;
        }
        out[k] = acc;
    }
    return status;
}

/* IEEE 754 binary16, round to nearest, ties to even; returns the rounded value as float. */
static float round_to_f16(float x)
{
    if (isnan(x)) return x;
    double a = fabs((double)x);
    if (a >= 65520.0) return copysignf(INFINITY, x);   /* at or past the rounding boundary of the max 65504 */
    if (a < ldexp(1.0, -25)) return copysignf(0.0f, x);
    int e;
    frexp(a, &e);                                        /* a = m * 2^e, m in [0.5, 1) */
    int exp_unbiased = e - 1;                            /* a in [2^(e-1), 2^e) */
    if (exp_unbiased < -14) exp_unbiased = -14;          /* subnormal spacing */
    double quantum = ldexp(1.0, exp_unbiased - 10);      /* 10 fraction bits */
    double q = a / quantum;                              /* exact: power-of-two scaling */
    double r = nearbyint(q);                             /* default mode: ties to even */
    return copysignf((float)(r * quantum), x);
}

/* bfloat16 (8 exponent, 7 fraction bits), round to nearest, ties to even. */
static float round_to_bf16(float x)
{
    if (isnan(x) || isinf(x)) return x;
    double a = fabs((double)x);
    if (a == 0.0) return x;
    int e;
    frexp(a, &e);
    int exp_unbiased = e - 1;
    if (exp_unbiased < -126) exp_unbiased = -126;
    double quantum = ldexp(1.0, exp_unbiased - 7);
    double r = nearbyint(a / quantum) * quantum;
    if (r > ldexp(255.0, 120)) return copysignf(INFINITY, x);   /* beyond the largest bfloat16, (2 - 2^-7) * 2^127 */
    return copysignf((float)r, x);
}

int rct_oracle_round_f16(const float *src, float *dst, int64_t n)
{
    if (n < 0 || (n > 0 && (!src || !dst))) return ORACLE_EINVAL;
    for (int64_t k = 0; k < n; ++k) dst[k] = round_to_f16(src[k]);
    return ORACLE_OK;
}

int rct_oracle_round_bf16(const float *src, float *dst, int64_t n)
{
    if (n < 0 || (n > 0 && (!src || !dst))) return ORACLE_EINVAL;
    for (int64_t k = 0; k < n; ++k) dst[k] = round_to_bf16(src[k]);
    return ORACLE_OK;
}

int rct_oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

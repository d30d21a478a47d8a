/*
 * rct_oracle.c -- plain, slow, FP64 definition of the voxel-driven
 * backprojection.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * The quantity (the paper, Section "Algorithm": the RabbitCT backprojection of
 * pre-filtered projections).  View i has a 3x4 projection matrix A_i and an
 * image I_i of W columns by H rows.  A voxel with indices (x, y, z) has the
 * world position (the centre of the voxel)
 *
 *     p = (o_x + x d_x, o_y + y d_y, o_z + z d_z)          origin o, spacing d
 *
 * and view i maps it projectively onto the detector:
 *
 *     (u, v, w) = A_i (p, 1),      detector point (s, t) = (u / w, v / w),
 *
 * where w (> 0 in front of the source) approximates the distance from the
 * source and supplies the distance weight 1 / w^2.  The backprojected value
 * of the voxel is
 *
 *     f(x, y, z) = sum_i  J_i(s_i, t_i) / w_i^2
 *
 * with J_i the bilinear interpolant of image i on its pixel grid, extended by
 * zero beyond the detector.  On the unit grid the interpolant is the
 * tensor-product hat sum
 *
 *     J(s, t) = sum_{a, b} E(a, b) h(s - a) h(t - b),    h(e) = max(0, 1 - |e|),
 *     E(a, b) = I[b][a] for 0 <= a < W and 0 <= b < H, else 0,
 *
 * which only the four grid points around (s, t) reach: with a0 = floor(s),
 * b0 = floor(t), alpha = s - a0, beta = t - b0, the weights are
 * (1 - alpha, alpha) along s and (1 - beta, beta) along t.
 *
 * The volume is stored z-major with x fastest (index z*L*L + y*L + x), the
 * projections as n_views images of H rows by W columns, row-major.
 *
 * Readings where the paper's printed kernel is ambiguous (each one is also
 * listed in the design notes):
 *   - The printed kernel selects the cell with an (int) cast, which truncates
 *     toward zero; that equals floor only for non-negative coordinates.  The
 *     default here is the zero-extended interpolant above (floor), the reading
 *     that the paper's zero-padded projection buffer (Section "SIMD
 *     Vectorization") computes, and the one under which J is continuous.
 *     index_rule = 1 selects the truncating cell instead (RabbitCT
 *     compatibility): a0 = trunc(s) and alpha = s - a0, negative for negative
 *     s, so the weights (1 - alpha, alpha) extrapolate from the two taps at the
 *     image edge.
 *   - The printed bounds test compares the row index with the width and the
 *     column index with the height while rows are addressed with stride W;
 *     here the column index is tested against W and the row index against H.
 *   - The printed kernel reads its matrix column-major; this oracle takes
 *     row-major matrices, A[r*4 + c].
 *   - Pixel (a, b) is the sample at detector coordinate (a, b) exactly.
 *   - The paper's CPU kernels use an approximate reciprocal (Section "SIMD
 *     Vectorization"); the oracle divides in FP64.
 *   - w <= 0 (a voxel at or behind the source) cannot occur in the scan
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
#define ORACLE_INDEX_TRUNC 1   /* the printed kernel's (int) cast: toward zero (RabbitCT compatibility) */

/* World position of the centre of voxel (x, y, z). */
static void voxel_centre(const double *origin, const double *spacing, int x, int y, int z, double p[3])
{
    p[0] = origin[0] + x * spacing[0];
    p[1] = origin[1] + y * spacing[1];
    p[2] = origin[2] + z * spacing[2];
}

/* Homogeneous detector coordinates q = A (p, 1) of a row-major 3x4 matrix. */
static void project(const double *A, const double p[3], double q[3])
{
    for (int r = 0; r < 3; ++r)
        q[r] = A[4 * r] * p[0] + A[4 * r + 1] * p[1] + A[4 * r + 2] * p[2] + A[4 * r + 3];
}

/* The zero-extended image E(a, b): pixel (a, b) on the detector, 0 beyond it. */
static double extended_pixel(const float *img, int W, int H, double a, double b)
{
    if (!(a >= 0.0 && a < (double)W && b >= 0.0 && b < (double)H)) return 0.0;
    return img[(long)b * W + (long)a];
}

/* Grid point below coordinate c and the weight of the point above it. */
static double cell_of(double c, int index_rule, double *frac)
{
    double base = (index_rule == ORACLE_INDEX_TRUNC) ? trunc(c) : floor(c);
    *frac = c - base;
    return base;
}

/* The interpolant J(s, t): the hat-weighted sum over the 2 x 2 grid points around (s, t). */
static double interpolant(const float *img, int W, int H, double s, double t, int index_rule)
{
    double alpha, beta;
    double a0 = cell_of(s, index_rule, &alpha);
    double b0 = cell_of(t, index_rule, &beta);
    const double ws[2] = {1.0 - alpha, alpha};
    const double wt[2] = {1.0 - beta, beta};
    double sum = 0.0;
    for (int db = 0; db < 2; ++db)
        for (int da = 0; da < 2; ++da)
            sum += ws[da] * wt[db] * extended_pixel(img, W, H, a0 + da, b0 + db);
    return sum;
}

/* One view's term J(s, t) / w^2 for the voxel at world position p. */
static int view_term(const double *A, const float *img, int W, int H, const double p[3], int index_rule,
                     double *term)
{
    double q[3];
    project(A, p, q);
    if (!(q[2] > 0.0)) return ORACLE_EBEHIND;
    *term = interpolant(img, W, H, q[0] / q[2], q[1] / q[2], index_rule) / (q[2] * q[2]);
    return ORACLE_OK;
}

static int check_args(int L, int W, int H, int n_views, const double *A, const double *origin,
                      const double *spacing, const float *proj, int index_rule)
{
    if (L <= 0 || W <= 0 || H <= 0 || n_views < 0) return ORACLE_EINVAL;
    if (!A || !origin || !spacing || (!proj && n_views > 0)) return ORACLE_EINVAL;
    if (index_rule != ORACLE_INDEX_FLOOR && index_rule != ORACLE_INDEX_TRUNC) return ORACLE_EINVAL;
    return ORACLE_OK;
}

/*
 * Add the terms of views [0, n_views) to z-planes [z_begin, z_end) of an L^3
 * volume.  `vol` holds (z_end - z_begin) planes of L*L doubles and is
 * accumulated into (the caller zeroes it for a fresh reconstruction).  The
 * views are added in order, each one over all planes before the next, as the
 * RabbitCT framework hands the module one projection at a time.  Planes are
 * independent (the paper's parallelisation, Section "Implementation");
 * n_threads > 1 spreads them over threads without changing any sum.
 */
int rct_oracle_backproject(int L, int W, int H, int n_views, const double *A,
                           const double *origin, const double *spacing, const float *proj,
                           int z_begin, int z_end, int n_threads, int index_rule, double *vol)
{
    int rc = check_args(L, W, H, n_views, A, origin, spacing, proj, index_rule);
    if (rc) return rc;
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
            double *fz = vol + (long)(z - z_begin) * plane;
            for (int y = 0; y < L; ++y) {
                for (int x = 0; x < L; ++x) {
                    double p[3], term;
                    voxel_centre(origin, spacing, x, y, z, p);
                    if (view_term(Ai, img, W, H, p, index_rule, &term) != ORACLE_OK) {
                        status = ORACLE_EBEHIND;
                        continue;
                    }
                    fz[(long)y * L + x] += term;
                }
            }
        }
    }
    return status;
}

/*
 * The same sums for a list of voxels given by flat index z*L*L + y*L + x.
 * out[k] (accumulated into) receives the sum over views [0, n_views), in view
 * order, for voxel idx[k].  Used to check very large volumes on samples.
 */
int rct_oracle_backproject_voxels(int L, int W, int H, int n_views, const double *A,
                                  const double *origin, const double *spacing, const float *proj,
                                  const int64_t *idx, int64_t n_idx, int n_threads, int index_rule,
                                  double *out)
{
    int rc = check_args(L, W, H, n_views, A, origin, spacing, proj, index_rule);
    if (rc) return rc;
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
        double p[3];
        voxel_centre(origin, spacing, (int)(f % L), (int)((f / L) % L), (int)(f / ((int64_t)L * L)), p);
        double sum = out[k];
        for (int i = 0; i < n_views; ++i) {
            double term;
            if (view_term(A + 12L * i, proj + img_px * i, W, H, p, index_rule, &term) != ORACLE_OK) {
                status = ORACLE_EBEHIND;
                continue;
            }
            sum += term;
        }
        out[k] = sum;
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

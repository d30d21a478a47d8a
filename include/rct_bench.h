/*
 * rct_bench.h -- throughput probes: a measurement library (librct_bench.so),
 * separate from librct.so, used by the benchmark to measure the ceilings it
 * reports the backprojection against.  The product path never loads it.
 *
 * The paper compares its kernels with measured machine limits: the streaming
 * update bandwidth of each machine (Table 1) and likwid-bench gather
 * microbenchmarks (Section "Gather performance").  These probes measure the
 * same kinds of limit on the GPU.  Every probe allocates its own small device
 * buffers, runs on the current device, synchronises it, and writes the best
 * of a few timed repetitions to *rate.  Errors: RCT_EINVAL for arguments out
 * of range, RCT_ENOMEM / RCT_ECUDA when a CUDA call fails.
 */
#ifndef RCT_BENCH_H
#define RCT_BENCH_H

#include "rct.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Fetches per second over the whole GPU for fetches of one kind -- mode 0 =
 * tld4 gather, 1 = point fetch, 2 = bilinear filtered fetch, 3 = four
 * predicated global loads of the 2x2 cell (FP32 only), 4 = one 16-byte quad
 * load, 5 = two 8-byte pair loads (4 and 5: FP32 staged layouts over a
 * 1280 x 1024-element buffer that lives in L2, not L1) -- from a 256x256
 * texture (or linear image) of dtype RCT_PROJ_F32 or RCT_PROJ_F16 that stays
 * cache resident; neighbouring lanes sample stride_px apart along x and each
 * fetch advances step_px along y (stride 0..10 px, step 0..8 px).
 */
RCT_API rct_status rct_probe_texture(int mode, int dtype, float stride_px, float step_px, int iters, double *rate);

/*
 * Bytes read + written per second by a float4 read-modify-write sweep over
 * `bytes` (>= 1 MiB) of device memory: the paper's "Node Update" benchmark
 * (Table 1), the HBM roofline of the volume stream.
 */
RCT_API rct_status rct_probe_update_stream(size_t bytes, double *rate);

/*
 * Bytes per second the L1 load data path delivers over the whole GPU: every
 * warp repeatedly reads a 16 KiB block of its own with coalesced 16-byte
 * loads (each load instruction reads 512 contiguous bytes), so after the
 * first pass every load hits L1.  The measured ceiling of the gather's load
 * path.  iters: loads per thread (>= 64).
 */
RCT_API rct_status rct_probe_l1_bandwidth(int iters, double *rate);

/*
 * Sectors per second L2 delivers to the SMs for scattered loads: every lane
 * loads 16 bytes from a pseudo-random 32-byte sector of a 64 MiB buffer (well
 * inside L2, far beyond L1) with L1-bypassing loads, so each warp load asks
 * for 32 distinct sectors.  The ceiling of a gather whose taps miss L1.
 * iters: loads per thread (>= 64).
 */
RCT_API rct_status rct_probe_l2_sectors(int iters, double *rate);

/*
 * Cells per second for the backprojection's plain-load gather (four 4-byte
 * taps of a 2x2 cell per lane) with a given warp footprint: lane l fetches
 * at (x + lane_uv[2l], y + lane_uv[2l + 1]) pixels from an L1-resident
 * 256 x 128 FP32 image, and every fetch moves the footprint by (step_u,
 * step_v), as the next voxel of a z-run does.  The caller passes a real
 * warp's projected voxel offsets, so the rate is the ceiling of that access
 * pattern.  Offsets within +-100 px, the rows they span within 40 px, steps
 * within +-16 px, iters >= 16; RCT_EINVAL otherwise.
 */
RCT_API rct_status rct_probe_gather_pattern(const float *lane_uv, float step_u, float step_v, int iters,
                                            double *rate);

#ifdef __cplusplus
}
#endif

#endif /* RCT_BENCH_H */

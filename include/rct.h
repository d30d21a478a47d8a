/*
 * rct.h -- C ABI of the GB300 voxel-driven cone-beam backprojector.
 *
 * The operation is the RabbitCT backprojection (the paper, Section
 * "Algorithm", Listing 1): for each view i with projection matrix
 * A_i in R^{3x4} and pre-filtered projection image I_i (W columns by H rows),
 * every voxel (x, y, z) of an L^3 volume is mapped to world coordinates
 * p = origin + (x, y, z) * spacing, projected to (u, v, w) = A_i (p, 1),
 * de-homogenised to (u/w, v/w), and the bilinear interpolation of the four
 * neighbouring pixels (zero outside the detector) weighted by 1/w^2 is added
 * into the voxel.  Floor, not truncation, selects the pixel cell, so the
 * image behaves as zero-extended (the paper's zero-padded projection buffer,
 * Section "SIMD Vectorization").
 *
 * Layouts
 *   volume      L^3 float32, z-major, x fastest: index z*L*L + y*L + x
 *   projection  n images, each H rows of W pixels, row-major (pixel (i, j) at
 *               j*W + i), element type as set by rct_set_precision
 *   matrices    n_views * 12 float64, row-major 3x4 per view (A[r*4 + c]);
 *               NOTE: the paper's listing reads its matrix column-major
 *
 * Conventions
 *   - Every call returns an rct_status; on failure rct_last_error() gives a
 *     message for the calling thread.  Argument errors are detected
 *     synchronously.  Asynchronous CUDA faults surface as RCT_ECUDA from a
 *     later call on the same context.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream only enqueue work on it unless
 *     stated otherwise; results are valid once the stream reaches them.
 *   - A context is bound to the CUDA device that is current when it is
 *     created; later calls must be made with that device current.  A context
 *     is not thread-safe, and the work of successive calls on one context
 *     must be ordered (one stream, or streams the caller synchronises):
 *     they share the context's staging buffers.  Distinct contexts may be
 *     used from distinct threads and streams concurrently.
 *   - The library never falls back to a CPU computation.
 *
 * Two more headers go with it: rct_debug.h (the bounds-checking build's
 * counters, exported by the same library) and rct_bench.h (throughput
 * probes, a separate measurement library librct_bench.so that the product
 * does not load).
 */
#ifndef RCT_H
#define RCT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RCT_API __attribute__((visibility("default")))
#else
#define RCT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rct_ctx rct_ctx;

typedef enum rct_status {
    RCT_OK = 0,
    RCT_EINVAL = 1,    /* bad argument (null pointer, size or range) */
    RCT_ENOMEM = 2,    /* device or host allocation failed */
    RCT_ECUDA = 3,     /* a CUDA runtime call or kernel failed */
    RCT_ESTATE = 4,    /* call not valid in the context's state (e.g. no geometry yet) */
    RCT_ETIMEOUT = 5,  /* a host-side wait gave up (serving deadlines) */
    RCT_ENOTSUP = 6    /* combination of options not supported */
} rct_status;

/* Element type of stored projections (the reduced-precision storage variants). */
typedef enum rct_proj_dtype {
    RCT_PROJ_F32 = 0,
    RCT_PROJ_F16 = 1,   /* IEEE binary16 */
    RCT_PROJ_BF16 = 2   /* bfloat16 */
} rct_proj_dtype;

/* How the four taps are interpolated. */
typedef enum rct_interp {
    RCT_INTERP_SOFT = 0,  /* software bilinear in FP32 (the paper's Part 3); parity-gated */
    RCT_INTERP_TEX = 1    /* texture-unit bilinear (low-precision fixed-point weights); not gated */
} rct_interp;

/*
 * Where the FP32 detector coordinate of a voxel is formed (software interpolation of FP32
 * projections).  The paper evaluates (u, v, w) = A (x, y, z, 1) per voxel (Section "Algorithm");
 * in FP32 the rounding of that sum grows with the distance from the origin of the coordinates.
 */
typedef enum rct_frame {
    RCT_FRAME_GLOBAL = 0, /* one frame per view: the folded matrix over centred voxel coordinates and
                             one integer detector shift (the pixel of the volume centre).  Fastest. */
    RCT_FRAME_BLOCK = 1   /* one frame per thread block and view: the block corner's (u', v', w) in
                             double-float and a block-local integer shift, so every FP32 coordinate is
                             a short local offset.  About 16x smaller error vs the FP64 oracle (at
                             L = 512), at a cost in speed (more registers per thread). */
} rct_frame;

/*
 * How the cell of a detector coordinate ix is chosen.  Listing 1 (Section "Algorithm") casts with
 * (int), which truncates toward zero: for ix in (-2, 0) that picks the cell one pixel to the right
 * of floor's and gives the tap at ix's right a negative weight (the listing extrapolates from the
 * image edge).  Floor treats the image as zero-extended and keeps the interpolant continuous; it is
 * the reading this library uses by default.  The two agree wherever ix >= 0 and iy >= 0.
 */
typedef enum rct_index_rule {
    RCT_INDEX_FLOOR = 0,  /* i0 = floor(ix) (default) */
    RCT_INDEX_TRUNC = 1   /* i0 = (int) ix as in Listing 1: RabbitCT compatibility */
} rct_index_rule;

/* How a software-interpolated kernel fetches its four taps (Part 2). */
typedef enum rct_gather {
    RCT_GATHER_AUTO = 0,  /* let the library (or the tuning cache) choose */
    RCT_GATHER_LDG = 1,   /* four predicated read-only loads from the caller's linear images */
    RCT_GATHER_TLD4 = 2,  /* one texture gather (tld4) of the 2x2 cell from a staged copy */
    RCT_GATHER_MIX = 3,   /* per z-run: the first tex_zrun positions by tld4, the rest by quad loads
                             (below), so the texture and load/store pipes work side by side */
    RCT_GATHER_QUAD = 4,  /* one 128-bit load (64-bit for 16-bit data) of a staged, zero-padded "quad"
                             copy of the image whose every element holds a whole 2x2 cell */
    RCT_GATHER_PAIR = 5,  /* two 64-bit loads (32-bit for 16-bit data) of a staged, zero-padded copy
                             whose every element holds two vertically adjacent pixels */
    RCT_GATHER_DQUAD = 6  /* FP32 only: one 128-bit load of a staged, zero-padded copy whose every
                             element holds a cell's left column and its two horizontal differences,
                             so both rows are interpolated along x by one packed FMA; bit for bit the
                             sums of RCT_GATHER_QUAD and RCT_GATHER_PAIR.  RCT_ENOTSUP at the first
                             backprojection call with 16-bit projections */
} rct_gather;

/* Kernel tuning.  Zero in any field means "keep the current value". */
typedef struct rct_tuning {
    int views_per_pass;  /* K: views accumulated in registers per volume pass, 1..32 */
    int zrun;            /* voxels per thread along z: 1, 2, 4, 8 or 16 (16 needs xvec <= 2) */
    int xvec;            /* voxels per thread along x: 1, 2 or 4 (4 needs L % 4 == 0) */
    int block_x;         /* threads per block along x */
    int block_y;         /* threads per block along y; block_x * block_y <= 512 */
    int gather;          /* rct_gather */
    int tex_zrun;        /* RCT_GATHER_MIX: z positions per run fetched by tld4, 1..zrun-1 */
    int view_split;      /* 1, 2, 4 or 8: deal each pass's views out to this many groups of blocks, each adding
                            into its own partial volume (the context holds view_split - 1 more volumes);
                            the partials are added into the volume after each call's last pass.  More blocks
                            per pass for small volumes; the per-voxel sum is regrouped (within the FP32
                            parity bar of the plain order, deterministic).  Software gathers, global frame
                            and floor rule only (RCT_ENOTSUP at the first backprojection call otherwise). */
} rct_tuning;

#define RCT_MAX_VIEWS_PER_PASS 32

/*
 * Create a context for an L^3 volume and a scan of n_views projections of
 * det_w x det_h pixels, on the current CUDA device.  Allocates the device
 * volume (L^3 floats).  The volume starts at zero.  Returns NULL on failure
 * (see rct_last_error).  Paper: the RabbitCT module receives L, the image
 * width and the matrices from the framework (Section "Algorithm").
 */
RCT_API rct_ctx *rct_create(int L, int det_w, int det_h, int n_views);

/*
 * A context that holds only the z planes [z_first, z_first + z_count) of the
 * L^3 volume (a z-slab): the paper parallelises the backprojection over
 * independent voxel planes (Section "Implementation"), and a slab context is
 * that split as a unit of work for one GPU.  Every call behaves as on a
 * whole-volume context restricted to those planes: the device volume, and the
 * buffers rct_read_volume / rct_write_volume / rct_backproject_host_read
 * exchange, hold z_count * L * L floats (plane z_first first, then z-major
 * with x fastest); projections and matrices are the whole scan's.  Slab
 * boundaries lie on multiples of 16 planes (z_first, and z_first + z_count
 * unless it equals L): every z-run length divides 16, so the threads' runs
 * are the whole-volume context's runs and each plane is bit for bit the same
 * plane of a whole-volume context with the same tuning.  NULL on failure:
 * an empty or out-of-range slab, or an unaligned boundary, gives RCT_EINVAL;
 * the other failures are rct_create's.
 */
RCT_API rct_ctx *rct_create_slab(int L, int det_w, int det_h, int n_views, int z_first, int z_count);
/* Writes the planes a context holds (0 and L for rct_create). */
RCT_API rct_status rct_get_slab(const rct_ctx *ctx, int *z_first, int *z_count);

/*
 * Release every device resource of the context.  It first waits for the work
 * enqueued for this context (not for other contexts' work); freeing device
 * memory may still synchronise the device.  NULL is ignored.
 */
RCT_API void rct_destroy(rct_ctx *ctx);

/*
 * Set the scan geometry: n_views row-major 3x4 FP64 matrices (pixel units:
 * (u/w, v/w) is the column/row of the pixel hit), the world position (mm) of
 * the centre of voxel (0,0,0) and the voxel spacing (mm) per axis.  The
 * library folds origin and spacing into each matrix in FP64 on the host
 * (the paper's O and MM, Section "Algorithm") and keeps its own copies; the
 * caller's arrays may be freed on return.  RCT_EINVAL for null pointers,
 * non-finite values or non-positive spacing, and for a view in which a
 * corner of the volume has w <= 0 (at or behind the source: Listing 1's
 * 1/w^2 weight assumes every voxel in front of it) or projects 2^21 pixels
 * or more from where the volume centre projects.  If work of this context
 * is still queued, the call waits for it (the new geometry replaces a table
 * those passes read); work of other contexts is not waited for.
 */
RCT_API rct_status rct_set_geometry(rct_ctx *ctx, const double *matrices, const double origin[3],
                            const double spacing[3]);

/*
 * Choose the element type of the projections passed to rct_backproject and
 * the interpolation.  Accumulation and the 1/w^2 weight stay FP32.
 * Default: RCT_PROJ_F32, RCT_INTERP_SOFT.
 * Paper: the RabbitCT projections are FP32 (Section "RabbitCT Benchmark"),
 * and Part 2 of Listing 1 (Section "Algorithm") reads four FP32 pixels.
 * 16-bit storage halves those gather bytes; the texture-unit bilinear
 * option follows the paper's account of why GPUs are fast at this kernel
 * (Section "Comparison to GPU Implementations").  Neither is in the
 * paper's own kernels: they are reduced-precision variants whose error
 * against the FP64 definition is stated, not assumed.
 * Errors: RCT_EINVAL for an unknown dtype or interp; RCT_ENOTSUP when the
 * context's frame or index rule needs FP32 software interpolation.
 * Takes effect at the next call; nothing is enqueued.
 */
RCT_API rct_status rct_set_precision(rct_ctx *ctx, int proj_dtype, int interp);
/* The element type and interpolation set for the context (either pointer may be NULL). */
RCT_API rct_status rct_get_precision(const rct_ctx *ctx, int *proj_dtype, int *interp);

/*
 * Choose the coordinate frame (rct_frame; default RCT_FRAME_GLOBAL).  RCT_FRAME_BLOCK needs FP32
 * projections and software interpolation (the rounding of 16-bit projections and the texture
 * unit's fixed-point weights are far larger than what it removes): RCT_ENOTSUP otherwise, here
 * and from a later rct_set_precision that would break that.  RCT_EINVAL for an unknown value.
 */
RCT_API rct_status rct_set_frame(rct_ctx *ctx, int frame);
RCT_API rct_status rct_get_frame(const rct_ctx *ctx, int *frame);

/*
 * RabbitCT compatibility (Listing 1's conventions, for data prepared for the RabbitCT framework).
 *
 * rct_set_index_rule chooses the cell rule (rct_index_rule; default RCT_INDEX_FLOOR).
 * RCT_INDEX_TRUNC needs FP32 projections, software interpolation and the global frame
 * (RCT_ENOTSUP otherwise, here and from a later rct_set_precision / rct_set_frame that would break
 * that); it reads the caller's images with plain loads, whatever gather route the tuning names.
 * The bounds test stays "column in [0, W), row in [0, H)" (the listing's test swaps width and
 * height in print; its row stride is the width).
 *
 * rct_set_geometry_rabbitct takes the geometry as the RabbitCT module receives it: n_views 3x4
 * FP32 matrices stored column-major (element (r, c) at A[3c + r], as Listing 1 reads A[0], A[3],
 * A[6], A[9] for u), and the scalar origin O and voxel size MM (mm) shared by the three axes
 * (world position of voxel (x, y, z) = (O + x MM, O + y MM, O + z MM)).  It widens them to FP64
 * and calls rct_set_geometry, with the same errors.
 */

RCT_API rct_status rct_set_index_rule(rct_ctx *ctx, int rule);
RCT_API rct_status rct_get_index_rule(const rct_ctx *ctx, int *rule);
RCT_API rct_status rct_set_geometry_rabbitct(rct_ctx *ctx, const float *matrices, float O, float MM);

/*
 * Pre-processing of raw projections on the device (the step before the path: RabbitCT supplies
 * projections already weighted and filtered, Section "RabbitCT Benchmark"; a scanner supplies line
 * integrals).  For view v and pixel (i, j), with D = sdd (source-detector distance, mm),
 * tau = pitch (detector pixel size, mm) and (u0, v0) the view's principal point (pixels):
 *
 *   cosine weight  p'(i, j) = p(i, j) * D / sqrt(D^2 + ((i - u0) tau)^2 + ((j - v0) tau)^2)
 *   ramp filter    q(i, j)  = tau * sum_{k=0}^{W-1} h[i - k] p'(k, j)
 *                  h[n]     = -2 / (pi^2 tau^2 (4 n^2 - 1))     (Shepp-Logan kernel, FDK method)
 *
 * i.e. each row is convolved linearly (zero outside the row) with the kernel.
 *
 * rct_set_filter stores the filter for the context: sdd and pitch (finite, > 0) and principal,
 * n_views pairs (u0, v0) in view order (copied; the caller's array may be freed on return).
 * Rows longer than 8192 pixels give RCT_ENOTSUP.  A set-up call: it waits for the work already
 * enqueued for this context (filter launches read the tables it replaces), not for other contexts.
 *
 * rct_filter_projections filters views [first_view, first_view + n): d_raw holds n FP32 images
 * [n][H][W] on the device; d_out receives n images in out_dtype (rct_proj_dtype, rounded to
 * nearest even for 16-bit types), the layout rct_backproject reads.  An FP32 output may be
 * written in place (d_out == d_raw); any other overlap of input and output is RCT_EINVAL.
 * Enqueued on `stream`; the caller keeps both buffers valid until the stream reaches the call.
 * RCT_ESTATE before rct_set_filter.  The arithmetic is FP32 (transforms of length >= 2W - 1 in
 * shared memory, see the design notes); the spectrum of h is computed on the host in FP64.
 */
RCT_API rct_status rct_set_filter(rct_ctx *ctx, double sdd, double pitch, const double *principal);
RCT_API rct_status rct_filter_projections(rct_ctx *ctx, const float *d_raw, void *d_out, int out_dtype,
                                          int first_view, int n, void *stream);

/* Override the kernel tuning (see rct_tuning).  Validated synchronously. */
RCT_API rct_status rct_set_tuning(rct_ctx *ctx, const rct_tuning *t);
/* Read the tuning the next launch will use (after AUTO resolution). */
RCT_API rct_status rct_get_tuning(const rct_ctx *ctx, rct_tuning *out);

/*
 * Zero the volume: the start of a reconstruction, before the first view is
 * added (the RabbitCT volume starts at zero and every view's Listing 1 pass,
 * Section "Algorithm", adds into it; layout z*L*L + y*L + x as Listing 1
 * indexes it).  Costs nothing on the device: the next pass overwrites
 * instead of adding (a read or write of the volume first clears it).
 * Errors: RCT_EINVAL for a null context, RCT_ESTATE when another device is
 * current.
 */
RCT_API rct_status rct_reset_volume(rct_ctx *ctx, void *stream);

/*
 * Backproject views [first_view, first_view + n) into the volume, in view
 * order: for each of those views and every voxel, Listing 1's three parts
 * (Section "Algorithm": project with the view's matrix and de-homogenise;
 * gather the 2x2 pixel cell, zero off the detector; interpolate bilinearly
 * and add val / w^2 into VOL[z*L*L + y*L + x]).  Views are accumulated K
 * at a time in registers (the tuning's views_per_pass), which changes the
 * order of the FP32 additions but not the sum's terms.  d_proj points to n device images (the first one belongs to view
 * first_view) in the element type set by rct_set_precision.  Texture routes
 * stage each batch of K views into the context's gather arrays on an
 * internal copy stream (forked from and joined back into `stream` with
 * events), so staging overlaps the previous batch's pass.  The caller
 * owns d_proj and must keep it valid and unchanged until the stream reaches
 * the end of this call's work.  Asynchronous on `stream`; allocates nothing
 * once the context's staging buffers exist (they are created by the first
 * call after rct_set_precision / rct_set_tuning changes them, so make one
 * call before capturing this into a CUDA graph).
 * Errors: RCT_ESTATE if no geometry was set; RCT_EINVAL for a null d_proj,
 * n < 0 or a view range outside [0, n_views).
 */
RCT_API rct_status rct_backproject(rct_ctx *ctx, const void *d_proj, int first_view, int n, void *stream);

/*
 * Same, with the n images in host memory (pinned memory makes the copies
 * asynchronous and lets them overlap the kernels).  Views are copied to the
 * device in batches through context-owned staging buffers on a second
 * stream, overlapped with the passes of the previous batch.  Returns once
 * all work is enqueued on `stream`; the host buffer must stay valid until the
 * stream reaches the end of this call's work.
 */
RCT_API rct_status rct_backproject_host(rct_ctx *ctx, const void *h_proj, int first_view, int n, void *stream);

/*
 * rct_backproject_host followed by rct_read_volume(ctx, dst, stream), with the read-back overlapped:
 * the last pass of the call runs as z-slabs and each slab's planes are copied to dst (host or
 * device, L^3 floats, z-major, x fastest) as soon as that slab is done, on the context's copy
 * stream; `stream` waits for the last copy, so dst is complete once `stream` reaches the call.
 * Same arguments and errors as the two calls (RCT_EINVAL for a null dst); the volume stays in the
 * context as well.  The result is bit for bit that of the two separate calls.
 */
RCT_API rct_status rct_backproject_host_read(rct_ctx *ctx, const void *h_proj, int first_view, int n, float *dst,
                                             void *stream);

/*
 * Copy the volume to dst, host or device memory: L^3 floats (z_count*L*L for a
 * slab context, see rct_create_slab), z-major with x fastest, the index
 * z*L*L + y*L + x of Listing 1 (Section "Algorithm").  Enqueued on stream;
 * dst must stay valid until the stream reaches the copy (pageable host
 * memory makes the call wait for it).  Errors: RCT_EINVAL for a null dst.
 */
RCT_API rct_status rct_read_volume(rct_ctx *ctx, float *dst, void *stream);

/* Overwrite the volume from src (host or device, L^3 floats): restores a checkpoint. */
RCT_API rct_status rct_write_volume(rct_ctx *ctx, const float *src, void *stream);

/* Device address of the volume (valid until rct_destroy); NULL on error. */
RCT_API float *rct_volume_device_ptr(rct_ctx *ctx);

/* Geometry of the context: writes L, det_w, det_h, n_views. */
RCT_API rct_status rct_get_shape(const rct_ctx *ctx, int *L, int *det_w, int *det_h, int *n_views);

/* Number of kernel launches the context has enqueued since creation. */
RCT_API int64_t rct_launch_count(const rct_ctx *ctx);

/*
 * Allocate, now, the staging resources that rct_backproject (and, when
 * host_input != 0, rct_backproject_host) will use with the current precision
 * and tuning, so that later calls allocate nothing and can be captured into
 * a CUDA graph.
 */
RCT_API rct_status rct_prepare(rct_ctx *ctx, int host_input);

/* Device bytes a context of this shape holds once prepared (volume + staging); 0 for bad input. */
RCT_API size_t rct_footprint_bytes(int L, int det_w, int det_h, int proj_dtype, int views_per_pass, int host_input);

/*
 * CUDA-graph capture of a sequence of calls on one stream (thread-local
 * capture mode).  Between rct_graph_begin(stream) and rct_graph_end(stream,
 * &g) every rct_* call on `stream` is recorded instead of run; the contexts
 * involved must have been prepared (rct_prepare) so that nothing allocates.
 * Kernel parameters (matrices, view range, pointers, the overwrite flag of a
 * first pass after a reset) are frozen into the graph; the caller keeps the
 * buffers it names alive while the graph exists.  rct_graph_launch replays
 * it on any stream; rct_graph_destroy releases it.  The default stream
 * cannot be captured (RCT_EINVAL).  The graph also points at state the
 * contexts own; rct_graph_launch returns RCT_ESTATE, and launches nothing,
 * once one of them has been destroyed or has replaced that state since the
 * capture: staging reallocated (a larger views_per_pass, another storage type
 * or gather route), a new geometry (rct_set_geometry*) or new filter tables
 * (rct_set_filter).  Capture again after such a change.
 */
typedef struct rct_graph rct_graph;
RCT_API rct_status rct_graph_begin(void *stream);
RCT_API rct_status rct_graph_end(void *stream, rct_graph **out);
RCT_API rct_status rct_graph_launch(rct_graph *graph, void *stream);
RCT_API void rct_graph_destroy(rct_graph *graph);

/*
 * Measurement support.  While enabled, every backprojection kernel the
 * context launches is bracketed by two CUDA events recorded on the launch
 * stream.  rct_profile_read waits for the last one, returns the summed
 * kernel time (ms) and the number of timed launches since the last read (or
 * since enabling), and starts a new count.  Enabling creates events lazily;
 * do not enable it inside a CUDA graph capture.
 */
RCT_API rct_status rct_profile_kernels(rct_ctx *ctx, int enable);
RCT_API rct_status rct_profile_read(rct_ctx *ctx, double *kernel_ms, int64_t *kernel_launches);

/*
 * Convert n FP32 values to the storage type dtype (round to nearest, ties
 * to even) on the device: dst receives n 16-bit values for F16/BF16 (or a
 * copy for F32).  Projection staging for the precision variants.
 */
RCT_API rct_status rct_convert_projections(const float *d_src, void *d_dst, size_t n, int dtype, void *stream);

/*
 * Host-only helper (no GPU needed): the FP64 fold that rct_set_geometry
 * applies.  For each view it writes 12 doubles, rows (u', v', w) such that
 * for centred voxel coordinates c = (x, y, z) - (L-1)/2
 *     u' = u - cu*w,  v' = v - cv*w,  w = w   with (u, v, w) = A (origin + (x,y,z)*spacing, 1),
 * and the integer detector shift (cu, cv): the pixel nearest to where the
 * volume centre projects (0 when that point is not in front of the source).
 * fold_out: n_views * 12 doubles; shift_out: n_views * 2 ints.  RCT_EINVAL
 * as rct_set_geometry (including the checks of the volume's corners).
 */
RCT_API rct_status rct_fold_geometry(int L, int n_views, const double *matrices, const double origin[3],
                             const double spacing[3], double *fold_out, int *shift_out);


/*
 * Allocation-free backprojection (the paper has no counterpart; it exists for
 * callers that cannot allocate device memory: code running inside another
 * framework that owns the memory pool, latency-critical loops where
 * cudaMalloc/cudaFree would synchronise the device, pipelines with a memory
 * budget fixed at start-up).  No context is needed and nothing is allocated:
 * the n FP32 device images d_proj (H x W row-major, views in order) are
 * narrowed to FP16 into a scratch array that is part of the loaded library
 * (a fixed 32 MiB of device memory per GPU, held until the process exits)
 * and backprojected with the FP16 predicated-load kernel into the caller's
 * L^3 FP32 device volume d_volume (overwritten when accumulate == 0, added to
 * otherwise).  matrices: n row-major 3x4 FP64 on the host; origin/spacing as
 * in rct_set_geometry (with its checks of the volume's corners).  Views go
 * through the scratch in batches of up to 32; one view must fit (det_w *
 * det_h <= 16 Mi pixels), and det_w, det_h must stay within the limits
 * rct_create takes (the device's texture-gather extents): RCT_EINVAL
 * otherwise.  The first call on a device looks up the scratch address with
 * cudaGetSymbolAddress (make it before any stream capture; a lookup that
 * fails returns RCT_ECUDA and is tried again by the next call); later calls
 * only enqueue work on `stream`.  All calls on a device share the one scratch:
 * calls whose work may overlap on the GPU (different streams without
 * ordering) race on it and give wrong volumes; order them on one stream.
 * Nothing in the scratch has to start at zero: each batch rewrites what it
 * reads.  Same kernel as the context path with RCT_PROJ_F16 and
 * RCT_GATHER_LDG, zrun 4, xvec 1, block 32x8.
 */
RCT_API rct_status rct_backproject_f16_noalloc(int L, int det_w, int det_h, const double *matrices, int n,
                                               const double origin[3], const double spacing[3],
                                               const float *d_proj, float *d_volume, int accumulate, void *stream);

/* Message describing the last failure on the calling thread ("" if none). */
RCT_API const char *rct_last_error(void);

/* ABI version: major * 10000 + minor * 100 + patch. */
RCT_API int rct_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RCT_H */

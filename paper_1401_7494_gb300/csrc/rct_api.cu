// C ABI of the backprojector: context, FP64 geometry fold, projection staging,
// batching of K views per volume pass, and kernel dispatch.  See include/rct.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/rct.h"
#include "../../include/rct_debug.h"
#include "rct_internal.h"

using namespace rct;

namespace {

thread_local std::string g_last_error;

rct_status fail(rct_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

rct_status cuda_fail(cudaError_t e, const char *what) {
    return fail(RCT_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define RCT_CUDA(call, what)                              \
    do {                                                  \
        cudaError_t rct_e_ = (call);                      \
        if (rct_e_ != cudaSuccess) return cuda_fail(rct_e_, what); \
    } while (0)

size_t dtype_size(int dt) { return dt == DT_F32 ? 4 : 2; }

constexpr double kPi = 3.14159265358979323846;
constexpr int kReadSlabs = 8;   // z-slabs of the last pass when the read-back overlaps it
constexpr int kSlabAlign = 16;  // slab contexts start and end on multiples of this many planes

// One staging slot: a 2D CUDA array that holds one view for texture sampling.
struct Slot {
    cudaArray_t arr = nullptr;
    cudaTextureObject_t tex = 0;
};

}  // namespace

void rct::set_view_geometry(ViewParams *vp, const double fold[12], int cu, int cv) {
    for (int k = 0; k < 4; ++k) {
        vp->muv[2 * k] = static_cast<float>(fold[k]);          // u' row
        vp->muv[2 * k + 1] = static_cast<float>(fold[4 + k]);  // v' row
        vp->mw[k] = static_cast<float>(fold[8 + k]);
    }
    vp->cu = cu;
    vp->cv = cv;
}

void rct::set_view_geo(ViewGeo *vg, const double fold[12], int cu, int cv) {
    for (int k = 0; k < 4; ++k) {
        const double u = fold[k], v = fold[4 + k], w = fold[8 + k];
        const float uh = static_cast<float>(u), vh = static_cast<float>(v), wh = static_cast<float>(w);
        vg->hu[2 * k] = uh;
        vg->hu[2 * k + 1] = vh;
        vg->hw[k] = wh;
        vg->lu[2 * k] = static_cast<float>(u - static_cast<double>(uh));
        vg->lu[2 * k + 1] = static_cast<float>(v - static_cast<double>(vh));
        vg->lw[k] = static_cast<float>(w - static_cast<double>(wh));
    }
    vg->cu = cu;
    vg->cv = cv;
    vg->pad_[0] = vg->pad_[1] = 0;
}

rct_status rct::rct_internal_fail(rct_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

struct rct_ctx {
    int L = 0, W = 0, H = 0, n_views = 0;
    int z_first = 0, z_count = 0;   // planes of the L^3 volume this context holds (all L unless a slab)
    int device = 0;
    uint64_t id = 0;                // registry key (graphs check their contexts through it)
    uint64_t gen = 0;               // bumped whenever device state a captured graph points at is replaced
    float *vol = nullptr;
    bool vol_zero_pending = true;   // the volume is logically zero; the next pass overwrites

    bool geometry_set = false;
    ViewGeo *geo_dev = nullptr;     // n_views block-frame geometries on the device

    bool filter_set = false;        // cosine weight + ramp filter of raw projections (rct_set_filter)
    FilterParams filt{};
    float2 *filt_twiddle = nullptr;
    float *filt_spectrum = nullptr;
    float2 *filt_principal = nullptr;
    std::vector<double> fold;       // n_views x 12, FP64: rows u', v', w over centred voxel coords
    std::vector<int> shift;         // n_views x 2: integer detector shift (cu, cv)

    int dtype = DT_F32;
    int interp = RCT_INTERP_SOFT;
    int frame = RCT_FRAME_GLOBAL;
    int index_rule = RCT_INDEX_FLOOR;
    rct_tuning tune{};              // gather may be RCT_GATHER_AUTO here
    bool tune_explicit_gather = false;

    // texture staging: slots for two batches of K views (ring) and what they were made for
    std::vector<Slot> slots;
    int slot_kind = -1;             // kernel gather kind the slots serve
    int slot_dtype = -1;

    // quad staging (quad-load route): 2K zero-padded quad images
    void *quad_buf = nullptr;
    size_t quad_alloc = 0;

    // view split: view_split - 1 partial volumes of the context's planes
    float *part = nullptr;
    size_t part_alloc = 0;              // floats

    // host-input path: linear device staging (LDG) and the copy stream
    void *lin_stage = nullptr;
    size_t lin_stage_bytes = 0;
    float *widen_buf = nullptr;     // BF16 -> FP32 widening for texture-filtered BF16
    size_t widen_elems = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_filled[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> ev_slab;   // read-back overlap: one per z-slab of the last pass, plus one for the end
    unsigned long long *viol_dev = nullptr;   // bounds-checking build: violation counter
    long long debug_qelems = 0;               // bounds-checking build: lowered staged-image limit (0: none)
    cudaEvent_t ev_free[2] = {nullptr, nullptr};

    int64_t launches = 0;

    // The end of the last work enqueued for this context (recorded after every call that enqueues work
    // outside a stream capture, and after every replay of a graph that uses the context): set-up calls
    // that replace device state wait for it instead of for the whole device.
    cudaEvent_t ev_done = nullptr;
    bool done_recorded = false;

    // optional per-launch timing (CUDA events around every backprojection kernel)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_events;  // pairs: start, stop
    size_t prof_used = 0;
};

namespace {

// Registry of live contexts and the state generation each one is at.  A CUDA graph freezes device
// pointers (staging arrays and buffers, filter tables) and reads tables in place (block-frame geometry);
// a graph remembers the (context, generation) pairs it was captured with and refuses to launch when one
// of its contexts has since been destroyed or has replaced such state.
std::mutex g_reg_mu;
struct LiveEntry {
    uint64_t gen;
    rct_ctx *ctx;
};
std::unordered_map<uint64_t, LiveEntry> g_live;                // context id -> generation, context
std::atomic<uint64_t> g_next_id{1};
thread_local int g_capturing = 0;                              // rct_graph_begin calls open on this thread
thread_local std::vector<std::pair<uint64_t, uint64_t>> g_captured;

void bump(rct_ctx *c) {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    ++c->gen;
    const auto it = g_live.find(c->id);      // absent once rct_destroy has begun: stays absent
    if (it != g_live.end()) it->second.gen = c->gen;
}

// Called by every call that enqueues work for a context: records it when `s` is being captured.
void note_capture(const rct_ctx *c, void *stream) {
    if (g_capturing <= 0 || !stream) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    if (cs == cudaStreamCaptureStatusActive) g_captured.emplace_back(c->id, c->gen);
}

int kernel_kind(const rct_ctx *c) { return c->interp == RCT_INTERP_TEX ? G_TEXLIN : G_SOFT; }

// The gather route the kernels use: the tuned one, except that the truncating index rule reads the
// caller's images with plain loads.
int gather_of(const rct_ctx *c) { return c->index_rule == RCT_INDEX_TRUNC ? RCT_GATHER_LDG : c->tune.gather; }

// Number of z positions of each run that fetch through the texture gather (the rest load).
// LDG, QUAD: none; TLD4 (and AUTO): all; MIX: the tuned split.
int tex_zrun_of(const rct_ctx *c) {
    const int R = c->tune.zrun;
    switch (gather_of(c)) {
        case RCT_GATHER_LDG:
        case RCT_GATHER_QUAD:
        case RCT_GATHER_PAIR:
        case RCT_GATHER_DQUAD: return 0;
        case RCT_GATHER_MIX: return R <= 1 ? R : std::min(std::max(c->tune.tex_zrun, 1), R - 1);
        default: return R;
    }
}

bool uses_tex(const rct_ctx *c) { return kernel_kind(c) == G_TEXLIN || tex_zrun_of(c) > 0; }

// Staged layout the load part of the software route reads: 0 = none (texture only, or the
// caller's linear image), 1 = quads (QUAD, MIX), 2 = vertical pairs (PAIR), 3 = difference quads (DQUAD).
int load_layout(const rct_ctx *c) {
    if (kernel_kind(c) != G_SOFT || gather_of(c) == RCT_GATHER_LDG || tex_zrun_of(c) >= c->tune.zrun) return 0;
    if (gather_of(c) == RCT_GATHER_PAIR) return 2;
    return gather_of(c) == RCT_GATHER_DQUAD ? 3 : 1;
}

bool uses_quad(const rct_ctx *c) { return load_layout(c) != 0; }

size_t layout_bytes(const rct_ctx *c) {
    return load_layout(c) == 2 ? pair_bytes(c->W, c->H, c->dtype) : quad_bytes(c->W, c->H, c->dtype);
}

// Stages n consecutive views (src: n linear images back to back) into n consecutive staging slots from
// dst, in one launch.
cudaError_t launch_stage_layout(const rct_ctx *c, const void *src, void *dst, int n, cudaStream_t s) {
    switch (load_layout(c)) {
        case 2: return launch_stage_pairs(src, dst, c->W, c->H, c->dtype, n, s);
        case 3: return launch_stage_dquads(static_cast<const float *>(src), dst, c->W, c->H, n, s);
        default: return launch_stage_quads(src, dst, c->W, c->H, c->dtype, n, s);
    }
}

// The difference-quad layout holds FP32 values only; the view split runs the software gathers in the
// global frame with the floor rule.
rct_status check_route(const rct_ctx *c) {
    if (gather_of(c) == RCT_GATHER_DQUAD && (c->dtype != DT_F32 || kernel_kind(c) != G_SOFT))
        return fail(RCT_ENOTSUP, "the difference-quad gather needs FP32 projections and software interpolation");
    if (c->tune.view_split > 1 &&
        (kernel_kind(c) != G_SOFT || c->frame != RCT_FRAME_GLOBAL || c->index_rule != RCT_INDEX_FLOOR))
        return fail(RCT_ENOTSUP, "the view split needs software interpolation, the global frame and the floor rule");
    return RCT_OK;
}

// The kernel reads the caller's linear image (LDG route), or BF16 must be widened before a
// filtered texture.
bool uses_linear(const rct_ctx *c) {
    if (kernel_kind(c) == G_TEXLIN) return c->dtype == DT_BF16;
    return gather_of(c) == RCT_GATHER_LDG;
}

// Host input must land in linear device memory first when a kernel or a staging step reads it there.
bool host_needs_linear(const rct_ctx *c) { return uses_linear(c) || uses_quad(c); }



rct_tuning default_tuning(int L) {
    rct_tuning t{};
    t.views_per_pass = 16;
    t.zrun = 4;
    t.xvec = 1;
    t.block_x = 32;
    t.block_y = 8;
    t.gather = RCT_GATHER_AUTO;
    t.view_split = 1;
    (void)L;
    return t;
}

rct_status check_ctx(const rct_ctx *c) {
    if (!c) return fail(RCT_EINVAL, "null context");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != c->device)
        return fail(RCT_ESTATE, "context belongs to device %d but device %d is current", c->device, dev);
    return RCT_OK;
}

bool stream_capturing(void *stream) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// Marks the end of the work a call just enqueued on `stream` for this context (nothing while the stream is
// being captured: that work runs when the graph is launched, which records the mark then).
cudaError_t mark_done(rct_ctx *c, void *stream) {
    if (stream_capturing(stream)) return cudaSuccess;
    if (!c->ev_done) {
        cudaError_t e = cudaEventCreateWithFlags(&c->ev_done, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaEventRecord(c->ev_done, static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess) c->done_recorded = true;
    return e;
}

// Waits until the device has finished every piece of work enqueued for this context (its passes on the
// caller's streams and its staging on its own copy stream); other contexts' work keeps running.
cudaError_t wait_idle(rct_ctx *c) {
    cudaError_t e = cudaSuccess;
    if (c->done_recorded && c->ev_done) e = cudaEventSynchronize(c->ev_done);
    if (e == cudaSuccess && c->copy_stream) e = cudaStreamSynchronize(c->copy_stream);
    return e;
}

// Passes already queued may still read a staging resource that is about to be replaced (a larger K, another
// storage type): wait for this context's work first.  Replacements happen on shape changes only, never per
// call.
void quiesce(rct_ctx *c) { (void)wait_idle(c); }

void free_slots(rct_ctx *c) {
    if (!c->slots.empty()) {
        quiesce(c);
        bump(c);
    }
    for (Slot &s : c->slots) {
        if (s.tex) cudaDestroyTextureObject(s.tex);
        if (s.arr) cudaFreeArray(s.arr);
    }
    c->slots.clear();
    c->slot_kind = -1;
    c->slot_dtype = -1;
}

// Channel format of a staged view for the given kernel kind and projection dtype.
cudaChannelFormatDesc slot_format(int kind, int dt) {
    if (dt == DT_F16) return cudaCreateChannelDescHalf();
    if (dt == DT_BF16 && kind == G_SOFT)
        return cudaCreateChannelDesc(16, 0, 0, 0, cudaChannelFormatKindUnsigned);
    return cudaCreateChannelDesc(32, 0, 0, 0, cudaChannelFormatKindFloat);  // F32, and BF16 widened
}

rct_status ensure_slots(rct_ctx *c, int n_slots) {
    if (!uses_tex(c)) return RCT_OK;
    const int kind = kernel_kind(c);
    if (c->slot_kind == kind && c->slot_dtype == c->dtype && (int)c->slots.size() >= n_slots) return RCT_OK;
    free_slots(c);
    const cudaChannelFormatDesc fmt = slot_format(kind, c->dtype);
    c->slots.resize(n_slots);
    for (int i = 0; i < n_slots; ++i) {
        Slot &s = c->slots[i];
        const unsigned flags = (kind == G_SOFT) ? cudaArrayTextureGather : cudaArrayDefault;
        cudaError_t e = cudaMallocArray(&s.arr, &fmt, c->W, c->H, flags);
        if (e != cudaSuccess) {
            free_slots(c);
            return e == cudaErrorMemoryAllocation ? fail(RCT_ENOMEM, "staging array allocation failed")
                                                  : cuda_fail(e, "cudaMallocArray");
        }
        cudaResourceDesc rd{};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = s.arr;
        cudaTextureDesc td{};
        td.addressMode[0] = cudaAddressModeBorder;   // zero outside the detector
        td.addressMode[1] = cudaAddressModeBorder;
        td.borderColor[0] = td.borderColor[1] = td.borderColor[2] = td.borderColor[3] = 0.0f;
        td.filterMode = (kind == G_TEXLIN) ? cudaFilterModeLinear : cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        e = cudaCreateTextureObject(&s.tex, &rd, &td, nullptr);
        if (e != cudaSuccess) {
            free_slots(c);
            return cuda_fail(e, "cudaCreateTextureObject");
        }
    }
    c->slot_kind = kind;
    c->slot_dtype = c->dtype;
    return RCT_OK;
}

rct_status ensure_copy_machinery(rct_ctx *c) {
    if (c->copy_stream) return RCT_OK;
    // Highest priority: staging work (copies and quad kernels) must get SMs while a large
    // backprojection grid is resident, or it would wait for the grid to drain.
    int least = 0, greatest = 0;
    RCT_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest), "cudaDeviceGetStreamPriorityRange");
    RCT_CUDA(cudaStreamCreateWithPriority(&c->copy_stream, cudaStreamNonBlocking, greatest), "cudaStreamCreate");
    for (int i = 0; i < 2; ++i) {
        RCT_CUDA(cudaEventCreateWithFlags(&c->ev_filled[i], cudaEventDisableTiming), "cudaEventCreate");
        RCT_CUDA(cudaEventCreateWithFlags(&c->ev_free[i], cudaEventDisableTiming), "cudaEventCreate");
    }
    return RCT_OK;
}

rct_status ensure_quads(rct_ctx *c, int n_slots) {
    if (!uses_quad(c)) return RCT_OK;
    const size_t need = (size_t)n_slots * layout_bytes(c);
    if (c->quad_alloc >= need) return RCT_OK;
    if (c->quad_buf) {
        quiesce(c);
        bump(c);
        cudaFree(c->quad_buf);
    }
    c->quad_buf = nullptr;
    c->quad_alloc = 0;
    cudaError_t e = cudaMalloc(&c->quad_buf, need);
    if (e != cudaSuccess) return fail(RCT_ENOMEM, "quad staging allocation of %zu bytes failed", need);
    c->quad_alloc = need;
    return RCT_OK;
}

void *quad_slot(const rct_ctx *c, int slot) {
    return static_cast<char *>(c->quad_buf) + (size_t)slot * layout_bytes(c);
}

size_t plane_floats(const rct_ctx *c) { return (size_t)c->L * c->L; }

rct_status ensure_parts(rct_ctx *c) {
    const int S = c->tune.view_split;
    if (S <= 1) return RCT_OK;
    const size_t need = (size_t)(S - 1) * c->z_count * plane_floats(c);
    if (c->part_alloc >= need) return RCT_OK;
    if (c->part) {
        quiesce(c);
        bump(c);
        cudaFree(c->part);
    }
    c->part = nullptr;
    c->part_alloc = 0;
    cudaError_t e = cudaMalloc(&c->part, need * sizeof(float));
    if (e != cudaSuccess) return fail(RCT_ENOMEM, "partial volumes of the view split: %zu bytes", need * sizeof(float));
    c->part_alloc = need;
    return RCT_OK;
}

// Adds the view split's partial volumes into planes [z, z + nz) of the volume (after a call's last pass).
rct_status add_partials(rct_ctx *c, int z, int nz, cudaStream_t s) {
    const int S = c->tune.view_split;
    if (S <= 1 || nz <= 0) return RCT_OK;
    const size_t at = (size_t)(z - c->z_first) * plane_floats(c);
    cudaError_t e = launch_add_partials(c->vol + at, c->part + at, (size_t)nz * plane_floats(c),
                                        (size_t)c->z_count * plane_floats(c), S - 1, s);
    return e == cudaSuccess ? RCT_OK : cuda_fail(e, "adding the partial volumes");
}

rct_status ensure_widen(rct_ctx *c, size_t elems) {
    if (c->widen_elems >= elems) return RCT_OK;
    if (c->widen_buf) {
        quiesce(c);
        bump(c);
        cudaFree(c->widen_buf);
    }
    c->widen_buf = nullptr;
    c->widen_elems = 0;
    cudaError_t e = cudaMalloc(&c->widen_buf, elems * sizeof(float));
    if (e != cudaSuccess) return fail(RCT_ENOMEM, "widening buffer allocation failed");
    c->widen_elems = elems;
    return RCT_OK;
}

LaunchConfig launch_config(const rct_ctx *c, int kind) {
    LaunchConfig lc{};
    lc.gather = kind;
    lc.dtype = c->dtype;
    lc.xv = c->tune.xvec;
    lc.zrun = c->tune.zrun;
    lc.bx = c->tune.block_x;
    lc.by = c->tune.block_y;
    lc.frame = (kind == G_SOFT && c->frame == RCT_FRAME_BLOCK) ? 1 : 0;
    lc.trunc = (kind == G_SOFT && c->index_rule == RCT_INDEX_TRUNC) ? 1 : 0;
    lc.split = c->tune.view_split;
    return lc;
}

void init_params(const rct_ctx *c, BpParams *p) {
    std::memset(p, 0, sizeof *p);
    // The kernels address plane z at vol + z * L * L; a slab context's buffer starts at plane z_first, so
    // the address it passes lies z_first planes before the buffer (integer arithmetic: only the slab's
    // planes are ever touched, the launches cover whole z-runs inside the slab).
    p->vol = reinterpret_cast<float *>(reinterpret_cast<uintptr_t>(c->vol) -
                                       static_cast<uintptr_t>(c->z_first) * c->L * c->L * sizeof(float));
    p->z_base = c->z_first;
    p->z_count = c->z_count;
#ifdef RCT_CHECK_BOUNDS
    p->vol_z0 = c->z_first;
    p->vol_elems = static_cast<long long>(c->z_count) * c->L * c->L;
#endif
    if (c->tune.view_split > 1 && c->part) {       // the partial volumes, addressed like vol
        p->part = reinterpret_cast<float *>(reinterpret_cast<uintptr_t>(c->part) -
                                            static_cast<uintptr_t>(c->z_first) * c->L * c->L * sizeof(float));
        p->part_stride = static_cast<long long>(c->z_count) * c->L * c->L;
    }
    p->L = c->L;
    p->W = c->W;
    p->H = c->H;
    p->cen = 0.5f * (c->L - 1);
    p->tex_zrun = tex_zrun_of(c);
    p->quad = load_layout(c);
    p->geo = (c->frame == RCT_FRAME_BLOCK) ? c->geo_dev : nullptr;
    p->viol = c->viol_dev;
    if (load_layout(c) != 0)
        p->qelems = static_cast<long long>(layout_bytes(c) /
                                           ((load_layout(c) == 2 ? 2 : 4) * dtype_size(c->dtype)));
    if (c->debug_qelems > 0) p->qelems = std::min(p->qelems, c->debug_qelems);
}

// FP32 view parameters for one view and kernel kind, from the FP64 fold.
void make_view(const rct_ctx *c, int view, int kind, ViewParams *vp) {
    const double *f = &c->fold[12 * (size_t)view];
    double m[12];
    std::memcpy(m, f, sizeof m);
    int cu = c->shift[2 * view], cv = c->shift[2 * view + 1];
    if (kind == G_TEXLIN) {
        // Hardware filtering samples texel centres at +0.5: fold (cu + 0.5, cv + 0.5) back in.
        for (int k = 0; k < 4; ++k) {
            m[k] += (cu + 0.5) * m[8 + k];
            m[4 + k] += (cv + 0.5) * m[8 + k];
        }
        cu = cv = 0;
    }
    set_view_geometry(vp, m, cu, cv);
    vp->tex = 0;
    vp->img = nullptr;
    vp->quad = nullptr;
}

cudaError_t prof_event(rct_ctx *c, cudaStream_t s) {
    if (c->prof_used == c->prof_events.size()) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        c->prof_events.push_back(e);
    }
    return cudaEventRecord(c->prof_events[c->prof_used++], s);
}

cudaError_t launch(rct_ctx *c, const LaunchConfig &lc, const BpParams &p, cudaStream_t s) {
    cudaError_t e;
    if (c->prof_on && (e = prof_event(c, s)) != cudaSuccess) return e;
    c->launches += 1;
    if (lc.gather == G_TEXLIN) {
        e = launch_bp_texlin(lc, p, s);
    } else if (lc.trunc) {
        e = lc.dtype == DT_F32 ? launch_bp_soft_f32_trunc(lc, p, s) : cudaErrorInvalidValue;
    } else {
        switch (lc.dtype) {
            case DT_F32: e = launch_bp_soft_f32(lc, p, s); break;
            case DT_F16: e = launch_bp_soft_f16(lc, p, s); break;
            case DT_BF16: e = launch_bp_soft_bf16(lc, p, s); break;
            default: e = cudaErrorInvalidValue;
        }
    }
    if (e == cudaSuccess && c->prof_on) e = prof_event(c, s);
    return e;
}

// Copy one view (device or host source) into a staging slot, widening BF16 for filtered textures.
rct_status stage_view(rct_ctx *c, Slot &slot, const void *src, bool from_host, cudaStream_t s) {
    const size_t px = (size_t)c->W * c->H;
    const cudaMemcpyKind kind = from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (c->dtype == DT_BF16 && c->slot_kind == G_TEXLIN) {
        const uint16_t *dev_src = static_cast<const uint16_t *>(src);
        if (from_host) return fail(RCT_ENOTSUP, "internal: host BF16 widening needs a device copy first");
        cudaError_t e = launch_widen_bf16(dev_src, c->widen_buf, px, s);
        if (e != cudaSuccess) return cuda_fail(e, "widen_bf16");
        RCT_CUDA(cudaMemcpy2DToArrayAsync(slot.arr, 0, 0, c->widen_buf, c->W * sizeof(float), c->W * sizeof(float),
                                          c->H, cudaMemcpyDeviceToDevice, s),
                 "cudaMemcpy2DToArrayAsync");
        return RCT_OK;
    }
    const size_t row = c->W * dtype_size(c->dtype);
    RCT_CUDA(cudaMemcpy2DToArrayAsync(slot.arr, 0, 0, src, row, row, c->H, kind, s), "cudaMemcpy2DToArrayAsync");
    return RCT_OK;
}

// Everything the host-input path needs: copy stream and events, 2K texture slots (two
// batches in flight), linear staging for LDG input and for BF16 bound to a filtered texture.
rct_status ensure_host_staging(rct_ctx *c) {
    rct_status st;
    const int kind = kernel_kind(c);
    const int K = c->tune.views_per_pass;
    const size_t view_bytes = (size_t)c->W * c->H * dtype_size(c->dtype);
    if ((st = ensure_copy_machinery(c))) return st;
    if ((st = ensure_slots(c, 2 * K))) return st;
    if ((st = ensure_quads(c, 2 * K))) return st;
    const bool linear = host_needs_linear(c);
    if (linear && c->lin_stage_bytes < 2 * K * view_bytes) {
        if (c->lin_stage) {
            quiesce(c);
            bump(c);
            cudaFree(c->lin_stage);
        }
        c->lin_stage = nullptr;
        c->lin_stage_bytes = 0;
        cudaError_t e = cudaMalloc(&c->lin_stage, 2 * K * view_bytes);
        if (e != cudaSuccess) return fail(RCT_ENOMEM, "host staging allocation failed");
        c->lin_stage_bytes = 2 * K * view_bytes;
    }
    if (kind == G_TEXLIN && c->dtype == DT_BF16 && (st = ensure_widen(c, (size_t)c->W * c->H))) return st;
    return RCT_OK;
}

// In-place iterative radix-2 DFT, X[k] = sum_n x[n] exp(-2 pi i k n / N), FP64 (host set-up only).
void host_fft(std::vector<std::complex<double>> &a) {
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = -2.0 * kPi / static_cast<double>(len);
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const std::complex<double> w(std::cos(ang * k), std::sin(ang * k));
                const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

rct_status validate_range(const rct_ctx *c, const void *proj, int first, int n) {
    if (!c->geometry_set) return fail(RCT_ESTATE, "rct_set_geometry has not been called");
    if (n < 0) return fail(RCT_EINVAL, "n = %d is negative", n);
    if (n > 0 && !proj) return fail(RCT_EINVAL, "null projection pointer");
    if (first < 0 || (long long)first + n > c->n_views)
        return fail(RCT_EINVAL, "views [%d, %lld) outside [0, %d)", first, (long long)first + n, c->n_views);
    return RCT_OK;
}

}  // namespace

// ----------------------------------------------------------------------------- C ABI

extern "C" {

int rct_version(void) { return 10000; }

const char *rct_last_error(void) { return g_last_error.c_str(); }

rct_status rct_fold_geometry(int L, int n_views, const double *matrices, const double origin[3],
                             const double spacing[3], double *fold_out, int *shift_out) {
    if (L <= 0 || n_views < 0) return fail(RCT_EINVAL, "L = %d, n_views = %d", L, n_views);
    if ((n_views > 0 && !matrices) || !origin || !spacing || (n_views > 0 && (!fold_out || !shift_out)))
        return fail(RCT_EINVAL, "null pointer");
    for (int k = 0; k < 3; ++k) {
        if (!std::isfinite(origin[k]) || !std::isfinite(spacing[k]) || !(spacing[k] > 0.0))
            return fail(RCT_EINVAL, "origin/spacing must be finite with spacing > 0");
    }
    const double cen = 0.5 * (L - 1);
    for (int v = 0; v < n_views; ++v) {
        const double *A = matrices + 12 * (size_t)v;
        for (int k = 0; k < 12; ++k)
            if (!std::isfinite(A[k])) return fail(RCT_EINVAL, "matrix of view %d is not finite", v);
        // P = A * S, S maps centred voxel coordinates to world: p_k = origin_k + (c_k + cen) * spacing_k
        double P[12];
        for (int r = 0; r < 3; ++r) {
            const double *a = A + 4 * r;
            P[4 * r + 0] = a[0] * spacing[0];
            P[4 * r + 1] = a[1] * spacing[1];
            P[4 * r + 2] = a[2] * spacing[2];
            P[4 * r + 3] = a[0] * (origin[0] + cen * spacing[0]) + a[1] * (origin[1] + cen * spacing[1]) +
                           a[2] * (origin[2] + cen * spacing[2]) + a[3];
        }
        // integer detector shift: the pixel nearest to where the volume centre projects
        int cu = 0, cv = 0;
        if (P[11] > 0.0) {
            const double pu = P[3] / P[11], pv = P[7] / P[11];
            if (std::fabs(pu) < 1.0e6) cu = static_cast<int>(std::lround(pu));
            if (std::fabs(pv) < 1.0e6) cv = static_cast<int>(std::lround(pv));
        }
        for (int k = 0; k < 4; ++k) {
            P[k] -= cu * P[8 + k];
            P[4 + k] -= cv * P[8 + k];
        }
        // Every voxel must lie in front of the source (w > 0), and its detector coordinate relative to
        // the shift must stay below 2^21 pixels, where the kernels' floor (an add of 1.5 * 2^23) is
        // exact.  (u', v', w) is affine in the voxel index and the view maps the volume's box onto the
        // convex hull of its corners' images while w > 0 on it, so the eight corners decide both.
        for (int corner = 0; corner < 8; ++corner) {
            const double c3[3] = {(corner & 1) ? cen : -cen, (corner & 2) ? cen : -cen, (corner & 4) ? cen : -cen};
            double q[3];
            for (int r = 0; r < 3; ++r) q[r] = P[4 * r] * c3[0] + P[4 * r + 1] * c3[1] + P[4 * r + 2] * c3[2] + P[4 * r + 3];
            if (!(q[2] > 0.0))
                return fail(RCT_EINVAL, "view %d: a corner of the volume lies at or behind the source plane (w = %g)",
                            v, q[2]);
            if (!(std::fabs(q[0] / q[2]) < 2097152.0 && std::fabs(q[1] / q[2]) < 2097152.0))
                return fail(RCT_EINVAL, "view %d: a corner of the volume projects 2^21 or more pixels from the "
                            "detector position of the volume centre", v);
        }
        std::memcpy(fold_out + 12 * (size_t)v, P, sizeof P);
        shift_out[2 * v] = cu;
        shift_out[2 * v + 1] = cv;
    }
    return RCT_OK;
}

rct_ctx *rct_create(int L, int det_w, int det_h, int n_views) {
    return rct_create_slab(L, det_w, det_h, n_views, 0, L);
}

rct_ctx *rct_create_slab(int L, int det_w, int det_h, int n_views, int z_first, int z_count) {
    if (L <= 0 || det_w <= 0 || det_h <= 0 || n_views <= 0) {
        fail(RCT_EINVAL, "rct_create: L=%d det_w=%d det_h=%d n_views=%d must be positive", L, det_w, det_h, n_views);
        return nullptr;
    }
    if (L > 2048) {
        fail(RCT_EINVAL, "rct_create: L=%d exceeds 2048", L);
        return nullptr;
    }
    if (z_first < 0 || z_count <= 0 || z_count > L - z_first) {
        fail(RCT_EINVAL, "rct_create_slab: planes [%d, %lld) are not a non-empty range inside [0, %d)", z_first,
             (long long)z_first + z_count, L);
        return nullptr;
    }
    // every z-run length divides kSlabAlign, so runs never cross a slab boundary
    if (z_first % kSlabAlign != 0 || ((z_first + z_count) % kSlabAlign != 0 && z_first + z_count != L)) {
        fail(RCT_EINVAL, "rct_create_slab: slab boundaries %d and %d must be multiples of %d planes (the end may "
             "be L = %d)", z_first, z_first + z_count, kSlabAlign, L);
        return nullptr;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cuda_fail(e, "rct_create: cudaGetDevice");
        return nullptr;
    }
    int max_w = 0, max_h = 0;
    cudaDeviceGetAttribute(&max_w, cudaDevAttrMaxTexture2DGatherWidth, dev);
    cudaDeviceGetAttribute(&max_h, cudaDevAttrMaxTexture2DGatherHeight, dev);
    if ((max_w > 0 && det_w > max_w) || (max_h > 0 && det_h > max_h)) {
        fail(RCT_EINVAL, "rct_create: detector %dx%d exceeds texture limits %dx%d", det_w, det_h, max_w, max_h);
        return nullptr;
    }
    rct_ctx *c = new rct_ctx();
    c->L = L;
    c->W = det_w;
    c->H = det_h;
    c->n_views = n_views;
    c->z_first = z_first;
    c->z_count = z_count;
    c->device = dev;
    c->tune = default_tuning(L);
    const size_t bytes = (size_t)z_count * L * L * sizeof(float);
    e = cudaMalloc(&c->vol, bytes);
    if (e != cudaSuccess) {
        fail(RCT_ENOMEM, "rct_create: volume allocation of %zu bytes failed (%s)", bytes, cudaGetErrorName(e));
        delete c;
        return nullptr;
    }
    c->fold.assign(12 * (size_t)n_views, 0.0);
    c->shift.assign(2 * (size_t)n_views, 0);
#ifdef RCT_CHECK_BOUNDS
    if (cudaMalloc(&c->viol_dev, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(c->viol_dev, 0, sizeof(unsigned long long)) != cudaSuccess) {
        fail(RCT_ENOMEM, "rct_create: violation counter allocation failed");
        cudaFree(c->vol);
        if (c->viol_dev) cudaFree(c->viol_dev);
        delete c;
        return nullptr;
    }
#endif
    c->id = g_next_id.fetch_add(1);
    {
        std::lock_guard<std::mutex> lk(g_reg_mu);
        g_live[c->id] = LiveEntry{c->gen, c};
    }
    return c;
}

void rct_destroy(rct_ctx *c) {
    if (!c) return;
    {
        std::lock_guard<std::mutex> lk(g_reg_mu);
        g_live.erase(c->id);
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    (void)wait_idle(c);
    free_slots(c);
    if (c->vol) cudaFree(c->vol);
    if (c->lin_stage) cudaFree(c->lin_stage);
    if (c->quad_buf) cudaFree(c->quad_buf);
    if (c->part) cudaFree(c->part);
    if (c->geo_dev) cudaFree(c->geo_dev);
    for (cudaEvent_t e : c->ev_slab) cudaEventDestroy(e);
    c->ev_slab.clear();
    if (c->viol_dev) cudaFree(c->viol_dev);
    if (c->filt_twiddle) cudaFree(c->filt_twiddle);
    if (c->filt_spectrum) cudaFree(c->filt_spectrum);
    if (c->filt_principal) cudaFree(c->filt_principal);
    if (c->widen_buf) cudaFree(c->widen_buf);
    for (int i = 0; i < 2; ++i) {
        if (c->ev_filled[i]) cudaEventDestroy(c->ev_filled[i]);
        if (c->ev_free[i]) cudaEventDestroy(c->ev_free[i]);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    for (cudaEvent_t e : c->prof_events) cudaEventDestroy(e);
    if (c->ev_done) cudaEventDestroy(c->ev_done);
    if (prev >= 0) cudaSetDevice(prev);
    delete c;
}

rct_status rct_set_geometry(rct_ctx *c, const double *matrices, const double origin[3], const double spacing[3]) {
    if (!c) return fail(RCT_EINVAL, "null context");
    if (!matrices || !origin || !spacing) return fail(RCT_EINVAL, "null geometry pointer");
    std::vector<double> fold(12 * (size_t)c->n_views);
    std::vector<int> shift(2 * (size_t)c->n_views);
    rct_status st = rct_fold_geometry(c->L, c->n_views, matrices, origin, spacing, fold.data(), shift.data());
    if (st != RCT_OK) return st;
    if ((st = check_ctx(c))) return st;
    std::vector<ViewGeo> geo(c->n_views);
    for (int v = 0; v < c->n_views; ++v) set_view_geo(&geo[v], &fold[12 * (size_t)v], shift[2 * v], shift[2 * v + 1]);
    if (!c->geo_dev) {
        cudaError_t e = cudaMalloc(&c->geo_dev, sizeof(ViewGeo) * c->n_views);
        if (e != cudaSuccess) {
            c->geo_dev = nullptr;
            return fail(RCT_ENOMEM, "geometry table allocation failed");
        }
    }
    // Passes already queued with a previous geometry read the block-frame table when they run:
    // let this context's work finish before it is overwritten (a fresh context has none).  Other
    // contexts' work on the device is not waited for.
    if (c->launches > 0) RCT_CUDA(wait_idle(c), "waiting for the context's queued work");
    if (c->geometry_set) bump(c);   // graphs captured before read the table in place
    if ((st = ensure_copy_machinery(c))) return st;
    RCT_CUDA(cudaMemcpyAsync(c->geo_dev, geo.data(), sizeof(ViewGeo) * c->n_views, cudaMemcpyHostToDevice,
                             c->copy_stream), "cudaMemcpyAsync(geometry)");
    RCT_CUDA(cudaStreamSynchronize(c->copy_stream), "cudaStreamSynchronize");
    c->fold.swap(fold);
    c->shift.swap(shift);
    c->geometry_set = true;
    return RCT_OK;
}

rct_status rct_set_precision(rct_ctx *c, int proj_dtype, int interp) {
    if (!c) return fail(RCT_EINVAL, "null context");
    if (proj_dtype < RCT_PROJ_F32 || proj_dtype > RCT_PROJ_BF16) return fail(RCT_EINVAL, "unknown dtype %d", proj_dtype);
    if (interp != RCT_INTERP_SOFT && interp != RCT_INTERP_TEX) return fail(RCT_EINVAL, "unknown interp %d", interp);
    if (c->frame == RCT_FRAME_BLOCK && (proj_dtype != RCT_PROJ_F32 || interp != RCT_INTERP_SOFT))
        return fail(RCT_ENOTSUP, "block frames need FP32 projections and software interpolation");
    if (c->index_rule == RCT_INDEX_TRUNC && (proj_dtype != RCT_PROJ_F32 || interp != RCT_INTERP_SOFT))
        return fail(RCT_ENOTSUP, "the truncating index rule needs FP32 projections and software interpolation");
    c->dtype = proj_dtype;
    c->interp = interp;
    return RCT_OK;
}

rct_status rct_set_frame(rct_ctx *c, int frame) {
    if (!c) return fail(RCT_EINVAL, "null context");
    if (frame != RCT_FRAME_GLOBAL && frame != RCT_FRAME_BLOCK) return fail(RCT_EINVAL, "unknown frame %d", frame);
    if (frame == RCT_FRAME_BLOCK && (c->dtype != DT_F32 || c->interp != RCT_INTERP_SOFT))
        return fail(RCT_ENOTSUP, "block frames need FP32 projections and software interpolation");
    if (frame == RCT_FRAME_BLOCK && c->index_rule == RCT_INDEX_TRUNC)
        return fail(RCT_ENOTSUP, "the truncating index rule runs in the global frame");
    c->frame = frame;
    return RCT_OK;
}

rct_status rct_set_filter(rct_ctx *c, double sdd, double pitch, const double *principal) {
    rct_status st = check_ctx(c);
    if (st) return st;
    if (!principal) return fail(RCT_EINVAL, "null principal points");
    if (!(std::isfinite(sdd) && sdd > 0.0 && std::isfinite(pitch) && pitch > 0.0))
        return fail(RCT_EINVAL, "source-detector distance and pitch must be finite and positive");
    for (int v = 0; v < 2 * c->n_views; ++v)
        if (!std::isfinite(principal[v])) return fail(RCT_EINVAL, "non-finite principal point");
    if (c->W > 8192) return fail(RCT_ENOTSUP, "ramp filter rows of %d pixels: at most 8192", c->W);
    int log2n = 4;                       // the transform works in blocks of 16 values per thread
    while ((1 << log2n) < 2 * c->W - 1) ++log2n;
    const int N = 1 << log2n;
    // The kernel h[n] = -2 / (pi^2 pitch^2 (4 n^2 - 1)) for |n| < W, placed circularly; its DFT is
    // real (h is real and even).  pitch (the convolution's quadrature weight) and 1/N (the inverse
    // transform's normalisation) are folded in.
    std::vector<std::complex<double>> hz(N, 0.0);
    for (int n = 0; n < c->W; ++n) {
        const double h = -2.0 / (kPi * kPi * pitch * pitch * (4.0 * n * n - 1.0));
        hz[n] = h;
        if (n > 0) hz[N - n] = h;
    }
    host_fft(hz);
    std::vector<float> spectrum(N);
    for (int k = 0; k < N; ++k) spectrum[k] = static_cast<float>(hz[k].real() * pitch / N);
    std::vector<float2> tw(N);
    for (int k = 0; k < N; ++k) {
        const double a = -2.0 * kPi * k / N;
        tw[k] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
    }
    std::vector<float2> pp(c->n_views);
    for (int v = 0; v < c->n_views; ++v)
        pp[v] = make_float2(static_cast<float>(principal[2 * v]), static_cast<float>(principal[2 * v + 1]));
    // Filter launches already queued read the old tables: let this context's work finish before they
    // are replaced (other contexts keep running).
    RCT_CUDA(wait_idle(c), "waiting for the context's queued work");
    if (c->filter_set) bump(c);     // graphs captured before point at the old tables
    if (c->filt_twiddle) cudaFree(c->filt_twiddle);
    if (c->filt_spectrum) cudaFree(c->filt_spectrum);
    if (c->filt_principal) cudaFree(c->filt_principal);
    c->filt_twiddle = nullptr;
    c->filt_spectrum = nullptr;
    c->filt_principal = nullptr;
    c->filter_set = false;
    if (cudaMalloc(&c->filt_twiddle, sizeof(float2) * N) != cudaSuccess ||
        cudaMalloc(&c->filt_spectrum, sizeof(float) * N) != cudaSuccess ||
        cudaMalloc(&c->filt_principal, sizeof(float2) * c->n_views) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(RCT_ENOMEM, "filter table allocation failed");
    }
    RCT_CUDA(cudaMemcpy(c->filt_twiddle, tw.data(), sizeof(float2) * N, cudaMemcpyHostToDevice), "cudaMemcpy");
    RCT_CUDA(cudaMemcpy(c->filt_spectrum, spectrum.data(), sizeof(float) * N, cudaMemcpyHostToDevice), "cudaMemcpy");
    RCT_CUDA(cudaMemcpy(c->filt_principal, pp.data(), sizeof(float2) * c->n_views, cudaMemcpyHostToDevice),
             "cudaMemcpy");
    c->filt.W = c->W;
    c->filt.H = c->H;
    c->filt.log2n = log2n;
    c->filt.sdd = static_cast<float>(sdd);
    c->filt.pitch = static_cast<float>(pitch);
    c->filt.twiddle = c->filt_twiddle;
    c->filt.spectrum = c->filt_spectrum;
    c->filt.principal = c->filt_principal;
    c->filter_set = true;
    return RCT_OK;
}

rct_status rct_filter_projections(rct_ctx *c, const float *d_raw, void *d_out, int out_dtype, int first_view, int n,
                                  void *stream) {
    rct_status st = check_ctx(c);
    if (st) return st;
    if (!c->filter_set) return fail(RCT_ESTATE, "rct_set_filter has not been called");
    if (out_dtype < RCT_PROJ_F32 || out_dtype > RCT_PROJ_BF16) return fail(RCT_EINVAL, "unknown dtype %d", out_dtype);
    if (n < 0) return fail(RCT_EINVAL, "n = %d is negative", n);
    if (first_view < 0 || (long long)first_view + n > c->n_views)
        return fail(RCT_EINVAL, "views [%d, %lld) outside [0, %d)", first_view, (long long)first_view + n, c->n_views);
    if (n == 0) return RCT_OK;
    if (!d_raw || !d_out) return fail(RCT_EINVAL, "null projection pointer");
    note_capture(c, stream);
    const size_t px = (size_t)c->W * c->H * n;
    if (out_dtype != RCT_PROJ_F32) {     // a narrower output written in place would overwrite unread input
        const char *r0 = reinterpret_cast<const char *>(d_raw), *r1 = r0 + px * sizeof(float);
        const char *o0 = static_cast<const char *>(d_out), *o1 = o0 + px * dtype_size(out_dtype);
        if (o0 < r1 && r0 < o1) return fail(RCT_EINVAL, "a 16-bit output must not overlap the raw input");
    } else if (d_out != static_cast<const void *>(d_raw)) {
        const char *r0 = reinterpret_cast<const char *>(d_raw), *r1 = r0 + px * sizeof(float);
        const char *o0 = static_cast<const char *>(d_out), *o1 = o0 + px * sizeof(float);
        if (o0 < r1 && r0 < o1) return fail(RCT_EINVAL, "output overlaps the input without coinciding with it");
    }
    FilterParams f = c->filt;
    f.principal = c->filt_principal + first_view;
    cudaError_t e = launch_ramp_filter(f, d_raw, d_out, out_dtype, n, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "ramp filter launch");
    RCT_CUDA(mark_done(c, stream), "cudaEventRecord");
    return RCT_OK;
}

rct_status rct_debug_bound_violations(rct_ctx *c, unsigned long long *count) {
    rct_status st = check_ctx(c);
    if (st) return st;
    if (!count) return fail(RCT_EINVAL, "null pointer");
#ifdef RCT_CHECK_BOUNDS
    if (!c->viol_dev) {
        *count = 0;
        return RCT_OK;
    }
    RCT_CUDA(wait_idle(c), "waiting for the context's queued work");
    RCT_CUDA(cudaMemcpy(count, c->viol_dev, sizeof *count, cudaMemcpyDeviceToHost), "cudaMemcpy");
    return RCT_OK;
#else
    return fail(RCT_ENOTSUP, "this library was built without bounds checks");
#endif
}

rct_status rct_debug_lower_bound_limit(rct_ctx *c, long long staged_elems) {
    rct_status st = check_ctx(c);
    if (st) return st;
    if (staged_elems < 0) return fail(RCT_EINVAL, "negative limit");
#ifdef RCT_CHECK_BOUNDS
    c->debug_qelems = staged_elems;
    return RCT_OK;
#else
    return fail(RCT_ENOTSUP, "this library was built without bounds checks");
#endif
}

rct_status rct_set_index_rule(rct_ctx *c, int rule) {
    if (!c) return fail(RCT_EINVAL, "null context");
    if (rule != RCT_INDEX_FLOOR && rule != RCT_INDEX_TRUNC) return fail(RCT_EINVAL, "unknown index rule %d", rule);
    if (rule == RCT_INDEX_TRUNC && (c->dtype != DT_F32 || c->interp != RCT_INTERP_SOFT || c->frame != RCT_FRAME_GLOBAL))
        return fail(RCT_ENOTSUP, "the truncating index rule needs FP32 projections, software interpolation and the "
                                 "global frame");
    c->index_rule = rule;
    return RCT_OK;
}

rct_status rct_get_index_rule(const rct_ctx *c, int *rule) {
    if (!c || !rule) return fail(RCT_EINVAL, "null pointer");
    *rule = c->index_rule;
    return RCT_OK;
}

rct_status rct_set_geometry_rabbitct(rct_ctx *c, const float *matrices, float O, float MM) {
    if (!c) return fail(RCT_EINVAL, "null context");
    if (!matrices) return fail(RCT_EINVAL, "null matrices");
    std::vector<double> rm(12 * (size_t)c->n_views);
    for (int v = 0; v < c->n_views; ++v)
        for (int r = 0; r < 3; ++r)
            for (int col = 0; col < 4; ++col)
                rm[12 * (size_t)v + 4 * r + col] = static_cast<double>(matrices[12 * (size_t)v + 3 * col + r]);
    const double origin[3] = {O, O, O}, spacing[3] = {MM, MM, MM};
    return rct_set_geometry(c, rm.data(), origin, spacing);
}

rct_status rct_get_frame(const rct_ctx *c, int *frame) {
    if (!c || !frame) return fail(RCT_EINVAL, "null pointer");
    *frame = c->frame;
    return RCT_OK;
}

rct_status rct_set_tuning(rct_ctx *c, const rct_tuning *t) {
    if (!c || !t) return fail(RCT_EINVAL, "null pointer");
    rct_tuning n = c->tune;
    if (t->views_per_pass) n.views_per_pass = t->views_per_pass;
    if (t->zrun) n.zrun = t->zrun;
    if (t->xvec) n.xvec = t->xvec;
    if (t->block_x) n.block_x = t->block_x;
    if (t->block_y) n.block_y = t->block_y;
    if (t->gather) n.gather = t->gather;
    if (t->tex_zrun) n.tex_zrun = t->tex_zrun;
    if (n.views_per_pass < 1 || n.views_per_pass > KMAX)
        return fail(RCT_EINVAL, "views_per_pass %d outside 1..%d", n.views_per_pass, KMAX);
    if (n.zrun != 1 && n.zrun != 2 && n.zrun != 4 && n.zrun != 8 && n.zrun != 16)
        return fail(RCT_EINVAL, "zrun %d not in {1,2,4,8,16}", n.zrun);
    if (n.zrun == 16 && n.xvec > 2) return fail(RCT_EINVAL, "zrun 16 needs xvec <= 2");
    if (n.xvec != 1 && n.xvec != 2 && n.xvec != 4) return fail(RCT_EINVAL, "xvec %d not in {1,2,4}", n.xvec);
    if (c->L % n.xvec != 0) return fail(RCT_EINVAL, "xvec %d does not divide L = %d", n.xvec, c->L);
    if (n.block_x < 1 || n.block_y < 1 || n.block_x * n.block_y > 512 || (n.block_x * n.block_y) % 32 != 0)
        return fail(RCT_EINVAL, "block %dx%d: need a multiple of 32 threads, at most 512", n.block_x, n.block_y);
    if (n.gather < RCT_GATHER_AUTO || n.gather > RCT_GATHER_DQUAD) return fail(RCT_EINVAL, "unknown gather %d", n.gather);
    if (n.tex_zrun < 0 || n.tex_zrun > 16) return fail(RCT_EINVAL, "tex_zrun %d outside 0..16", n.tex_zrun);
    if (t->view_split) n.view_split = t->view_split;
    if (n.view_split != 1 && n.view_split != 2 && n.view_split != 4 && n.view_split != 8)
        return fail(RCT_EINVAL, "view_split %d not in {1,2,4,8}", n.view_split);
    c->tune = n;
    return RCT_OK;
}

rct_status rct_get_tuning(const rct_ctx *c, rct_tuning *out) {
    if (!c || !out) return fail(RCT_EINVAL, "null pointer");
    *out = c->tune;
    if (out->gather == RCT_GATHER_AUTO) out->gather = RCT_GATHER_TLD4;
    out->tex_zrun = tex_zrun_of(c);
    return RCT_OK;
}

rct_status rct_reset_volume(rct_ctx *c, void *stream) {
    rct_status st = check_ctx(c);
    if (st) return st;
    note_capture(c, stream);
    c->vol_zero_pending = true;
    return RCT_OK;
}

static rct_status materialise_zero(rct_ctx *c, cudaStream_t s) {
    if (!c->vol_zero_pending) return RCT_OK;
    RCT_CUDA(cudaMemsetAsync(c->vol, 0, (size_t)c->z_count * c->L * c->L * sizeof(float), s), "cudaMemsetAsync");
    c->vol_zero_pending = false;
    return RCT_OK;
}

rct_status rct_backproject(rct_ctx *c, const void *d_proj, int first_view, int n, void *stream) {
    rct_status st = check_ctx(c);
    if (st) return st;
    note_capture(c, stream);
    if ((st = validate_range(c, d_proj, first_view, n))) return st;
    if (n == 0) return RCT_OK;
    if ((st = check_route(c))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int kind = kernel_kind(c);
    const int K = c->tune.views_per_pass;
    const bool tex = uses_tex(c);
    const bool quad = uses_quad(c);
    const bool staged = tex || quad;
    if (staged && (st = ensure_copy_machinery(c))) return st;
    if ((st = ensure_slots(c, 2 * K))) return st;
    if ((st = ensure_quads(c, 2 * K))) return st;
    if ((st = ensure_parts(c))) return st;
    if (kind == G_TEXLIN && c->dtype == DT_BF16 && (st = ensure_widen(c, (size_t)c->W * c->H))) return st;
    const LaunchConfig lc = launch_config(c, kind);
    const size_t view_bytes = (size_t)c->W * c->H * dtype_size(c->dtype);
    const char *base = static_cast<const char *>(d_proj);

    // Staged routes (texture arrays, quad images) stage each batch into one of two slot groups
    // on the copy stream, so the staging of batch b+1 overlaps the pass of batch b.  Fork: the
    // copy stream first waits for the work already queued on `stream`.
    if (staged) {
        RCT_CUDA(cudaEventRecord(c->ev_free[0], s), "cudaEventRecord");
        RCT_CUDA(cudaEventRecord(c->ev_free[1], s), "cudaEventRecord");
    }
    BpParams p;
    init_params(c, &p);
    int batch = 0;
    for (int b = 0; b < n; b += K, ++batch) {
        const int g = batch & 1;
        const int kb = std::min(K, n - b);
        p.K = kb;
        p.first_view = first_view + b;
        p.accumulate = c->vol_zero_pending ? 0 : 1;
        p.accumulate_part = b > 0 ? 1 : 0;       // the call's first pass writes the partial volumes
        if (staged) RCT_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_free[g], 0), "cudaStreamWaitEvent");
        for (int k = 0; k < kb; ++k) {
            ViewParams &vp = p.view[k];
            make_view(c, first_view + b + k, kind, &vp);
            const void *src = base + (size_t)(b + k) * view_bytes;
            vp.img = src;
            if (tex) {
                Slot &slot = c->slots[g * K + k];
                if ((st = stage_view(c, slot, src, false, c->copy_stream))) return st;
                vp.tex = slot.tex;
            }
            if (quad) vp.quad = quad_slot(c, g * K + k);
        }
        if (quad) {                  // the batch's views into its consecutive slots, one launch
            cudaError_t e = launch_stage_layout(c, base + (size_t)b * view_bytes, quad_slot(c, g * K), kb,
                                                c->copy_stream);
            if (e != cudaSuccess) return cuda_fail(e, "quad/pair staging kernel");
        }
        if (staged) {
            RCT_CUDA(cudaEventRecord(c->ev_filled[g], c->copy_stream), "cudaEventRecord");
            RCT_CUDA(cudaStreamWaitEvent(s, c->ev_filled[g], 0), "cudaStreamWaitEvent");
        }
        cudaError_t e = launch(c, lc, p, s);
        if (e != cudaSuccess) return cuda_fail(e, "backprojection launch");
        c->vol_zero_pending = false;
        if (staged) RCT_CUDA(cudaEventRecord(c->ev_free[g], s), "cudaEventRecord");
    }
    if ((st = add_partials(c, c->z_first, c->z_count, s))) return st;
    RCT_CUDA(mark_done(c, stream), "cudaEventRecord");
    return RCT_OK;
}

namespace {

// The host-input path (see rct_backproject_host).  With read_dst, the last pass runs as z-slabs and
// each slab's planes are copied to read_dst on the copy stream as soon as that slab is done, so the
// read-back overlaps the rest of the pass; `stream` then waits for the last copy.
rct_status backproject_host_impl(rct_ctx *c, const void *h_proj, int first_view, int n, void *stream,
                                 float *read_dst) {
    rct_status st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int kind = kernel_kind(c);
    const int K = c->tune.views_per_pass;
    const size_t view_bytes = (size_t)c->W * c->H * dtype_size(c->dtype);
    if ((st = check_route(c))) return st;
    if ((st = ensure_host_staging(c))) return st;
    if ((st = ensure_parts(c))) return st;
    const bool tex = uses_tex(c);
    const bool quad = uses_quad(c);
    const bool linear = host_needs_linear(c);
    const LaunchConfig lc = launch_config(c, kind);
    const char *base = static_cast<const char *>(h_proj);

    // Fork: the copy stream must not run ahead of work already queued on `stream`
    // that still reads the staging buffers.
    RCT_CUDA(cudaEventRecord(c->ev_free[0], s), "cudaEventRecord");
    RCT_CUDA(cudaEventRecord(c->ev_free[1], s), "cudaEventRecord");

    BpParams p;
    init_params(c, &p);
    int batch = 0;
    for (int b = 0; b < n; b += K, ++batch) {
        const int g = batch & 1;
        const int kb = std::min(K, n - b);
        // copy stream: wait until group g's previous pass is done, then fill it
        RCT_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_free[g], 0), "cudaStreamWaitEvent");
        p.K = kb;
        p.first_view = first_view + b;
        p.accumulate = c->vol_zero_pending ? 0 : 1;
        p.accumulate_part = b > 0 ? 1 : 0;
        // the batch's views sit back to back in host memory and go to consecutive linear slots: one copy
        char *lin0 = linear ? static_cast<char *>(c->lin_stage) + (size_t)(g * K) * view_bytes : nullptr;
        if (linear)
            RCT_CUDA(cudaMemcpyAsync(lin0, base + (size_t)b * view_bytes, (size_t)kb * view_bytes,
                                     cudaMemcpyHostToDevice, c->copy_stream), "cudaMemcpyAsync");
        for (int k = 0; k < kb; ++k) {
            const void *src = base + (size_t)(b + k) * view_bytes;
            ViewParams &vp = p.view[k];
            make_view(c, first_view + b + k, kind, &vp);
            Slot *slot = tex ? &c->slots[g * K + k] : nullptr;
            if (linear) {
                char *lin = lin0 + (size_t)k * view_bytes;
                if (slot && (st = stage_view(c, *slot, lin, false, c->copy_stream))) return st;
                if (quad) vp.quad = quad_slot(c, g * K + k);
                vp.img = lin;
            } else if (slot) {
                if ((st = stage_view(c, *slot, src, true, c->copy_stream))) return st;
            }
            if (slot) vp.tex = slot->tex;
        }
        if (linear && quad) {        // the batch's views into its consecutive slots, one launch
            cudaError_t e = launch_stage_layout(c, lin0, quad_slot(c, g * K), kb, c->copy_stream);
            if (e != cudaSuccess) return cuda_fail(e, "quad/pair staging kernel");
        }
        RCT_CUDA(cudaEventRecord(c->ev_filled[g], c->copy_stream), "cudaEventRecord");
        RCT_CUDA(cudaStreamWaitEvent(s, c->ev_filled[g], 0), "cudaStreamWaitEvent");
        if (read_dst && b + kb >= n) {
            // last pass: z-slabs of a whole number of z-runs, each copied out when it is done
            const int R = c->tune.zrun;
            const int slab = ((c->z_count + kReadSlabs - 1) / kReadSlabs + R - 1) / R * R;
            const size_t plane = (size_t)c->L * c->L;
            const int z_end = c->z_first + c->z_count;
            int i = 0;
            for (int z = c->z_first; z < z_end; z += slab, ++i) {
                p.z_base = z;
                p.z_count = std::min(slab, z_end - z);
                cudaError_t e = launch(c, lc, p, s);
                if (e != cudaSuccess) return cuda_fail(e, "backprojection launch");
                if ((st = add_partials(c, z, p.z_count, s))) return st;
                const size_t at = (size_t)(z - c->z_first) * plane;
                RCT_CUDA(cudaEventRecord(c->ev_slab[i], s), "cudaEventRecord");
                RCT_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_slab[i], 0), "cudaStreamWaitEvent");
                RCT_CUDA(cudaMemcpyAsync(read_dst + at, c->vol + at, sizeof(float) * plane * p.z_count,
                                         cudaMemcpyDefault, c->copy_stream),
                         "cudaMemcpyAsync(volume slab)");
            }
            p.z_base = c->z_first;
            p.z_count = c->z_count;
            RCT_CUDA(cudaEventRecord(c->ev_slab[i], c->copy_stream), "cudaEventRecord");
            RCT_CUDA(cudaStreamWaitEvent(s, c->ev_slab[i], 0), "cudaStreamWaitEvent");
        } else {
            cudaError_t e = launch(c, lc, p, s);
            if (e != cudaSuccess) return cuda_fail(e, "backprojection launch");
            if (b + kb >= n && (st = add_partials(c, c->z_first, c->z_count, s))) return st;
        }
        c->vol_zero_pending = false;
        RCT_CUDA(cudaEventRecord(c->ev_free[g], s), "cudaEventRecord");
    }
    RCT_CUDA(mark_done(c, stream), "cudaEventRecord");
    return RCT_OK;
}

}  // namespace

rct_status rct_backproject_host(rct_ctx *c, const void *h_proj, int first_view, int n, void *stream) {
    rct_status st = check_ctx(c);
    if (st) return st;
    note_capture(c, stream);
    if ((st = validate_range(c, h_proj, first_view, n))) return st;
    if (n == 0) return RCT_OK;
    return backproject_host_impl(c, h_proj, first_view, n, stream, nullptr);
}

rct_status rct_backproject_host_read(rct_ctx *c, const void *h_proj, int first_view, int n, float *dst,
                                     void *stream) {
    rct_status st = check_ctx(c);
    if (st) return st;
    note_capture(c, stream);
    if ((st = validate_range(c, h_proj, first_view, n))) return st;
    if (!dst) return fail(RCT_EINVAL, "null destination");
    if (n == 0) return rct_read_volume(c, dst, stream);
    if ((st = ensure_copy_machinery(c))) return st;
    while (c->ev_slab.size() < kReadSlabs + 1) {
        cudaEvent_t e;
        RCT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
        c->ev_slab.push_back(e);
    }
    return backproject_host_impl(c, h_proj, first_view, n, stream, dst);
}

rct_status rct_read_volume(rct_ctx *c, float *dst, void *stream) {
    rct_status st = check_ctx(c);
    if (st) return st;
    note_capture(c, stream);
    if (!dst) return fail(RCT_EINVAL, "null destination");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = materialise_zero(c, s))) return st;
    RCT_CUDA(cudaMemcpyAsync(dst, c->vol, (size_t)c->z_count * c->L * c->L * sizeof(float), cudaMemcpyDefault, s),
             "cudaMemcpyAsync(volume)");
    RCT_CUDA(mark_done(c, stream), "cudaEventRecord");
    return RCT_OK;
}

rct_status rct_write_volume(rct_ctx *c, const float *src, void *stream) {
    rct_status st = check_ctx(c);
    if (st) return st;
    note_capture(c, stream);
    if (!src) return fail(RCT_EINVAL, "null source");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    RCT_CUDA(cudaMemcpyAsync(c->vol, src, (size_t)c->z_count * c->L * c->L * sizeof(float), cudaMemcpyDefault, s),
             "cudaMemcpyAsync(volume)");
    c->vol_zero_pending = false;
    RCT_CUDA(mark_done(c, stream), "cudaEventRecord");
    return RCT_OK;
}

float *rct_volume_device_ptr(rct_ctx *c) {
    if (!c) {
        fail(RCT_EINVAL, "null context");
        return nullptr;
    }
    if (c->vol_zero_pending) {
        // A caller reading the buffer directly must see zeros: materialise on the legacy stream.
        if (materialise_zero(c, nullptr) != RCT_OK) return nullptr;
        (void)mark_done(c, nullptr);
    }
    return c->vol;
}

rct_status rct_get_shape(const rct_ctx *c, int *L, int *det_w, int *det_h, int *n_views) {
    if (!c) return fail(RCT_EINVAL, "null context");
    if (L) *L = c->L;
    if (det_w) *det_w = c->W;
    if (det_h) *det_h = c->H;
    if (n_views) *n_views = c->n_views;
    return RCT_OK;
}

rct_status rct_get_slab(const rct_ctx *c, int *z_first, int *z_count) {
    if (!c) return fail(RCT_EINVAL, "null context");
    if (z_first) *z_first = c->z_first;
    if (z_count) *z_count = c->z_count;
    return RCT_OK;
}

rct_status rct_get_precision(const rct_ctx *c, int *proj_dtype, int *interp) {
    if (!c) return fail(RCT_EINVAL, "null context");
    if (proj_dtype) *proj_dtype = c->dtype;
    if (interp) *interp = c->interp;
    return RCT_OK;
}

int64_t rct_launch_count(const rct_ctx *c) { return c ? c->launches : -1; }

rct_status rct_prepare(rct_ctx *c, int host_input) {
    rct_status st = check_ctx(c);
    if (st) return st;
    if ((st = check_route(c))) return st;
    if ((uses_tex(c) || uses_quad(c)) && (st = ensure_copy_machinery(c))) return st;
    if ((st = ensure_slots(c, 2 * c->tune.views_per_pass))) return st;
    if ((st = ensure_quads(c, 2 * c->tune.views_per_pass))) return st;
    if ((st = ensure_parts(c))) return st;
    if (kernel_kind(c) == G_TEXLIN && c->dtype == DT_BF16 && (st = ensure_widen(c, (size_t)c->W * c->H))) return st;
    if (host_input && (st = ensure_host_staging(c))) return st;
    return RCT_OK;
}

size_t rct_footprint_bytes(int L, int det_w, int det_h, int proj_dtype, int views_per_pass, int host_input) {
    if (L <= 0 || det_w <= 0 || det_h <= 0 || views_per_pass <= 0) return 0;
    const size_t vol = (size_t)L * L * L * sizeof(float);
    const size_t px = (size_t)det_w * det_h;
    const size_t esz = dtype_size(proj_dtype);
    const size_t slots = (size_t)2 * views_per_pass;                        // two batches in flight
    size_t bytes = vol + slots * px * (proj_dtype == DT_BF16 ? 4 : esz);   // BF16 may be widened for TEX
    bytes += slots * quad_bytes(det_w, det_h, proj_dtype);                    // quad staging (worst case)
    if (host_input) bytes += 2 * (size_t)views_per_pass * px * esz;         // linear staging (worst case)
    return bytes;
}

struct rct_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<std::pair<uint64_t, uint64_t>> uses;   // (context id, generation) at capture
};

rct_status rct_graph_begin(void *stream) {
    if (!stream) return fail(RCT_EINVAL, "graph capture needs a non-default stream");
    RCT_CUDA(cudaStreamBeginCapture(static_cast<cudaStream_t>(stream), cudaStreamCaptureModeThreadLocal),
             "cudaStreamBeginCapture");
    if (g_capturing++ == 0) g_captured.clear();
    return RCT_OK;
}

rct_status rct_graph_end(void *stream, rct_graph **out) {
    if (!stream || !out) return fail(RCT_EINVAL, "null argument");
    *out = nullptr;
    std::vector<std::pair<uint64_t, uint64_t>> uses = g_captured;
    if (g_capturing > 0 && --g_capturing == 0) g_captured.clear();
    cudaGraph_t g = nullptr;
    RCT_CUDA(cudaStreamEndCapture(static_cast<cudaStream_t>(stream), &g), "cudaStreamEndCapture");
    // Kernel nodes keep the priority of the stream they were captured on (the staging kernels run on a
    // high-priority copy stream so that they slip in between the blocks of a running pass); a graph
    // honours those priorities only when instantiated with this flag, else every node runs at the
    // launch stream's priority and each staging waits for the pass ahead of it to drain.
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiateWithFlags(&exec, g, cudaGraphInstantiateFlagUseNodePriority);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    rct_graph *r = new rct_graph();
    r->graph = g;
    r->exec = exec;
    std::sort(uses.begin(), uses.end());
    uses.erase(std::unique(uses.begin(), uses.end()), uses.end());
    r->uses = std::move(uses);
    *out = r;
    return RCT_OK;
}

rct_status rct_graph_launch(rct_graph *g, void *stream) {
    if (!g) return fail(RCT_EINVAL, "null graph");
    std::vector<rct_ctx *> used;
    {
        std::lock_guard<std::mutex> lk(g_reg_mu);
        for (const auto &u : g->uses) {
            const auto it = g_live.find(u.first);
            if (it == g_live.end())
                return fail(RCT_ESTATE, "a context this graph was captured with has been destroyed");
            if (it->second.gen != u.second)
                return fail(RCT_ESTATE, "a context this graph was captured with has replaced its staging, "
                                        "geometry table or filter tables since: capture the graph again");
            used.push_back(it->second.ctx);
        }
    }
    RCT_CUDA(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)), "cudaGraphLaunch");
    // the replay is now the last work of every context it uses
    for (rct_ctx *c : used) RCT_CUDA(mark_done(c, stream), "cudaEventRecord");
    return RCT_OK;
}

void rct_graph_destroy(rct_graph *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

rct_status rct_profile_kernels(rct_ctx *c, int enable) {
    rct_status st = check_ctx(c);
    if (st) return st;
    c->prof_on = enable != 0;
    c->prof_used = 0;
    return RCT_OK;
}

rct_status rct_profile_read(rct_ctx *c, double *kernel_ms, int64_t *kernel_launches) {
    rct_status st = check_ctx(c);
    if (st) return st;
    if (!kernel_ms || !kernel_launches) return fail(RCT_EINVAL, "null pointer");
    double total = 0.0;
    if (c->prof_used > 0) RCT_CUDA(cudaEventSynchronize(c->prof_events[c->prof_used - 1]), "cudaEventSynchronize");
    for (size_t i = 0; i + 1 < c->prof_used; i += 2) {
        float ms = 0.f;
        RCT_CUDA(cudaEventElapsedTime(&ms, c->prof_events[i], c->prof_events[i + 1]), "cudaEventElapsedTime");
        total += ms;
    }
    *kernel_ms = total;
    *kernel_launches = static_cast<int64_t>(c->prof_used / 2);
    c->prof_used = 0;
    return RCT_OK;
}

rct_status rct_convert_projections(const float *d_src, void *d_dst, size_t n, int dtype, void *stream) {
    if (n > 0 && (!d_src || !d_dst)) return fail(RCT_EINVAL, "null pointer");
    if (dtype < RCT_PROJ_F32 || dtype > RCT_PROJ_BF16) return fail(RCT_EINVAL, "unknown dtype %d", dtype);
    cudaError_t e = launch_convert(d_src, d_dst, n, dtype, static_cast<cudaStream_t>(stream));
    if (e == cudaErrorMisalignedAddress) return fail(RCT_EINVAL, "source must be 16-byte and destination 8-byte aligned");
    if (e != cudaSuccess) return cuda_fail(e, "conversion kernel");
    return RCT_OK;
}

}  // extern "C"

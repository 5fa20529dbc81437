// api.cu -- the C ABI of libtsplat.so (include/tsplat.h): argument checks,
// workspace management and the order of the pipeline steps.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "launch.h"

using namespace tsp;

namespace {

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct tsp_context {
    int device = 0;
    tsp_options opt{};
    std::string err;
    size_t held = 0;
    // per (view, Gaussian)
    Buf rect, depth, touched, rec, oref, color, moments, vres0, vres1, vres2, vres3;
    // per tile
    Buf tiles, tile_off, span_sum, queue;
    Buf gacc;                       // render backward: per (view, Gaussian) 2D gradients
    Buf reg;                        // regularization: neighbour grid, components, neighbours
    int resident_ctas = 0;          // CTAs of the persistent raster resident at once
    // pairs
    Buf pairs, pairs_tmp;
    uint64_t want_pairs = 0;
    Buf dstatus, stats;
    uint32_t* h_status = nullptr;   // pinned, 8 words (the device status word's copy)
    // track gate (tsp_set_track_gate): device word, value it must reach, limit
    const uint32_t* gate_flag = nullptr;
    uint32_t gate_value = 0;
    long long gate_timeout_us = 0;
    // workspace allocator (tsp_set_allocator); nullptr: cudaMalloc / cudaFree
    tsp_alloc_fn alloc_fn = nullptr;
    tsp_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    cudaEvent_t ev[8] = {};         // stage boundaries (stage_timing)
    bool timed = false;             // the last call recorded ev[]
    // staging for tsp_fit_motion_host: tracks stream in on copy_stream, one event
    // per view group, while the Gaussians are binned on the caller's stream
    Buf st_in, st_out, st_tracks;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t group_ev[32] = {};
    // last call
    size_t last_R = 0;              // (view, Gaussian) records of the last call
    uint32_t last_NT = 0;
    // moments of the last single-frame fit: [last_fit_V][last_fit_n][16], else -1
    int last_fit_n = -1, last_fit_V = -1;
    const uint32_t* last_knn_path = nullptr;   // device [2] of the last neighbour search
    // the tile lists in the workspace come from tsp_render with these arguments
    // (then tsp_render_backward on the same arguments reuses them)
    bool render_bins = false;
    const void* render_ptrs[4] = {};
    int render_n = 0, render_deg = 0;
    std::vector<tsp_camera> render_cams;
};

namespace {

constexpr size_t kAlign = 256;
// Autotuner candidates (tile width, tile height, raster variant), in the order of
// tsp_autotune's fit_ms: the warp-shuffle variant exists for 16 x 16 tiles only.
constexpr int kTuneCandidates = TSP_TUNE_CANDIDATES;
constexpr int kTuneTable[kTuneCandidates][3] = {{16, 16, 0}, {16, 16, 5}, {16, 16, 2}, {16, 16, 1},
                                                 {16, 16, 4}, {32, 8, 0}, {32, 8, 5}};

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// An NVTX range over the launches of one pipeline step ("tsp:raster", ...), so
// that profiler captures can be sliced by step (ncu --nvtx --nvtx-include).
struct StageRange {
    explicit StageRange(const char* name) { nvtxRangePushA(name); }
    ~StageRange() { nvtxRangePop(); }
    StageRange(const StageRange&) = delete;
    StageRange& operator=(const StageRange&) = delete;
};

tsp_status fail(tsp_context* c, tsp_status s, const std::string& msg)
{
    if (c) c->err = msg;
    return s;
}

tsp_status cuda_fail(tsp_context* c, cudaError_t e, const char* what)
{
    return fail(c, TSP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define TSP_CUDA(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

class DeviceGuard {
public:
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&old_);
        if (old_ != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() { cudaSetDevice(old_); }

private:
    int old_ = 0;
};

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

tsp_status ensure(tsp_context* ctx, Buf& b, size_t need)
{
    if (need <= b.bytes) return TSP_OK;
    size_t nb = align_up(need > b.bytes + b.bytes / 4 ? need : b.bytes + b.bytes / 4);
    const size_t after = ctx->held - b.bytes + nb;
    if (ctx->opt.budget_bytes > 0 && after > (size_t)ctx->opt.budget_bytes) {
        nb = align_up(need);
        if (ctx->held - b.bytes + nb > (size_t)ctx->opt.budget_bytes)
            return fail(ctx, TSP_ERR_BUDGET, "workspace of " + std::to_string(ctx->held - b.bytes + nb) +
                                                 " bytes exceeds the budget");
    }
    if (b.p) {
        if (ctx->free_fn) {
            // work queued earlier may still use the block: hand it back only once
            // the device is idle, as cudaFree would
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaDeviceSynchronize");
            ctx->free_fn(b.p, b.bytes, ctx->device, ctx->alloc_user);
        } else {
            cudaError_t e = cudaFree(b.p);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFree");
        }
        ctx->held -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    if (ctx->alloc_fn) {
        void* p = ctx->alloc_fn(nb, ctx->device, ctx->alloc_user);
        if (!p) return fail(ctx, TSP_ERR_OOM, "the allocator refused " + std::to_string(nb) + " bytes");
        if (!aligned(p, kAlign)) {
            ctx->free_fn(p, nb, ctx->device, ctx->alloc_user);
            return fail(ctx, TSP_ERR_OOM, "the allocator returned a block not aligned to 256 bytes");
        }
        b.p = p;
    } else {
        cudaError_t e = cudaMalloc(&b.p, nb);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return fail(ctx, TSP_ERR_OOM, "cudaMalloc of " + std::to_string(nb) + " bytes failed");
        }
    }
    b.bytes = nb;
    ctx->held += nb;
    return TSP_OK;
}

void release(tsp_context* ctx, Buf& b)
{
    if (b.p) {
        if (ctx->free_fn) ctx->free_fn(b.p, b.bytes, ctx->device, ctx->alloc_user);
        else cudaFree(b.p);
    }
    ctx->held -= b.bytes;
    b = Buf{};
}

// Every device buffer of the workspace (not the pinned status words).
void release_workspace(tsp_context* ctx)
{
    Buf* all[] = {&ctx->rect, &ctx->depth, &ctx->touched, &ctx->rec, &ctx->oref, &ctx->color,
                  &ctx->moments, &ctx->vres0, &ctx->vres1, &ctx->vres2, &ctx->vres3, &ctx->tiles, &ctx->tile_off,
                  &ctx->span_sum, &ctx->queue, &ctx->gacc, &ctx->reg, &ctx->pairs, &ctx->pairs_tmp, &ctx->dstatus,
                  &ctx->stats, &ctx->st_in, &ctx->st_out, &ctx->st_tracks};
    for (Buf* b : all) release(ctx, *b);
    ctx->last_R = 0;
    ctx->last_NT = 0;
    ctx->last_fit_n = ctx->last_fit_V = -1;
    ctx->last_knn_path = nullptr;
    ctx->render_bins = false;
}


bool device_accessible(const void* p, int dev)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

tsp_status check_options(tsp_context* ctx, const tsp_options& o)
{
    const bool square = o.tile_w == 16 && o.tile_h == 16, wide = o.tile_w == 32 && o.tile_h == 8;
    if (!square && !wide) return fail(ctx, TSP_ERR_INVALID_ARG, "tiles must be 16x16 or 32x8");
    if (!(o.det_min >= 0.f) || !(o.sumw_min_view >= 0.f) || !(o.lam_min_px2 >= 0.f) ||
        !(o.sumw_min_total >= 0.f) || !(o.cov_rcond_min >= 0.f) || !std::isfinite(o.det_min) ||
        !std::isfinite(o.sumw_min_view) || !std::isfinite(o.lam_min_px2) ||
        !std::isfinite(o.sumw_min_total) || !std::isfinite(o.cov_rcond_min))
        return fail(ctx, TSP_ERR_INVALID_ARG, "thresholds must be finite and >= 0");
    if (!(o.cov_rcond_min >= 1e-12f && o.cov_rcond_min < 1.f))
        return fail(ctx, TSP_ERR_INVALID_ARG, "cov_rcond_min must lie in [1e-12, 1)");
    if (o.min_px_view < 0 || o.min_views < 0 || o.min_px_total < 0)
        return fail(ctx, TSP_ERR_INVALID_ARG, "counts must be >= 0");
    if (o.raster_variant != 0 && o.raster_variant != 1 && o.raster_variant != 2 &&
        o.raster_variant != 4 && o.raster_variant != 5)
        return fail(ctx, TSP_ERR_INVALID_ARG, "raster_variant must be 0, 1, 2, 4 or 5");
    if (!square && o.raster_variant != 0 && o.raster_variant != 5)
        return fail(ctx, TSP_ERR_INVALID_ARG, "32x8 tiles need raster_variant 0 or 5");
    if (o.pair_capacity < 0 || o.pair_capacity > INT32_MAX || o.budget_bytes < 0)
        return fail(ctx, TSP_ERR_INVALID_ARG, "bad pair_capacity or budget_bytes");
    if (o.checked != 0 && o.checked != 1) return fail(ctx, TSP_ERR_INVALID_ARG, "checked must be 0 or 1");
    return TSP_OK;
}

FitParams fit_params(const tsp_options& o)
{
    FitParams f;
    f.det_min = o.det_min;
    f.sumw_min_view = o.sumw_min_view;
    f.lam_min_px2 = o.lam_min_px2;
    f.sumw_min_total = o.sumw_min_total;
    f.cov_rcond_min = o.cov_rcond_min;
    f.min_px_view = o.min_px_view;
    f.min_views = o.min_views;
    f.min_px_total = o.min_px_total;
    return f;
}

// Validate cameras and build the per-call view description.
// Fill the kernels' view set for the frames of one launch: cameras (validated),
// tile offsets, each view's frame, Gaussian count and record base.  g_of(f)
// gives frame f's Gaussian arrays.  NT = tiles of all views, R = records.
tsp_status make_viewset(tsp_context* ctx, const tsp_frame* frames, int F, ViewSet& vs, uint32_t& NT,
                        uint64_t& R)
{
    if (F < 0 || F > TSP_MAX_FRAMES) return fail(ctx, TSP_ERR_INVALID_ARG, "num_frames must be in [0, 16]");
    if (F > 0 && !frames) return fail(ctx, TSP_ERR_INVALID_ARG, "frames is NULL");
    std::memset(&vs, 0, sizeof(vs));
    vs.tw = ctx->opt.tile_w;
    vs.th = ctx->opt.tile_h;
    uint64_t off = 0, rec = 0;
    int V = 0;
    for (int f = 0; f < F; ++f) {
        const tsp_frame& fr = frames[f];
        const int Vf = fr.num_views, n = fr.g.n;
        if (Vf < 0 || Vf > TSP_MAX_VIEWS) return fail(ctx, TSP_ERR_INVALID_ARG, "num_views must be in [0, 32]");
        if (V + Vf > TSP_MAX_BATCH_VIEWS)
            return fail(ctx, TSP_ERR_INVALID_ARG, "more than 192 views in one batch");
        if (Vf > 0 && !fr.cams) return fail(ctx, TSP_ERR_INVALID_ARG, "cams is NULL");
        if (n < 0 || n >= (int)kMaxGaussians) return fail(ctx, TSP_ERR_INVALID_ARG, "n must be in [0, 2^28)");
        vs.fview[f] = V;
        vs.fn[f] = n;
        vs.fmo[f] = (const float4*)fr.g.means_opacity;
        vs.fq[f] = (const float4*)fr.g.quats;
        vs.fs[f] = (const float4*)fr.g.scales;
        vs.nmax = std::max(vs.nmax, n);
        for (int k = 0; k < Vf; ++k, ++V) {
            const tsp_camera& c = fr.cams[k];
            const std::string where = "frame " + std::to_string(f) + " camera " + std::to_string(k);
            if (c.width < 1 || c.height < 1 || c.width > TSP_MAX_IMAGE || c.height > TSP_MAX_IMAGE)
                return fail(ctx, TSP_ERR_INVALID_ARG, where + ": size out of range");
            if (!(c.fx > 0.f) || !(c.fy > 0.f) || !std::isfinite(c.fx) || !std::isfinite(c.fy) ||
                !std::isfinite(c.cx) || !std::isfinite(c.cy))
                return fail(ctx, TSP_ERR_INVALID_ARG, where + ": bad intrinsics");
            for (int j = 0; j < 9; ++j)
                if (!std::isfinite(c.R[j])) return fail(ctx, TSP_ERR_INVALID_ARG, where + ": R not finite");
            for (int j = 0; j < 3; ++j)
                if (!std::isfinite(c.t[j])) return fail(ctx, TSP_ERR_INVALID_ARG, where + ": t not finite");
            DevCam& d = vs.cam[V];
            d.W = c.width; d.H = c.height;
            d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
            std::memcpy(d.R, c.R, sizeof(d.R));
            std::memcpy(d.t, c.t, sizeof(d.t));
            vs.tiles_x[V] = (c.width + vs.tw - 1) / vs.tw;
            vs.tiles_y[V] = (c.height + vs.th - 1) / vs.th;
            vs.toff[V] = (uint32_t)off;
            off += (uint64_t)vs.tiles_x[V] * vs.tiles_y[V];
            vs.vframe[V] = f;
            vs.vn[V] = n;
            vs.vrec[V] = rec;
            rec += (uint64_t)n;
        }
    }
    vs.V = V;
    vs.F = F;
    vs.fview[F] = V;
    vs.toff[V] = (uint32_t)off;
    if (off > 0xffffffffull) return fail(ctx, TSP_ERR_INVALID_ARG, "too many tiles");
    NT = (uint32_t)off;
    R = rec;
    return TSP_OK;
}

tsp_status check_gaussians(tsp_context* ctx, const tsp_gaussians* g, bool device)
{
    if (!g) return fail(ctx, TSP_ERR_INVALID_ARG, "g is NULL");
    if (g->n < 0 || g->n >= (int)kMaxGaussians) return fail(ctx, TSP_ERR_INVALID_ARG, "n must be in [0, 2^28)");
    if (g->n == 0) return TSP_OK;
    const void* ps[3] = {g->means_opacity, g->quats, g->scales};
    for (const void* p : ps) {
        if (!p) return fail(ctx, TSP_ERR_INVALID_ARG, "Gaussian array is NULL");
        if (!aligned(p, 16)) return fail(ctx, TSP_ERR_INVALID_ARG, "Gaussian arrays must be 16-byte aligned");
        if (device && !device_accessible(p, ctx->device))
            return fail(ctx, TSP_ERR_INVALID_ARG, "Gaussian array is not device memory of the context's device");
    }
    return TSP_OK;
}

tsp_status check_result(tsp_context* ctx, const tsp_result* out, int n, bool device)
{
    if (!out) return fail(ctx, TSP_ERR_INVALID_ARG, "out is NULL");
    if (n == 0) return TSP_OK;
    const void* ps[4] = {out->means, out->quats, out->scales, out->status};
    for (int k = 0; k < 4; ++k) {
        if (!ps[k]) return fail(ctx, TSP_ERR_INVALID_ARG, "result array is NULL");
        if (!aligned(ps[k], k < 3 ? 16 : 4)) return fail(ctx, TSP_ERR_INVALID_ARG, "result array misaligned");
        if (device && !device_accessible(ps[k], ctx->device))
            return fail(ctx, TSP_ERR_INVALID_ARG, "result array is not device memory of the context's device");
    }
    const void* opt[3] = {out->view_affine, out->view_moments, out->view_flags};
    for (const void* p : opt) {
        if (!p) continue;
        if (!device) return fail(ctx, TSP_ERR_INVALID_ARG, "optional outputs are not supported by the host call");
        if (!aligned(p, 16) && p == out->view_moments)
            return fail(ctx, TSP_ERR_INVALID_ARG, "view_moments must be 16-byte aligned");
        if (!aligned(p, 4)) return fail(ctx, TSP_ERR_INVALID_ARG, "optional output misaligned");
        if (!device_accessible(p, ctx->device))
            return fail(ctx, TSP_ERR_INVALID_ARG, "optional output is not device memory");
    }
    return TSP_OK;
}

tsp_status ensure_work(tsp_context* ctx, uint64_t R, uint32_t NT, bool render, Work& w)
{
    const size_t vn = (size_t)R;
    const size_t vn1 = vn > 0 ? vn : 1;
    tsp_status s;
    if ((s = ensure(ctx, ctx->rect, vn1 * sizeof(short4)))) return s;
    if ((s = ensure(ctx, ctx->depth, vn1 * 4))) return s;
    if ((s = ensure(ctx, ctx->touched, vn1 * 4))) return s;
    if ((s = ensure(ctx, ctx->rec, vn1 * 64))) return s;
    if (!render && (s = ensure(ctx, ctx->oref, vn1 * 4))) return s;
    if (render) {
        if ((s = ensure(ctx, ctx->color, vn1 * 16))) return s;
    } else {
        if ((s = ensure(ctx, ctx->moments, vn1 * 64))) return s;
        if ((s = ensure(ctx, ctx->vres0, vn1 * 16))) return s;
        if ((s = ensure(ctx, ctx->vres1, vn1 * 16))) return s;
        if ((s = ensure(ctx, ctx->vres2, vn1 * 8))) return s;
        if ((s = ensure(ctx, ctx->vres3, vn1 * 16))) return s;
    }
    if ((s = ensure(ctx, ctx->tiles, (size_t)2 * (NT + 1) * kCounterStride * 4))) return s;
    if ((s = ensure(ctx, ctx->tile_off, (size_t)(NT + 1) * 4))) return s;
    if ((s = ensure(ctx, ctx->span_sum, ((size_t)NT / 1024 + 2) * 8))) return s;
    if ((s = ensure(ctx, ctx->queue, 16))) return s;
    uint64_t cap = ctx->want_pairs;
    if (cap == 0) cap = ctx->opt.pair_capacity > 0 ? (uint64_t)ctx->opt.pair_capacity : (uint64_t)8 * vn;
    if (cap < (1u << 16)) cap = 1u << 16;
    if (cap > (uint64_t)INT32_MAX) cap = INT32_MAX;
    if ((s = ensure(ctx, ctx->pairs, cap * 8))) return s;
    if ((s = ensure(ctx, ctx->pairs_tmp, cap * 8))) return s;
    if ((s = ensure(ctx, ctx->dstatus, 32))) return s;
    if ((s = ensure(ctx, ctx->stats, 64))) return s;
    w.stats = (unsigned long long*)ctx->stats.p;
    w.rect = (short4*)ctx->rect.p;
    w.depth = (uint32_t*)ctx->depth.p;
    w.touched = (uint32_t*)ctx->touched.p;
    w.rec = (float4*)ctx->rec.p;
    w.oref = (uint32_t*)ctx->oref.p;
    w.color = (float4*)ctx->color.p;
    w.moments = (float4*)ctx->moments.p;
    w.vres0 = (float4*)ctx->vres0.p;
    w.vres1 = (float4*)ctx->vres1.p;
    w.vres2 = (uint2*)ctx->vres2.p;
    w.vres3 = (float4*)ctx->vres3.p;
    w.tile_count = (uint32_t*)ctx->tiles.p;
    w.tile_fill = (uint32_t*)ctx->tiles.p + (size_t)(NT + 1) * kCounterStride;
    w.tile_off = (uint32_t*)ctx->tile_off.p;
    w.span_sum = (unsigned long long*)ctx->span_sum.p;
    w.queue = (uint32_t*)ctx->queue.p;
    w.pairs = (uint64_t*)ctx->pairs.p;
    w.pairs_tmp = (uint64_t*)ctx->pairs_tmp.p;
    const uint64_t have = ctx->pairs.bytes / 8 < ctx->pairs_tmp.bytes / 8 ? ctx->pairs.bytes / 8 : ctx->pairs_tmp.bytes / 8;
    w.cap = (uint32_t)(have > (uint64_t)INT32_MAX ? INT32_MAX : have);
    w.dstatus = (uint32_t*)ctx->dstatus.p;
    w.nt = NT;
    w.checked = ctx->opt.checked ? 1u : 0u;
    return TSP_OK;
}

inline cudaError_t mark(tsp_context* ctx, int k, cudaStream_t st)
{
    return ctx->opt.stage_timing ? cudaEventRecord(ctx->ev[k], st) : cudaSuccess;
}

// a1 + a2 (count, scan) and, unless async, the wait that sizes the pair buffer.
tsp_status bin_front(tsp_context* ctx, const ViewSet& vs, const float* sh, int sh_degree, int mode,
                     uint32_t NT, Work& w, cudaStream_t st)
{
    TSP_CUDA(mark(ctx, 0, st));
    {
        StageRange r("tsp:project");
        TSP_CUDA(cudaMemsetAsync(ctx->tiles.p, 0, (size_t)2 * (NT + 1) * kCounterStride * 4, st));
        TSP_CUDA(cudaMemsetAsync(w.dstatus, 0, 32, st));
        if (ctx->opt.collect_stats) TSP_CUDA(cudaMemsetAsync(w.stats, 0, 64, st));
        TSP_CUDA(launch_preprocess(vs, sh, sh_degree, mode, w, st));
    }
    TSP_CUDA(mark(ctx, 1, st));
    {
        StageRange r("tsp:scan");
        TSP_CUDA(launch_scan(w, NT, st));
    }
    TSP_CUDA(mark(ctx, 2, st));
    if (!ctx->opt.async_pairs) {
        TSP_CUDA(cudaMemcpyAsync(ctx->h_status, w.dstatus, 16, cudaMemcpyDeviceToHost, st));
        TSP_CUDA(cudaStreamSynchronize(st));
        const uint64_t K = (uint64_t)ctx->h_status[1] | ((uint64_t)ctx->h_status[2] << 32);
        if (K > w.cap) {
            if (K > (uint64_t)INT32_MAX)
                return fail(ctx, TSP_ERR_OVERFLOW, "more than 2^31 - 1 (tile, Gaussian) pairs");
            ctx->want_pairs = K + K / 8;
            tsp_status s;
            if ((s = ensure(ctx, ctx->pairs, ctx->want_pairs * 8))) return s;
            if ((s = ensure(ctx, ctx->pairs_tmp, ctx->want_pairs * 8))) return s;
            w.pairs = (uint64_t*)ctx->pairs.p;
            w.pairs_tmp = (uint64_t*)ctx->pairs_tmp.p;
            w.cap = (uint32_t)(ctx->want_pairs > (uint64_t)INT32_MAX ? INT32_MAX : ctx->want_pairs);
            TSP_CUDA(cudaMemsetAsync(w.dstatus, 0, 4, st));
        }
    }
    {
        StageRange r("tsp:emit");
        TSP_CUDA(launch_scatter(vs, w, st));
    }
    TSP_CUDA(mark(ctx, 3, st));
    {
        StageRange r("tsp:tile_sort");
        TSP_CUDA(launch_tile_sort(w, NT, st));
    }
    TSP_CUDA(mark(ctx, 4, st));
    return TSP_OK;
}

// The whole path a1-a9 for the frames of one launch, on device buffers.  With
// ready != nullptr the tracks of views [k*group, (k+1)*group) (views of all
// frames numbered together) are still being copied and ready[k] is recorded on
// the copy stream once they have landed: the tracks-free steps (projection,
// binning, sorting) run first, then each view group's reference gather and
// raster wait for their own copy.
tsp_status fit_device(tsp_context* ctx, const tsp_frame* frames, int F, cudaStream_t st, bool check_ptrs,
                      int group = 0, const cudaEvent_t* ready = nullptr)
{
    tsp_status s;
    if (F > 0 && !frames) return fail(ctx, TSP_ERR_INVALID_ARG, "frames is NULL");
    for (int f = 0; f < F; ++f) {
        if ((s = check_gaussians(ctx, &frames[f].g, check_ptrs))) return s;
        if ((s = check_result(ctx, &frames[f].out, frames[f].g.n, check_ptrs))) return s;
    }
    ViewSet vs;
    uint32_t NT = 0;
    uint64_t R = 0;
    if ((s = make_viewset(ctx, frames, F, vs, NT, R))) return s;
    FrameOut fo{};
    for (int f = 0; f < F; ++f) {
        const tsp_frame& fr = frames[f];
        fo.means[f] = (float4*)fr.out.means;
        fo.quats[f] = (float4*)fr.out.quats;
        fo.scales[f] = (float4*)fr.out.scales;
        fo.status[f] = fr.out.status;
        fo.view_affine[f] = fr.out.view_affine;
        fo.view_flags[f] = fr.out.view_flags;
        if (fr.g.n == 0 || fr.num_views == 0) continue;
        if (!fr.tracks) return fail(ctx, TSP_ERR_INVALID_ARG, "tracks is NULL");
        for (int k = 0; k < fr.num_views; ++k) {
            const std::string where = "frame " + std::to_string(f) + " view " + std::to_string(k);
            const tsp_view_tracks& tr = fr.tracks[k];
            if (!tr.disp || !tr.vis) return fail(ctx, TSP_ERR_INVALID_ARG, where + ": track pointer is NULL");
            if (!aligned(tr.disp, 8)) return fail(ctx, TSP_ERR_INVALID_ARG, where + ": disp must be 8-byte aligned");
            if (check_ptrs && (!device_accessible(tr.disp, ctx->device) || !device_accessible(tr.vis, ctx->device)))
                return fail(ctx, TSP_ERR_INVALID_ARG, where + ": tracks are not device memory");
            vs.disp[vs.fview[f] + k] = (const float2*)tr.disp;
            vs.vis[vs.fview[f] + k] = tr.vis;
        }
    }
    Work w{};
    ctx->last_fit_n = ctx->last_fit_V = -1;
    ctx->render_bins = false;
    if ((s = ensure_work(ctx, R, NT, false, w))) return s;
    ctx->last_R = (size_t)R;
    ctx->last_NT = NT;
    if (F == 1) {
        ctx->last_fit_n = frames[0].g.n;
        ctx->last_fit_V = frames[0].num_views;
    }
    if (vs.nmax == 0) return TSP_OK;
    const FitParams fp = fit_params(ctx->opt);
    const int V = vs.V;
    ctx->timed = false;
    // the gate applies to calls on caller-owned device tracks
    w.gated = (ctx->gate_flag && !ready) ? 1u : 0u;
    if ((s = bin_front(ctx, vs, nullptr, 0, 0, NT, w, st))) return s;
    if (w.gated) {
        StageRange r("tsp:track_gate");
        TSP_CUDA(launch_track_gate(ctx->gate_flag, ctx->gate_value, ctx->gate_timeout_us, w, st));
    }
    if (group <= 0) group = V;
    {
        StageRange r("tsp:raster");
        for (int v0 = 0, k = 0; v0 < V; v0 += group, ++k) {
            const int v1 = std::min(V, v0 + group);
            if (ready) TSP_CUDA(cudaStreamWaitEvent(st, ready[k], 0));
            TSP_CUDA(launch_dref(vs, w, v0, v1, st));
            TSP_CUDA(launch_raster_accumulate(vs, w, vs.toff[v0], vs.toff[v1] - vs.toff[v0],
                                              ctx->opt.collect_stats != 0, ctx->opt.raster_variant,
                                              ctx->resident_ctas, st));
        }
    }
    TSP_CUDA(mark(ctx, 5, st));
    {
        StageRange r("tsp:view_solve");
        TSP_CUDA(launch_view_solve(vs, fp, w, fo, st));
    }
    TSP_CUDA(mark(ctx, 6, st));
    {
        StageRange r("tsp:multiview");
        TSP_CUDA(launch_multiview(vs, fp, w, fo, st));
    }
    TSP_CUDA(mark(ctx, 7, st));
    ctx->timed = ctx->opt.stage_timing != 0;
    for (int f = 0; f < F; ++f) {
        const tsp_frame& fr = frames[f];
        const size_t recs = (size_t)fr.num_views * (size_t)fr.g.n;
        if (fr.out.view_moments && recs > 0)
            TSP_CUDA(cudaMemcpyAsync(fr.out.view_moments, w.moments + 4 * vs.vrec[vs.fview[f]], recs * 64,
                                     cudaMemcpyDeviceToDevice, st));
    }
    return TSP_OK;
}

// Neighbour-grid scratch (and, with rp, the regularization arrays) for n points,
// carved from one buffer.
tsp_status ensure_reg(tsp_context* ctx, int n, int k, KnnWork& kw, RegParams* rp)
{
    const size_t C = knn_max_cells(n);
    const size_t G = kMaxGrids;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    const size_t nn = (size_t)n;
    const size_t zero_bytes = G * 8 * 4 + G * C * 4;
    const size_t o_zero = take(zero_bytes), o_gp = take(G * sizeof(GridParam)), o_st = take(16);
    const size_t o_off = take((G * C + 1) * 4), o_span = take((G * C / 1024 + 2) * 8);
    const size_t o_slot = take(G * nn * 8), o_sorted = take(G * nn * 16);
    // BVH fallback (two candidate sets)
    const size_t K = kMortonBuckets;
    const size_t bvh_zero_bytes = 2 * K * 4 + 2 * nn * 4 + 2 * 8 + 4 * 4;
    const size_t o_bzero = take(bvh_zero_bytes), o_boff = take((2 * K + 1) * 4);
    const size_t o_bspan = take((2 * K / 1024 + 2) * 8), o_bst = take(16), o_bslot = take(2 * nn * 8);
    const size_t o_keys = take(2 * nn * 8), o_ktmp = take(2 * nn * 8), o_long = take(2 * K * 4 + 4);
    const size_t o_nodes = take(2 * nn * 64), o_par = take(2 * 2 * nn * 4);
    size_t o_mask = 0, o_vec = 0, o_nbr = 0;
    if (rp) {
        o_mask = take(nn);
        o_vec = take(nn * 16 * 6);
        o_nbr = take(nn * (size_t)k * 4 * 2);
    }
    tsp_status s;
    if ((s = ensure(ctx, ctx->reg, off))) return s;
    if (!ctx->dstatus.p) {
        if ((s = ensure(ctx, ctx->dstatus, 32))) return s;
        TSP_CUDA(cudaMemset(ctx->dstatus.p, 0, 16));
    }
    kw.err = (uint32_t*)ctx->dstatus.p;
    char* b = (char*)ctx->reg.p;
    kw.zero = (uint32_t*)(b + o_zero);
    kw.zero_bytes = zero_bytes;
    kw.acc = kw.zero;
    kw.count = kw.zero + G * 8;
    kw.gp = (GridParam*)(b + o_gp);
    kw.status = (uint32_t*)(b + o_st);
    kw.cell_off = (uint32_t*)(b + o_off);
    kw.span_sum = (unsigned long long*)(b + o_span);
    kw.slot = (uint2*)(b + o_slot);
    kw.sorted = (float4*)(b + o_sorted);
    kw.bvh_zero = (uint32_t*)(b + o_bzero);
    kw.bvh_zero_bytes = bvh_zero_bytes;
    kw.bcount = kw.bvh_zero;
    kw.flag = kw.bcount + 2 * K;
    kw.skew = (unsigned long long*)(kw.flag + 2 * nn);                  // even word offset: 8-byte aligned
    kw.use_bvh = (uint32_t*)(kw.skew + 2);
    ctx->last_knn_path = kw.use_bvh;
    kw.boff = (uint32_t*)(b + o_boff);
    kw.bspan = (unsigned long long*)(b + o_bspan);
    kw.bstatus = (uint32_t*)(b + o_bst);
    kw.bslot = (uint2*)(b + o_bslot);
    kw.keys = (uint64_t*)(b + o_keys);
    kw.keys_tmp = (uint64_t*)(b + o_ktmp);
    kw.long_list = (uint32_t*)(b + o_long);
    kw.long_count = kw.long_list + 2 * K;
    kw.nodes = (float4*)(b + o_nodes);
    kw.parent = (int32_t*)(b + o_par);
    if (rp) {
        rp->mask = (uint8_t*)(b + o_mask);
        float4* v = (float4*)(b + o_vec);
        rp->dpos = v;
        rp->dscale = v + nn;
        rp->drot = v + 2 * nn;
        rp->fpos = v + 3 * nn;
        rp->fscale = v + 4 * nn;
        rp->frot = v + 5 * nn;
        if (!rp->nbr_pos) rp->nbr_pos = (int32_t*)(b + o_nbr);
        if (!rp->nbr_cov) rp->nbr_cov = (int32_t*)(b + o_nbr) + nn * (size_t)k;
    }
    return TSP_OK;
}

tsp_status check_device_array(tsp_context* ctx, const void* p, size_t align, const char* what, bool optional)
{
    if (!p) return optional ? TSP_OK : fail(ctx, TSP_ERR_INVALID_ARG, std::string(what) + " is NULL");
    if (!aligned(p, align)) return fail(ctx, TSP_ERR_INVALID_ARG, std::string(what) + " misaligned");
    if (!device_accessible(p, ctx->device))
        return fail(ctx, TSP_ERR_INVALID_ARG, std::string(what) + " is not device memory of the context's device");
    return TSP_OK;
}

void note_render_bins(tsp_context* ctx, const tsp_gaussians* g, const float* sh, int sh_degree,
                      const tsp_camera* cams, int V)
{
    ctx->render_bins = true;
    ctx->render_ptrs[0] = g->means_opacity;
    ctx->render_ptrs[1] = g->quats;
    ctx->render_ptrs[2] = g->scales;
    ctx->render_ptrs[3] = sh;
    ctx->render_n = g->n;
    ctx->render_deg = sh_degree;
    ctx->render_cams.assign(cams, cams + V);
}

bool same_render_bins(const tsp_context* ctx, const tsp_gaussians* g, const float* sh, int sh_degree,
                      const tsp_camera* cams, int V)
{
    if (!ctx->render_bins || ctx->render_n != g->n || ctx->render_deg != sh_degree ||
        (int)ctx->render_cams.size() != V)
        return false;
    if (ctx->render_ptrs[0] != g->means_opacity || ctx->render_ptrs[1] != g->quats ||
        ctx->render_ptrs[2] != g->scales || ctx->render_ptrs[3] != sh)
        return false;
    return V == 0 || std::memcmp(ctx->render_cams.data(), cams, sizeof(tsp_camera) * (size_t)V) == 0;
}

// One frame as a batch of one.
tsp_status single_frame(tsp_context* ctx, const tsp_gaussians* g, const tsp_camera* cams, int V,
                        const tsp_view_tracks* tracks, const tsp_result* out, tsp_frame& fr)
{
    if (!g) return fail(ctx, TSP_ERR_INVALID_ARG, "g is NULL");
    if (!out) return fail(ctx, TSP_ERR_INVALID_ARG, "out is NULL");
    fr.g = *g;
    fr.cams = cams;
    fr.num_views = V;
    fr.tracks = tracks;
    fr.out = *out;
    return TSP_OK;
}

}  // namespace

extern "C" {

int tsp_version(void) { return TSP_VERSION; }

const char* tsp_status_string(tsp_status s)
{
    switch (s) {
    case TSP_OK: return "ok";
    case TSP_ERR_INVALID_ARG: return "invalid argument";
    case TSP_ERR_OOM: return "out of device memory";
    case TSP_ERR_CUDA: return "CUDA error";
    case TSP_ERR_TIMEOUT: return "timed out";
    case TSP_ERR_BUDGET: return "workspace budget exceeded";
    case TSP_ERR_OVERFLOW: return "pair buffer overflow";
    }
    return "unknown status";
}

const char* tsp_last_error(const tsp_context* ctx)
{
    if (!ctx) return "no context";
    return ctx->err.c_str();
}

tsp_status tsp_default_options(tsp_options* o)
{
    if (!o) return TSP_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    o->tile_w = kTile;
    o->tile_h = kTile;
    o->det_min = 1e-12f;
    o->sumw_min_view = 1e-3f;
    o->min_px_view = 2;
    o->lam_min_px2 = 1e-4f;
    o->min_views = 2;
    o->sumw_min_total = 1e-3f;
    o->min_px_total = 3;
    o->cov_rcond_min = 1e-6f;
    return TSP_OK;
}

tsp_status tsp_create(int device, const tsp_options* opt, tsp_context** out)
{
    if (!out) return TSP_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return device < 0 ? TSP_ERR_INVALID_ARG : TSP_ERR_CUDA;
    }
    tsp_context* ctx = new tsp_context();
    ctx->device = device;
    if (opt) ctx->opt = *opt;
    else tsp_default_options(&ctx->opt);
    tsp_status s = check_options(ctx, ctx->opt);
    if (s) { delete ctx; return s; }
    DeviceGuard dg(device);
    if (cudaMallocHost(&ctx->h_status, 32) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return TSP_ERR_CUDA;
    }
    if (raster_prepare() != cudaSuccess || backward_prepare() != cudaSuccess) {
        cudaGetLastError();
        tsp_destroy(ctx);
        return TSP_ERR_CUDA;
    }
    ctx->resident_ctas = raster_resident_ctas(device);
    for (cudaEvent_t& e : ctx->ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            tsp_destroy(ctx);
            return TSP_ERR_CUDA;
        }
    *out = ctx;
    return TSP_OK;
}

tsp_status tsp_destroy(tsp_context* ctx)
{
    if (!ctx) return TSP_OK;
    DeviceGuard dg(ctx->device);
    cudaDeviceSynchronize();
    release_workspace(ctx);
    for (cudaEvent_t e : ctx->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->group_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    delete ctx;
    return TSP_OK;
}

tsp_status tsp_set_allocator(tsp_context* ctx, tsp_alloc_fn alloc, tsp_free_fn release_fn, void* user)
{
    if (!ctx || (alloc == nullptr) != (release_fn == nullptr)) return TSP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    TSP_CUDA(cudaDeviceSynchronize());
    release_workspace(ctx);
    ctx->alloc_fn = alloc;
    ctx->free_fn = release_fn;
    ctx->alloc_user = user;
    return TSP_OK;
}

tsp_status tsp_set_track_gate(tsp_context* ctx, const uint32_t* flag, uint32_t value, int64_t timeout_us)
{
    if (!ctx) return TSP_ERR_INVALID_ARG;
    if (!flag) {
        ctx->gate_flag = nullptr;
        return TSP_OK;
    }
    if (!aligned(flag, 4) || timeout_us < 1 || timeout_us > 10000000)
        return fail(ctx, TSP_ERR_INVALID_ARG, "the gate flag must be 4-byte aligned and the limit in [1, 1e7] us");
    DeviceGuard dg(ctx->device);
    if (!device_accessible(flag, ctx->device))
        return fail(ctx, TSP_ERR_INVALID_ARG, "the gate flag is not device memory");
    ctx->gate_flag = flag;
    ctx->gate_value = value;
    ctx->gate_timeout_us = timeout_us;
    return TSP_OK;
}

tsp_status tsp_set_budget(tsp_context* ctx, int64_t budget_bytes)
{
    if (!ctx || budget_bytes < 0) return TSP_ERR_INVALID_ARG;
    ctx->opt.budget_bytes = budget_bytes;
    return TSP_OK;
}

tsp_status tsp_fit_motion(tsp_context* ctx, const tsp_gaussians* g, const tsp_camera* cams, int num_views,
                          const tsp_view_tracks* tracks, const tsp_result* out, void* stream)
{
    if (!ctx) return TSP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    tsp_frame fr;
    tsp_status s;
    if ((s = single_frame(ctx, g, cams, num_views, tracks, out, fr))) return s;
    return fit_device(ctx, &fr, 1, (cudaStream_t)stream, true);
}

tsp_status tsp_fit_motion_batch(tsp_context* ctx, const tsp_frame* frames, int num_frames, void* stream)
{
    if (!ctx) return TSP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    return fit_device(ctx, frames, num_frames, (cudaStream_t)stream, true);
}

tsp_status tsp_fit_motion_host(tsp_context* ctx, const tsp_gaussians* g, const tsp_camera* cams,
                               int num_views, const tsp_view_tracks* tracks, const tsp_result* out,
                               void* stream)
{
    if (!ctx) return TSP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    tsp_status s;
    if ((s = check_gaussians(ctx, g, false))) return s;
    if ((s = check_result(ctx, out, g->n, false))) return s;
    {
        tsp_frame probe;
        if ((s = single_frame(ctx, g, cams, num_views, tracks, out, probe))) return s;
        ViewSet vs;
        uint32_t NT = 0;
        uint64_t R = 0;
        if ((s = make_viewset(ctx, &probe, 1, vs, NT, R))) return s;   // validates the cameras
    }
    const int n = g->n, V = num_views;
    if (n > 0 && V > 0 && !tracks) return fail(ctx, TSP_ERR_INVALID_ARG, "tracks is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t gb = (size_t)n * 16;
    if ((s = ensure(ctx, ctx->st_in, 3 * align_up(gb) + kAlign))) return s;
    if ((s = ensure(ctx, ctx->st_out, 3 * align_up(gb) + align_up((size_t)n * 4) + kAlign))) return s;
    std::vector<size_t> toff(V + 1, 0);
    for (int v = 0; v < V; ++v) {
        const size_t px = (size_t)cams[v].width * cams[v].height;
        toff[v + 1] = toff[v] + align_up(px * 8) + align_up(px);
    }
    if ((s = ensure(ctx, ctx->st_tracks, toff[V] + kAlign))) return s;
    char* in = (char*)ctx->st_in.p;
    char* ob = (char*)ctx->st_out.p;
    char* tb = (char*)ctx->st_tracks.p;
    tsp_gaussians dg_{n, (const float*)in, (const float*)(in + align_up(gb)), (const float*)(in + 2 * align_up(gb))};
    tsp_result dr{(float*)ob, (float*)(ob + align_up(gb)), (float*)(ob + 2 * align_up(gb)),
                  (uint32_t*)(ob + 3 * align_up(gb)), nullptr, nullptr, nullptr};
    std::vector<tsp_view_tracks> dt(V > 0 ? V : 1);
    // one view per copy group: each view's raster starts as soon as its tracks
    // have landed, so only the last view's raster and the solves follow the last
    // copy (three-view groups: 5.9-6.0 ms per capture frame end to end; one view:
    // 5.76 ms, the copy alone 5.2 ms)
    const int group = 1;
    if (n > 0 && V > 0) {
        if (!ctx->copy_stream &&
            cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            ctx->copy_stream = nullptr;
            return fail(ctx, TSP_ERR_CUDA, "cannot create the copy stream");
        }
        for (int k = 0; k * group < V; ++k)
            if (!ctx->group_ev[k] && cudaEventCreateWithFlags(&ctx->group_ev[k], cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                ctx->group_ev[k] = nullptr;
                return fail(ctx, TSP_ERR_CUDA, "cannot create a copy event");
            }
        for (int v = 0; v < V; ++v)
            if (!tracks[v].disp || !tracks[v].vis)
                return fail(ctx, TSP_ERR_INVALID_ARG, "view " + std::to_string(v) + ": track pointer is NULL");
    }
    if (n > 0) {
        TSP_CUDA(cudaMemcpyAsync((void*)dg_.means_opacity, g->means_opacity, gb, cudaMemcpyHostToDevice, st));
        TSP_CUDA(cudaMemcpyAsync((void*)dg_.quats, g->quats, gb, cudaMemcpyHostToDevice, st));
        TSP_CUDA(cudaMemcpyAsync((void*)dg_.scales, g->scales, gb, cudaMemcpyHostToDevice, st));
        for (int v = 0; v < V; ++v) {
            const size_t px = (size_t)cams[v].width * cams[v].height;
            dt[v].disp = (const float*)(tb + toff[v]);
            dt[v].vis = (const uint8_t*)(tb + toff[v] + align_up(px * 8));
            TSP_CUDA(cudaMemcpyAsync((void*)dt[v].disp, tracks[v].disp, px * 8, cudaMemcpyHostToDevice,
                                     ctx->copy_stream));
            TSP_CUDA(cudaMemcpyAsync((void*)dt[v].vis, tracks[v].vis, px, cudaMemcpyHostToDevice, ctx->copy_stream));
            if ((v + 1) % group == 0 || v + 1 == V)
                TSP_CUDA(cudaEventRecord(ctx->group_ev[v / group], ctx->copy_stream));
        }
    }
    tsp_frame dfr{dg_, cams, V, dt.data(), dr};
    if ((s = fit_device(ctx, &dfr, 1, st, false, group, n > 0 && V > 0 ? ctx->group_ev : nullptr))) {
        // the caller may release its host buffers once we return: finish reading them
        if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
        return s;
    }
    if (n > 0) {
        TSP_CUDA(cudaMemcpyAsync(out->means, dr.means, gb, cudaMemcpyDeviceToHost, st));
        TSP_CUDA(cudaMemcpyAsync(out->quats, dr.quats, gb, cudaMemcpyDeviceToHost, st));
        TSP_CUDA(cudaMemcpyAsync(out->scales, dr.scales, gb, cudaMemcpyDeviceToHost, st));
        TSP_CUDA(cudaMemcpyAsync(out->status, dr.status, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
    }
    return tsp_sync(ctx, stream, -1);
}

tsp_status tsp_render(tsp_context* ctx, const tsp_gaussians* g, const float* sh, int sh_degree,
                      const tsp_camera* cams, int num_views, float* const* rgb, float* const* final_T,
                      void* stream)
{
    if (!ctx) return TSP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    tsp_status s;
    if ((s = check_gaussians(ctx, g, true))) return s;
    if (sh_degree < 0 || sh_degree > 3) return fail(ctx, TSP_ERR_INVALID_ARG, "sh_degree must be 0..3");
    const int n = g->n, V = num_views;
    if (n > 0 && (!sh || !device_accessible(sh, ctx->device)))
        return fail(ctx, TSP_ERR_INVALID_ARG, "sh must be device memory");
    ViewSet vs;
    uint32_t NT = 0;
    uint64_t R = 0;
    tsp_frame fr{};
    fr.g = *g;
    fr.cams = cams;
    fr.num_views = V;
    if ((s = make_viewset(ctx, &fr, 1, vs, NT, R))) return s;
    if (V > 0 && (!rgb || !final_T)) return fail(ctx, TSP_ERR_INVALID_ARG, "rgb / final_T is NULL");
    for (int v = 0; v < V; ++v) {
        if (!rgb[v] || !final_T[v] || !aligned(rgb[v], 4) || !aligned(final_T[v], 4))
            return fail(ctx, TSP_ERR_INVALID_ARG, "view " + std::to_string(v) + ": bad output image");
        if (!device_accessible(rgb[v], ctx->device) || !device_accessible(final_T[v], ctx->device))
            return fail(ctx, TSP_ERR_INVALID_ARG, "view " + std::to_string(v) + ": output is not device memory");
    }
    Work w{};
    if ((s = ensure_work(ctx, R, NT, true, w))) return s;
    ctx->last_R = (size_t)R;
    ctx->last_NT = NT;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->timed = false;
    ctx->render_bins = false;
    if ((s = bin_front(ctx, vs, sh, sh_degree, 1, NT, w, st))) return s;
    note_render_bins(ctx, g, sh, sh_degree, cams, V);
    TSP_CUDA(launch_raster_render(vs, w, NT, rgb, final_T, st));
    TSP_CUDA(mark(ctx, 5, st));
    TSP_CUDA(mark(ctx, 6, st));
    TSP_CUDA(mark(ctx, 7, st));
    ctx->timed = ctx->opt.stage_timing != 0;
    return TSP_OK;
}

tsp_status tsp_render_backward(tsp_context* ctx, const tsp_gaussians* g, const float* sh, int sh_degree,
                               const tsp_camera* cams, int num_views, const float* const* rgb,
                               const float* const* grad_rgb, const tsp_render_grads* out, void* stream)
{
    if (!ctx) return TSP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    tsp_status s;
    if ((s = check_gaussians(ctx, g, true))) return s;
    if (sh_degree < 0 || sh_degree > 3) return fail(ctx, TSP_ERR_INVALID_ARG, "sh_degree must be 0..3");
    const int n = g->n, V = num_views;
    if (n > 0 && (!sh || !device_accessible(sh, ctx->device)))
        return fail(ctx, TSP_ERR_INVALID_ARG, "sh must be device memory");
    if (!out) return fail(ctx, TSP_ERR_INVALID_ARG, "out is NULL");
    if (n > 0) {
        const void* ps[4] = {out->means, out->scales, out->quats, out->sh};
        for (int k = 0; k < 4; ++k)
            if (!ps[k] || !aligned(ps[k], k < 3 ? 16 : 4) || !device_accessible(ps[k], ctx->device))
                return fail(ctx, TSP_ERR_INVALID_ARG, "gradient output is not aligned device memory");
    }
    ViewSet vs;
    uint32_t NT = 0;
    uint64_t R = 0;
    tsp_frame fr{};
    fr.g = *g;
    fr.cams = cams;
    fr.num_views = V;
    if ((s = make_viewset(ctx, &fr, 1, vs, NT, R))) return s;
    if (V > 0 && (!rgb || !grad_rgb)) return fail(ctx, TSP_ERR_INVALID_ARG, "rgb / grad_rgb is NULL");
    RenderGrad rg{};
    for (int v = 0; v < V; ++v) {
        if (!rgb[v] || !grad_rgb[v] || !aligned(rgb[v], 4) || !aligned(grad_rgb[v], 4) ||
            !device_accessible(rgb[v], ctx->device) || !device_accessible(grad_rgb[v], ctx->device))
            return fail(ctx, TSP_ERR_INVALID_ARG, "view " + std::to_string(v) + ": bad colour or gradient image");
        rg.rgb[v] = rgb[v];
        rg.grad[v] = grad_rgb[v];
    }
    Work w{};
    if ((s = ensure_work(ctx, R, NT, true, w))) return s;
    if ((s = ensure(ctx, ctx->gacc, (size_t)std::max<uint64_t>(R, 1) * kGradStride * 4))) return s;
    ctx->last_R = (size_t)R;
    ctx->last_NT = NT;
    rg.acc = (float*)ctx->gacc.p;
    rg.g_means = (float4*)out->means;
    rg.g_scales = (float4*)out->scales;
    rg.g_quats = (float4*)out->quats;
    rg.g_sh = out->sh;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->timed = false;
    if (n == 0) return TSP_OK;
    // the tile lists of the render this call differentiates: still in the
    // workspace when the previous binning was that render, else built again
    if (!same_render_bins(ctx, g, sh, sh_degree, cams, V)) {
        ctx->render_bins = false;
        if ((s = bin_front(ctx, vs, sh, sh_degree, 1, NT, w, st))) return s;
        note_render_bins(ctx, g, sh, sh_degree, cams, V);
    }
    TSP_CUDA(launch_render_backward(vs, w, NT, rg, sh, sh_degree, (size_t)R, st));
    return TSP_OK;
}

tsp_status tsp_sync(tsp_context* ctx, void* stream, int timeout_ms)
{
    if (!ctx) return TSP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (timeout_ms < 0) {
        TSP_CUDA(cudaStreamSynchronize(st));
    } else {
        const auto t0 = std::chrono::steady_clock::now();
        for (;;) {
            const cudaError_t e = cudaStreamQuery(st);
            if (e == cudaSuccess) break;
            if (e != cudaErrorNotReady) return cuda_fail(ctx, e, "cudaStreamQuery");
            const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                                std::chrono::steady_clock::now() - t0).count();
            if (ms >= timeout_ms) return fail(ctx, TSP_ERR_TIMEOUT, "stream still busy");
            std::this_thread::sleep_for(std::chrono::microseconds(100));
        }
    }
    if (!ctx->dstatus.p) return TSP_OK;
    TSP_CUDA(cudaMemcpyAsync(ctx->h_status, ctx->dstatus.p, 32, cudaMemcpyDeviceToHost, st));
    TSP_CUDA(cudaStreamSynchronize(st));
    if (ctx->h_status[0] & kStatusChecked) {
        const uint32_t site = ctx->h_status[4], count = ctx->h_status[5];
        TSP_CUDA(cudaMemsetAsync(ctx->dstatus.p, 0, 32, st));
        TSP_CUDA(cudaStreamSynchronize(st));
        return fail(ctx, TSP_ERR_CUDA, std::string("checked mode: an index left its buffer at ") +
                                           check_site_name(site) + " (site " + std::to_string(site) + ", " +
                                           std::to_string(count) + " times); results are invalid");
    }
    if (ctx->h_status[0] & kStatusGate) {
        TSP_CUDA(cudaMemsetAsync(ctx->dstatus.p, 0, 4, st));
        TSP_CUDA(cudaStreamSynchronize(st));
        return fail(ctx, TSP_ERR_TIMEOUT, "the track gate's wait ran out: the flag never reached its value; "
                                          "nothing was computed from the tracks and no fitted output written");
    }
    if (ctx->h_status[0] & kStatusInternal) {
        TSP_CUDA(cudaMemsetAsync(ctx->dstatus.p, 0, 4, st));
        TSP_CUDA(cudaStreamSynchronize(st));
        return fail(ctx, TSP_ERR_CUDA, "a bounded device loop gave up (neighbour search); results are invalid");
    }
    if (ctx->h_status[0] & kStatusOverflow) {
        const uint64_t K = (uint64_t)ctx->h_status[1] | ((uint64_t)ctx->h_status[2] << 32);
        ctx->want_pairs = K + K / 4;
        TSP_CUDA(cudaMemsetAsync(ctx->dstatus.p, 0, 4, st));
        TSP_CUDA(cudaStreamSynchronize(st));
        return fail(ctx, TSP_ERR_OVERFLOW, "pair buffer overflow: " + std::to_string(K) + " pairs");
    }
    return TSP_OK;
}

tsp_status tsp_inspect(tsp_context* ctx, int which, void* dst, size_t bytes, size_t* size_out)
{
    if (!ctx) return TSP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    const size_t vn = ctx->last_R;
    const void* src = nullptr;
    size_t size = 0;
    int64_t counts[4] = {0, 0, 0, 0};
    if (ctx->dstatus.p) {
        TSP_CUDA(cudaDeviceSynchronize());
        uint32_t h[4];
        TSP_CUDA(cudaMemcpy(h, ctx->dstatus.p, 16, cudaMemcpyDeviceToHost));
        counts[0] = (int64_t)((uint64_t)h[1] | ((uint64_t)h[2] << 32));
        counts[3] = h[0] & kStatusOverflow;
    }
    counts[1] = ctx->last_NT;
    counts[2] = (int64_t)(ctx->pairs.bytes / 8 < ctx->pairs_tmp.bytes / 8 ? ctx->pairs.bytes / 8 : ctx->pairs_tmp.bytes / 8);
    switch (which) {
    case TSP_I_COUNTS: size = sizeof(counts); break;
    case TSP_I_RECT: src = ctx->rect.p; size = vn * 8; break;
    case TSP_I_DEPTH: src = ctx->depth.p; size = vn * 4; break;
    case TSP_I_TILES_TOUCHED: src = ctx->touched.p; size = vn * 4; break;
    case TSP_I_TILE_OFFSETS: src = ctx->tile_off.p; size = ((size_t)ctx->last_NT + 1) * 4; break;
    case TSP_I_PAIRS: {
        // the lists as (depth bits << 32 | Gaussian index): the walks' block masks
        // are dropped from the stored keys
        const int64_t K = counts[0] < counts[2] ? counts[0] : counts[2];
        size = (size_t)K * 8;
        if (size_out) *size_out = size;
        if (!dst) return TSP_OK;
        const size_t nk = (bytes < size ? bytes : size) / 8;
        std::vector<uint64_t> keys(nk);
        if (nk) TSP_CUDA(cudaMemcpy(keys.data(), ctx->pairs.p, nk * 8, cudaMemcpyDeviceToHost));
        for (uint64_t& k : keys) k = (k & 0xffffffff00000000ull) | ((k & 0xffffffffull) >> 4);
        std::memcpy(dst, keys.data(), nk * 8);
        return TSP_OK;
    }
    case TSP_I_MOMENTS: src = ctx->moments.p; size = vn * 64; break;
    case TSP_I_STATS: src = ctx->stats.p; size = ctx->stats.p ? 64 : 0; break;
    case TSP_I_KNN_PATH: src = ctx->last_knn_path; size = ctx->last_knn_path ? 8 : 0; break;
    case TSP_I_VIEW_MEANS: src = ctx->vres0.p; size = vn * 16; break;
    case TSP_I_VIEW_COV: {
        // two planes (vres1, vres3) interleaved per (view, Gaussian) on the host
        size = vn * 32;
        if (size_out) *size_out = size;
        if (!dst) return TSP_OK;
        std::vector<float4> a(vn), b(vn);
        if (vn) {
            TSP_CUDA(cudaMemcpy(a.data(), ctx->vres1.p, vn * 16, cudaMemcpyDeviceToHost));
            TSP_CUDA(cudaMemcpy(b.data(), ctx->vres3.p, vn * 16, cudaMemcpyDeviceToHost));
        }
        std::vector<float4> ab(2 * vn);
        for (size_t i = 0; i < vn; ++i) { ab[2 * i] = a[i]; ab[2 * i + 1] = b[i]; }
        std::memcpy(dst, ab.data(), bytes < size ? bytes : size);
        return TSP_OK;
    }
    default: return fail(ctx, TSP_ERR_INVALID_ARG, "unknown intermediate");
    }
    if (size_out) *size_out = size;
    if (!dst) return TSP_OK;
    const size_t nb = bytes < size ? bytes : size;
    if (which == TSP_I_COUNTS) {
        std::memcpy(dst, counts, nb);
        return TSP_OK;
    }
    if (nb > 0 && !src) return fail(ctx, TSP_ERR_INVALID_ARG, "intermediate not available");
    if (nb > 0) TSP_CUDA(cudaMemcpy(dst, src, nb, cudaMemcpyDeviceToHost));
    return TSP_OK;
}

tsp_status tsp_stage_times(tsp_context* ctx, float* ms, int max_n, int* count)
{
    if (!ctx || (!ms && max_n > 0)) return TSP_ERR_INVALID_ARG;
    if (count) *count = 7;
    if (!ctx->timed) return fail(ctx, TSP_ERR_INVALID_ARG, "no call with stage_timing = 1 yet");
    DeviceGuard dg(ctx->device);
    TSP_CUDA(cudaEventSynchronize(ctx->ev[7]));
    for (int k = 0; k < 7 && k < max_n; ++k) TSP_CUDA(cudaEventElapsedTime(&ms[k], ctx->ev[k], ctx->ev[k + 1]));
    return TSP_OK;
}

tsp_status tsp_autotune(tsp_context* ctx, const tsp_frame* frames, int num_frames, int repeats, void* stream,
                        int* chosen, float* fit_ms)
{
    if (!ctx || repeats < 1 || repeats > 100) return TSP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    const tsp_options saved = ctx->opt;
    cudaStream_t st = (cudaStream_t)stream;
    ctx->opt.stage_timing = 1;
    ctx->opt.collect_stats = 0;
    ctx->opt.async_pairs = 0;                 // each tile shape sizes its own pair buffer
    int best_c = -1;
    float best = 3.0e38f;
    tsp_status s = TSP_OK;
    for (int c = 0; c < kTuneCandidates && s == TSP_OK; ++c) {
        ctx->opt.tile_w = kTuneTable[c][0];
        ctx->opt.tile_h = kTuneTable[c][1];
        ctx->opt.raster_variant = kTuneTable[c][2];
        std::vector<float> t;
        for (int r = 0; r <= repeats && s == TSP_OK; ++r) {        // the first run is a warm-up
            if ((s = fit_device(ctx, frames, num_frames, st, true))) break;
            if ((s = tsp_sync(ctx, stream, -1))) break;
            if (r == 0 || !ctx->timed) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[7]) != cudaSuccess) {
                cudaGetLastError();
                s = fail(ctx, TSP_ERR_CUDA, "cudaEventElapsedTime");
                break;
            }
            t.push_back(ms);
        }
        if (s != TSP_OK || t.empty()) break;
        std::sort(t.begin(), t.end());
        const float med = t[t.size() / 2];
        if (fit_ms) fit_ms[c] = med;
        if (med < best) { best = med; best_c = c; }
    }
    ctx->opt = saved;
    if (s != TSP_OK) return s;
    if (best_c >= 0) {
        ctx->opt.tile_w = kTuneTable[best_c][0];
        ctx->opt.tile_h = kTuneTable[best_c][1];
        ctx->opt.raster_variant = kTuneTable[best_c][2];
    }
    if (chosen) *chosen = best_c;
    return TSP_OK;
}

// Cache key of a tuning call: bit length of the total Gaussian count, total
// views, the largest view's pixel count.
struct TuneKey {
    long long bits, views, pixels;
};

tsp_status tune_key(const tsp_frame* frames, int num_frames, TuneKey& k)
{
    if (!frames || num_frames < 1 || num_frames > TSP_MAX_FRAMES) return TSP_ERR_INVALID_ARG;
    long long n = 0;
    k = TuneKey{0, 0, 0};
    for (int f = 0; f < num_frames; ++f) {
        const tsp_frame& fr = frames[f];
        if (fr.g.n < 0 || fr.num_views < 0 || fr.num_views > TSP_MAX_VIEWS || (fr.num_views > 0 && !fr.cams))
            return TSP_ERR_INVALID_ARG;
        n += fr.g.n;
        k.views += fr.num_views;
        for (int v = 0; v < fr.num_views; ++v)
            k.pixels = std::max(k.pixels, (long long)fr.cams[v].width * (long long)fr.cams[v].height);
    }
    while (n > 0) { ++k.bits; n >>= 1; }
    return TSP_OK;
}

tsp_status tsp_autotune_cached(tsp_context* ctx, const tsp_frame* frames, int num_frames, int repeats,
                               void* stream, const char* cache_path, int* chosen, float* fit_ms,
                               int* from_cache)
{
    if (from_cache) *from_cache = 0;
    if (!cache_path) return tsp_autotune(ctx, frames, num_frames, repeats, stream, chosen, fit_ms);
    if (!ctx || repeats < 1 || repeats > 100) return TSP_ERR_INVALID_ARG;
    TuneKey key;
    if (tune_key(frames, num_frames, key) != TSP_OK) return fail(ctx, TSP_ERR_INVALID_ARG, "autotune: bad frames");
    // the last line of this key in the file, if any
    int hit = -1;
    float hit_ms = -1.f;
    if (FILE* f = std::fopen(cache_path, "r")) {
        char line[256];
        while (std::fgets(line, sizeof line, f)) {
            long long b, v, p;
            int c;
            float ms;
            char tag[32];
            if (std::sscanf(line, "%31s %lld %lld %lld %d %f", tag, &b, &v, &p, &c, &ms) == 6 &&
                std::strcmp(tag, "tsp-autotune-v1") == 0 && b == key.bits && v == key.views && p == key.pixels &&
                c >= 0 && c < kTuneCandidates) {
                hit = c;
                hit_ms = ms;
            }
        }
        std::fclose(f);
    }
    if (hit >= 0) {
        ctx->opt.tile_w = kTuneTable[hit][0];
        ctx->opt.tile_h = kTuneTable[hit][1];
        ctx->opt.raster_variant = kTuneTable[hit][2];
        if (chosen) *chosen = hit;
        if (fit_ms)
            for (int c = 0; c < kTuneCandidates; ++c) fit_ms[c] = c == hit ? hit_ms : -1.f;
        if (from_cache) *from_cache = 1;
        return TSP_OK;
    }
    FILE* out = std::fopen(cache_path, "a");
    if (!out) return fail(ctx, TSP_ERR_INVALID_ARG, std::string("autotune: cannot append to ") + cache_path);
    int c = -1;
    float ms[kTuneCandidates];
    const tsp_status s = tsp_autotune(ctx, frames, num_frames, repeats, stream, &c, ms);
    if (s == TSP_OK && c >= 0)
        std::fprintf(out, "tsp-autotune-v1 %lld %lld %lld %d %.4f\n", key.bits, key.views, key.pixels, c, ms[c]);
    std::fclose(out);
    if (s != TSP_OK) return s;
    if (chosen) *chosen = c;
    if (fit_ms) std::memcpy(fit_ms, ms, sizeof ms);
    return TSP_OK;
}

tsp_status tsp_default_reg_options(tsp_reg_options* o)
{
    if (!o) return TSP_ERR_INVALID_ARG;
    o->k = 8;
    o->static_min_px = 9.0f;
    o->static_frac = 0.9f;
    o->static_min_views = 2;
    return TSP_OK;
}

tsp_status tsp_regularize(tsp_context* ctx, const tsp_gaussians* before, const tsp_result* fitted,
                          const float* view_moments, int num_views, const tsp_reg_options* opt,
                          const tsp_reg_result* out, void* stream)
{
    if (!ctx) return TSP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    tsp_reg_options o;
    if (opt) o = *opt;
    else tsp_default_reg_options(&o);
    if (o.k < 1 || o.k > TSP_REG_MAX_K) return fail(ctx, TSP_ERR_INVALID_ARG, "k must be in [1, TSP_REG_MAX_K]");
    if (!(o.static_min_px >= 0.0f && o.static_min_px < 1e30f))
        return fail(ctx, TSP_ERR_INVALID_ARG, "static_min_px must be finite and >= 0");
    if (!(o.static_frac >= 0.0f && o.static_frac <= 1.0f))
        return fail(ctx, TSP_ERR_INVALID_ARG, "static_frac must be in [0, 1]");
    if (o.static_min_views < 1) return fail(ctx, TSP_ERR_INVALID_ARG, "static_min_views must be >= 1");
    if (num_views < 0 || num_views > TSP_MAX_VIEWS) return fail(ctx, TSP_ERR_INVALID_ARG, "num_views out of range");
    tsp_status s;
    if ((s = check_gaussians(ctx, before, true))) return s;
    if (!fitted || !out) return fail(ctx, TSP_ERR_INVALID_ARG, "fitted or out is NULL");
    const int n = before->n;
    if (n == 0) return TSP_OK;
    if ((s = check_device_array(ctx, fitted->means, 16, "fitted means", false))) return s;
    if ((s = check_device_array(ctx, fitted->quats, 16, "fitted quats", false))) return s;
    if ((s = check_device_array(ctx, fitted->scales, 16, "fitted scales", false))) return s;
    if ((s = check_device_array(ctx, fitted->status, 4, "fitted status", false))) return s;
    if ((s = check_device_array(ctx, out->means_opacity, 16, "out means_opacity", false))) return s;
    if ((s = check_device_array(ctx, out->quats, 16, "out quats", false))) return s;
    if ((s = check_device_array(ctx, out->scales, 16, "out scales", false))) return s;
    if ((s = check_device_array(ctx, out->flags, 4, "out flags", false))) return s;
    if ((s = check_device_array(ctx, out->nbr_pos, 4, "out nbr_pos", true))) return s;
    if ((s = check_device_array(ctx, out->nbr_cov, 4, "out nbr_cov", true))) return s;
    const void* ins[7] = {before->means_opacity, before->quats, before->scales, fitted->means, fitted->quats,
                          fitted->scales, fitted->status};
    const void* outs[4] = {out->means_opacity, out->quats, out->scales, out->flags};
    for (const void* a : ins)
        for (const void* b : outs)
            if (a == b) return fail(ctx, TSP_ERR_INVALID_ARG, "outputs must not overlap inputs");
    const float* mom = view_moments;
    if (mom) {
        if ((s = check_device_array(ctx, mom, 16, "view_moments", false))) return s;
    } else if (num_views > 0) {
        if (ctx->last_fit_n != n || ctx->last_fit_V != num_views || !ctx->moments.p)
            return fail(ctx, TSP_ERR_INVALID_ARG,
                        "view_moments is NULL and the context's last fit had another n or number of views");
        mom = (const float*)ctx->moments.p;
    }
    RegParams rp{};
    rp.n = n;
    rp.V = num_views;
    rp.k = o.k;
    rp.min_views = o.static_min_views;
    rp.min_px = o.static_min_px;
    rp.frac = o.static_frac;
    rp.moments = mom;
    rp.status = fitted->status;
    rp.mo0 = (const float4*)before->means_opacity;
    rp.q0 = (const float4*)before->quats;
    rp.s0 = (const float4*)before->scales;
    rp.mo1 = (const float4*)fitted->means;
    rp.q1 = (const float4*)fitted->quats;
    rp.s1 = (const float4*)fitted->scales;
    rp.nbr_pos = out->nbr_pos;
    rp.nbr_cov = out->nbr_cov;
    rp.mo_out = (float4*)out->means_opacity;
    rp.q_out = (float4*)out->quats;
    rp.s_out = (float4*)out->scales;
    rp.flags = out->flags;
    KnnWork kw{};
    if ((s = ensure_reg(ctx, n, o.k, kw, &rp))) return s;
    TSP_CUDA(launch_regularize(rp, kw, (cudaStream_t)stream));
    return TSP_OK;
}

tsp_status tsp_knn(tsp_context* ctx, const float* means_opacity, const uint8_t* mask, int n, int k,
                   int32_t* nbr, void* stream)
{
    if (!ctx) return TSP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    if (n < 0) return fail(ctx, TSP_ERR_INVALID_ARG, "n < 0");
    if (k < 1 || k > TSP_REG_MAX_K) return fail(ctx, TSP_ERR_INVALID_ARG, "k must be in [1, TSP_REG_MAX_K]");
    if (n == 0) return TSP_OK;
    tsp_status s;
    if ((s = check_device_array(ctx, means_opacity, 16, "means_opacity", false))) return s;
    if ((s = check_device_array(ctx, mask, 1, "mask", false))) return s;
    if ((s = check_device_array(ctx, nbr, 4, "nbr", false))) return s;
    KnnWork kw{};
    if ((s = ensure_reg(ctx, n, k, kw, nullptr))) return s;
    const uint8_t bits = 0xff;
    TSP_CUDA(launch_knn((const float4*)means_opacity, mask, &bits, 1, n, k, kw, nbr, nbr, (cudaStream_t)stream));
    return TSP_OK;
}

tsp_status tsp_workspace_bytes(const tsp_context* ctx, size_t* bytes)
{
    if (!ctx || !bytes) return TSP_ERR_INVALID_ARG;
    *bytes = ctx->held;
    return TSP_OK;
}

}  // extern "C"

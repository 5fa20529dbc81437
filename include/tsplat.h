/*
 * tsplat.h -- C ABI of libtsplat.so: the TrackerSplat motion-compensation hot path
 * (arXiv 2604.02586, Sec. 4.2-4.4) on one NVIDIA B300 (sm_103a).
 *
 * Problem statement (Sec. 4.1, 4.3.1, 4.4): frame-0 3D Gaussians, calibrated
 * cameras and, per view, a dense track x -> x' for every pixel go in; every
 * Gaussian comes out relocated, rotated and rescaled, with a status word.
 *
 * Conventions shared by every entry point
 *   - Camera: world -> camera p = R X + t (R row-major), +z forward; pixel (i, j)
 *     (column i, row j) has centre (i + 0.5, j + 0.5); u = fx p_x / p_z + cx.
 *   - Gaussian: mean, opacity in (0,1), quaternion (w, x, y, z) (need not be unit),
 *     linear scales > 0; Sigma_3D = R(q) diag(s^2) R(q)^T (Sec. 3.1).
 *   - Images are row-major [H][W]; tracks are x' - x in pixels (FP32 pairs).
 *   - "device" pointers are CUDA device (or managed) memory on the context's device,
 *     "host" pointers are ordinary CPU memory.  The caller owns every buffer passed
 *     in; the context owns its workspace (per-view records, tile lists, moments).
 *   - Every call returns a tsp_status and never throws.  Argument errors are
 *     reported synchronously, before any work is enqueued.  Work is enqueued on
 *     the caller's stream (a cudaStream_t passed as void*, NULL = legacy default
 *     stream); device-side conditions (pair-buffer overflow) are latched in a
 *     device status word that tsp_sync() reports.
 *   - A context is not thread-safe: use one context per host thread.  Two calls
 *     on one context must not overlap on the GPU (the workspace is shared); the
 *     library does not order them for you if they use different streams.
 */
#ifndef TSPLAT_H
#define TSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSP_VERSION 1
#define TSP_MAX_VIEWS 32          /* views of one frame                                */
#define TSP_MAX_FRAMES 16         /* frames of one tsp_fit_motion_batch call           */
#define TSP_MAX_BATCH_VIEWS 192   /* views of all frames of one tsp_fit_motion_batch   */
#define TSP_MAX_IMAGE 8192

typedef enum {
    TSP_OK = 0,
    TSP_ERR_INVALID_ARG = 1,   /* bad pointer, size, alignment or option     */
    TSP_ERR_OOM = 2,           /* workspace allocation failed                */
    TSP_ERR_CUDA = 3,          /* a CUDA runtime call failed (see last error) */
    TSP_ERR_TIMEOUT = 4,       /* tsp_sync gave up before the work finished  */
    TSP_ERR_BUDGET = 5,        /* workspace would exceed the context budget  */
    TSP_ERR_OVERFLOW = 6       /* more (tile, Gaussian) pairs than capacity  */
} tsp_status;

/* Per-view flags (tsp_result.view_flags) -- Sec. 4.3.5 and Sec. 5.1. */
#define TSP_VIEW_OK 1u          /* affine solved in this view                      */
#define TSP_VIEW_FEW_PX 2u      /* fewer than min_px_view pixels added moments     */
#define TSP_VIEW_LOW_ALPHA 4u   /* accumulated alpha (sum of w) < sumw_min_view    */
#define TSP_VIEW_SINGULAR 8u    /* det V1 < det_min or pixel scatter too thin      */
#define TSP_VIEW_CULLED 16u     /* behind the near plane, off-frustum or no tile   */

/* Per-Gaussian status bits (tsp_result.status) -- Sec. 4.4 and Sec. 5.1.
 * Bits 16..23 hold the number of views whose affine was solved. */
#define TSP_POS_OK 1u           /* mu_3D' triangulated                             */
#define TSP_COV_OK 2u           /* Sigma_3D' fitted, rotation and scale updated    */
#define TSP_NEG_EIG 4u          /* Sigma_3D' had an eigenvalue <= 0 (Sec. 4.4.3)   */
#define TSP_FEW_VIEWS 8u        /* fewer than min_views solved views               */
#define TSP_LOW_ALPHA 16u       /* accumulated alpha over views < sumw_min_total   */
#define TSP_FEW_PX 32u          /* fewer than min_px_total pixels over views       */
#define TSP_COV_SINGULAR 64u    /* covariance system rank-deficient                */
#define TSP_TRI_SINGULAR 128u   /* triangulation system rank-deficient             */

typedef struct tsp_camera {
    int32_t width, height;      /* pixels, 1..TSP_MAX_IMAGE                        */
    float fx, fy, cx, cy;       /* pinhole intrinsics in pixels, fx, fy > 0        */
    float R[9];                 /* world -> camera rotation, row-major             */
    float t[3];                 /* world -> camera translation                     */
} tsp_camera;

typedef struct tsp_gaussians {
    int32_t n;                  /* number of Gaussians, 0 <= n < 2^28 (INVALID_ARG) */
    const float* means_opacity; /* [n][4] (x, y, z, opacity); 16-byte aligned      */
    const float* quats;         /* [n][4] (w, x, y, z); 16-byte aligned            */
    const float* scales;        /* [n][4] (sx, sy, sz, unused), linear; 16-byte al. */
} tsp_gaussians;

typedef struct tsp_view_tracks {
    const float* disp;          /* [H][W][2] tracked x' - x in pixels; 8-byte al.  */
    const uint8_t* vis;         /* [H][W] non-zero = the track is valid            */
} tsp_view_tracks;

typedef struct tsp_result {
    float* means;               /* [n][4] new (x, y, z, opacity unchanged)         */
    float* quats;               /* [n][4] new (w, x, y, z), unit                   */
    float* scales;              /* [n][4] new (sx, sy, sz, 0)                      */
    uint32_t* status;           /* [n] TSP_* bits                                  */
    float* view_affine;         /* optional [V][n][6]: A00 A01 A10 A11 b0 b1 (Eq. 2) */
    float* view_moments;        /* optional [V][n][16] PWI-LS moments, see below    */
    uint32_t* view_flags;       /* optional [V][n] TSP_VIEW_* bits                 */
} tsp_result;
/* view_moments layout, w = alpha T (Eq. 4), d = x' - x the tracked displacement and
 * (x~, y~) = pixel centre minus the moment origin o, where o is mu_2D clamped to
 * the image rectangle [0, W] x [0, H] (o = mu_2D whenever the centre is on-image):
 *   0 sum w            1 sum w x~         2 sum w y~        3 sum w x~^2
 *   4 sum w x~ y~      5 sum w y~^2       6 sum w dx        7 sum w dy
 *   8 sum w x~ dx      9 sum w x~ dy     10 sum w y~ dx    11 sum w y~ dy
 *  12 sum w over static pixels (|d| < 1)  13 pixels added    14 static pixels  15 0
 * In slots 6-11, d is taken relative to a reference displacement r (the track at
 * the pixel holding o), which leaves [A] unchanged and adds r to the intercept.
 * Eq. 4's V1 and V2 follow: V1 = [[3,4,1],[4,5,2],[1,2,0]] and
 * V2 = V1[:, 0:2] + [[8,9],[10,11],[6,7]] + V1[:, 2] r^T in this (x~, y~, 1) basis. */

/* One frame pair of a batch: its Gaussians, cameras, tracks and outputs, with
 * the same meaning and memory rules as the arguments of tsp_fit_motion. */
typedef struct tsp_frame {
    tsp_gaussians g;
    const tsp_camera* cams;     /* host [num_views]                                */
    int32_t num_views;          /* 0..TSP_MAX_VIEWS                                */
    const tsp_view_tracks* tracks; /* host [num_views] of device pointers          */
    tsp_result out;
} tsp_frame;

typedef struct tsp_options {
    int32_t tile_w, tile_h;     /* raster tile: 16 x 16 (default) or 32 x 8; with */
                                /*    32 x 8, raster_variant must be 0 or 5        */
    float det_min;              /* Sec. 5.1: 1e-12                                 */
    float sumw_min_view;        /* Sec. 5.1: 1e-3                                  */
    int32_t min_px_view;        /* Sec. 5.1: 2                                     */
    float lam_min_px2;          /* thin-pixel-set guard: 1e-4 px^2                 */
    int32_t min_views;          /* Sec. 5.1: 2                                     */
    float sumw_min_total;       /* Sec. 5.1: 1e-3                                  */
    int32_t min_px_total;       /* Sec. 5.1: 3                                     */
    float cov_rcond_min;        /* covariance system sigma_min/sigma_max floor:    */
                                /*    1e-6, in [1e-12, 1).  Two views always leave */
                                /*    the system rank 5 (Sec. 4.4.2), so a Gaussian */
                                /*    solved in exactly two views is COV_SINGULAR   */
    int32_t async_pairs;        /* 0: tsp_fit_motion waits for the pair count and  */
                                /*    grows the pair buffer before sorting;        */
                                /* 1: never waits; overflow -> TSP_ERR_OVERFLOW at  */
                                /*    tsp_sync, capacity grows for the next call   */
    int32_t stage_timing;       /* 1: record CUDA events between the steps of each  */
                                /*    call; read them with tsp_stage_times          */
    int32_t collect_stats;      /* 1: the raster step also counts its work (slower; */
                                /*    for measurement only), see TSP_I_STATS        */
    int32_t raster_variant;     /* a5 kernel: 0 = two-phase (blend, then per-hit */
                                /*    moment sums; 8x8 warp blocks), the default;  */
                                /*    5 = the same, persistent: resident CTAs whose */
                                /*    warps take (tile, block) items from a queue;  */
                                /*    1, 2, 4 = warp-shuffle reduction with 1, 2, 4 */
                                /*    pixels per thread (8x4, 8x8, 8x16 blocks)     */
    int64_t pair_capacity;      /* initial (tile, Gaussian) pair capacity, 0 = auto */
    int64_t budget_bytes;       /* workspace ceiling, 0 = unlimited                */
    int32_t checked;            /* 1: checked mode (debugging): every index a      */
                                /*    kernel takes from data -- a (record, tile)   */
                                /*    item's tile and list slot, tile ranges, the  */
                                /*    moment origin's pixel, a list entry's        */
                                /*    Gaussian -- is tested against its buffer     */
                                /*    before use; a failed test skips the access   */
                                /*    and is recorded in the device status word,   */
                                /*    which tsp_sync reports as TSP_ERR_CUDA with  */
                                /*    the site.  0 (default): no tests             */
} tsp_options;

typedef struct tsp_context tsp_context;

/* Fill *out with the defaults above.  Errors: INVALID_ARG if out is NULL. */
tsp_status tsp_default_options(tsp_options* out);

/* Create a context on CUDA device `device`.  opt may be NULL (defaults).
 * Errors: INVALID_ARG (bad option), CUDA (device unusable).  *out is set to NULL
 * on failure. */
tsp_status tsp_create(int device, const tsp_options* opt, tsp_context** out);

/* Free the workspace and the context (synchronizes the device). NULL is a no-op. */
tsp_status tsp_destroy(tsp_context* ctx);

/* The motion-compensation step (Sec. 4.2-4.4), enqueued on `stream`:
 *   a1 project every (view, Gaussian) (Eq. 1), cull, key = (tile, depth);
 *   a2 count and emit (tile, Gaussian) pairs; a3 sort each tile's list by depth;
 *   a5 blend front to back per pixel and add w = alpha T weighted track moments
 *      per Gaussian (Eq. 4, Sec. 4.3.5);
 *   a6 per (view, Gaussian): discard tests (Sec. 5.1), [A|b] = V1^-1 V2 (Eq. 4),
 *      mu_2D' and Sigma_2D' (Eq. 2);
 *   a7 triangulate mu_3D' (Sec. 4.4.1); a8 fit Sigma_3D' (Sec. 4.4.2);
 *   a9 eigen-decompose, reorder, update rotation and scale (Sec. 4.4.3).
 * g: device arrays; cams: host [num_views]; tracks: host [num_views] of device
 * pointers sized by each camera; out: host struct of device pointers (optional
 * members may be NULL).  Unsolvable Gaussians keep their input values.
 * Unless options.async_pairs is set, the call waits once (after a2's count) so
 * that it can size the pair buffer.  Errors: INVALID_ARG, OOM, BUDGET, CUDA. */
tsp_status tsp_fit_motion(tsp_context* ctx, const tsp_gaussians* g, const tsp_camera* cams,
                          int num_views, const tsp_view_tracks* tracks, const tsp_result* out,
                          void* stream);

/* Several frame pairs (Sec. 4.6: frame pairs are independent units) in one
 * launch of each step: up to TSP_MAX_FRAMES frames of uneven Gaussian counts and
 * view counts, at most TSP_MAX_BATCH_VIEWS views in all.  Each frame's outputs
 * are those tsp_fit_motion would give it alone (floating-point sums may differ in
 * the last bits: atomic additions run in another order).  The pair buffer holds
 * the pairs of all frames; tsp_inspect reports the records of all frames, frame
 * by frame, view-major within a frame.  Errors as tsp_fit_motion. */
tsp_status tsp_fit_motion_batch(tsp_context* ctx, const tsp_frame* frames, int num_frames, void* stream);

/* Autotuner: runs the motion fit on the given frames (outputs are written) with
 * each candidate (tile shape, raster kernel and block shape), in this order:
 *   0: 16 x 16, two-phase, 8x8 warp blocks, one CTA per tile (variant 0)
 *   1: 16 x 16, two-phase persistent over a work queue (variant 5)
 *   2, 3, 4: 16 x 16, warp-shuffle with 8x8, 8x4, 8x16 blocks (variants 2, 1, 4)
 *   5: 32 x 8, variant 0          6: 32 x 8, variant 5
 * `repeats` timed times after one warm-up each (the pair buffer is sized
 * synchronously for each tile shape), and keeps the candidate whose median time
 * of the whole fit (binning differs between tile shapes) is lowest: the context's
 * tile_w, tile_h and raster_variant become its values.  chosen (nullable)
 * receives its index, fit_ms (nullable, [TSP_TUNE_CANDIDATES]) the medians in
 * that order.  Synchronises the stream.  Errors as tsp_fit_motion_batch; the
 * options are left unchanged on error. */
#define TSP_TUNE_CANDIDATES 7
tsp_status tsp_autotune(tsp_context* ctx, const tsp_frame* frames, int num_frames, int repeats, void* stream,
                        int* chosen, float* fit_ms);

/* The autotuner with a cache file, so that a workload is timed once per machine
 * and its choice reused by later processes (a tuning choice of the batched launch,
 * the paper's per-frame parallelism of Sec. 4.6).  The key of a call is (bit length
 * of the frames' total Gaussian count, total views, largest view's W x H); the
 * file (cache_path, a host path) holds one text line per tuned key,
 * "tsp-autotune-v1 <bits> <views> <pixels> <candidate> <median ms>", and the last
 * line of a key wins.  A key found in the file: its candidate's options are set
 * and nothing runs on the GPU (*from_cache = 1, fit_ms[candidate] = the stored
 * median, the other entries -1).  Otherwise tsp_autotune runs as above and a line
 * is appended (*from_cache = 0).  Lines of another form are skipped.  cache_path
 * NULL: tsp_autotune alone.  chosen, fit_ms, from_cache are nullable.
 * Errors: INVALID_ARG (bad frames, or the file cannot be opened for appending:
 * checked before any tuning), those of tsp_autotune. */
tsp_status tsp_autotune_cached(tsp_context* ctx, const tsp_frame* frames, int num_frames, int repeats,
                               void* stream, const char* cache_path, int* chosen, float* fit_ms,
                               int* from_cache);

/* Same step for callers that hold everything in host memory: g, tracks and out
 * point to host arrays (pinned memory gives full copy speed and lets the copies
 * overlap the computation).  The Gaussians are copied on `stream` and projected,
 * binned and sorted while the tracks are copied on a context-owned stream, one
 * view at a time; each view's raster starts once its tracks have landed.
 * Results are copied back and the call returns after both streams have finished
 * with the caller's buffers.  Errors as tsp_fit_motion, plus OVERFLOW if the pair
 * buffer overflowed. */
tsp_status tsp_fit_motion_host(tsp_context* ctx, const tsp_gaussians* g, const tsp_camera* cams,
                               int num_views, const tsp_view_tracks* tracks,
                               const tsp_result* out, void* stream);

/* Render colour and final transmittance (Sec. 3.1 blending, same tiles and order
 * as tsp_fit_motion).  sh: device [n][(sh_degree+1)^2][3] real spherical-harmonic
 * colour coefficients (degree 0..3, colour = sum c_k Y_k(view dir) + 0.5, clamped
 * at 0); rgb, final_T: host arrays [num_views] of device pointers to [H][W][3] and
 * [H][W] FP32.  Errors: INVALID_ARG, OOM, BUDGET, CUDA. */
tsp_status tsp_render(tsp_context* ctx, const tsp_gaussians* g, const float* sh, int sh_degree,
                      const tsp_camera* cams, int num_views, float* const* rgb,
                      float* const* final_T, void* stream);

/* Gradients of a render with respect to the Gaussians (gradient refinement). */
typedef struct tsp_render_grads {
    float* means;               /* [n][4]: dL/d(mean x, y, z), dL/dopacity in w    */
    float* scales;              /* [n][4]: dL/d(linear scale x, y, z), 0           */
    float* quats;               /* [n][4]: dL/d(raw quaternion w, x, y, z)         */
    float* sh;                  /* [n][(sh_degree+1)^2][3]                         */
} tsp_render_grads;

/* Adjoint of tsp_render (the blend of Sec. 3.1): given the colour rgb that
 * tsp_render gave for these Gaussians, colour coefficients and cameras, and
 * grad_rgb = dL/dcolour ([num_views] device pointers to [H][W][3] FP32 each), the
 * gradient of L with respect to every Gaussian's mean, opacity, linear scales,
 * raw quaternion and colour coefficients, with the blend's decisions (tile
 * rectangle, footprint box, alpha >= 1/255, transmittance cut-off, clamps of
 * alpha at 0.99 and of the colour at 0) held fixed.  The tile lists are rebuilt
 * and the blend is recomputed tile by tile; nothing per pixel is kept between the
 * two calls.  When the previous binning on this context was tsp_render with the
 * same Gaussian and colour arrays and cameras (the render whose rgb is passed in),
 * its tile lists are still in the workspace and are reused; any other binning in
 * between (a fit, another render) makes the call build them again.  All arrays are
 * device memory.  Errors as tsp_render. */
tsp_status tsp_render_backward(tsp_context* ctx, const tsp_gaussians* g, const float* sh, int sh_degree,
                               const tsp_camera* cams, int num_views, const float* const* rgb,
                               const float* const* grad_rgb, const tsp_render_grads* out, void* stream);

/* ---- Motion regularization (Sec. 4.5) ------------------------------------ */
/* Per-Gaussian bits of tsp_reg_result.flags. */
#define TSP_REG_STATIC 1u           /* static (Sec. 4.5.2): motion discarded           */
#define TSP_REG_POS_MEDIAN 2u       /* position change median-filtered (Sec. 4.5.1)    */
#define TSP_REG_POS_PROPAGATED 4u   /* position change propagated from neighbours      */
#define TSP_REG_COV_MEDIAN 8u       /* scale and rotation change median-filtered       */
#define TSP_REG_COV_PROPAGATED 16u  /* scale and rotation change propagated            */
#define TSP_REG_MAX_K 16

typedef struct tsp_reg_options {
    int32_t k;                  /* nearest neighbours, 1..TSP_REG_MAX_K; Sec. 5.1: 8 */
    float static_min_px;        /* Sec. 4.5.2: a static view has more than 9 pixels  */
    float static_frac;          /*    and more than 0.9 of them static (|d| < 1 px), */
    int32_t static_min_views;   /*    in at least 2 views                            */
} tsp_reg_options;

tsp_status tsp_default_reg_options(tsp_reg_options* o);

typedef struct tsp_reg_result {
    float* means_opacity;       /* [n][4] regularized (x, y, z, opacity of before)  */
    float* quats;               /* [n][4] regularized (w, x, y, z), unit             */
    float* scales;              /* [n][4] regularized (sx, sy, sz, w of before)      */
    uint32_t* flags;            /* [n] TSP_REG_* bits                                */
    int32_t* nbr_pos;           /* optional [n][k]: the k nearest Gaussians with a   */
    int32_t* nbr_cov;           /*    solved position / covariance, -1 padded        */
} tsp_reg_result;

/* Motion regularization of one frame pair (Sec. 4.5), after tsp_fit_motion.
 * before: the Gaussians the fit started from; fitted: its outputs (means, quats,
 * scales, status; the optional view arrays are not read).  A Gaussian's motion
 * components are its position change dmu = mu' - mu (when TSP_POS_OK) and, when
 * TSP_COV_OK, its scale change ds = s' - s and rotation change dR = R' R^T as
 * Euler angles (x, y, z), dR = Rz(ez) Ry(ey) Rx(ex).
 *  - Static (Sec. 4.5.2): more than static_min_px pixels and more than
 *    static_frac of them static (view_moments slots 13 and 14, compared in FP32
 *    as nstat > frac * npix) in at least static_min_views views.  Its motion is
 *    discarded and it takes no part in the filtering or the propagation.
 *  - Median filter (Sec. 4.5.1): a Gaussian with a component takes, coordinate by
 *    coordinate, the median of that component over itself and its k nearest
 *    other Gaussians with the component.
 *  - Propagation (Sec. 4.5.2), from the filtered values: a non-static Gaussian
 *    without a component takes the mean of the component over its k nearest
 *    Gaussians with it (none: unchanged).
 *  - Nearness is the FP32 squared distance between `before` means, computed as
 *    ((dx*dx + dy*dy) + dz*dz) with dx = x_query - x_other and no fused
 *    multiply-add, ties by the smaller index; the neighbour sets are exact.
 * The outputs are mu + dmu, s + ds and R(e) R (quaternion sign kept on the side
 * of the old one).  view_moments: device [num_views][n][16] as
 * tsp_result.view_moments, or NULL for the moments the context holds from its
 * last tsp_fit_motion / tsp_fit_motion_host call, which must have had the same
 * n and num_views (INVALID_ARG otherwise).  Means must be finite.  All arrays are
 * device memory of the context's device, 16-byte aligned ([n][4], view_moments)
 * or 4-byte aligned (flags, nbr_*); outputs must not overlap inputs.  The neighbour
 * search (a uniform grid, or an exact bounding-volume hierarchy for point sets
 * whose density varies by orders of magnitude) is sized and chosen on the device:
 * no host wait; enqueues on `stream` and may be captured in a CUDA graph once the
 * workspace for this n and k exists.  Errors: INVALID_ARG, OOM, BUDGET, CUDA; a
 * search whose bounded walk gave up (not expected for finite means) is reported
 * by the next tsp_sync as CUDA. */
tsp_status tsp_regularize(tsp_context* ctx, const tsp_gaussians* before, const tsp_result* fitted,
                          const float* view_moments, int num_views, const tsp_reg_options* opt,
                          const tsp_reg_result* out, void* stream);

/* The k nearest members of `mask` (device uint8 [n], non-zero = member) other
 * than the point itself, for every point of means_opacity (device [n][4]), by
 * the FP32 squared distance and tie rule of tsp_regularize; nbr: device
 * int32 [n][k], -1 padded when fewer than k members exist.  1 <= k <=
 * TSP_REG_MAX_K.  Enqueues on `stream`.  Errors as tsp_regularize. */
tsp_status tsp_knn(tsp_context* ctx, const float* means_opacity, const uint8_t* mask, int n, int k,
                   int32_t* nbr, void* stream);

/* Wait up to timeout_ms (< 0: forever) for `stream`, then read and clear the
 * device status word.  Returns OK, TIMEOUT (work still running; call again),
 * OVERFLOW (the last step ran out of pair capacity; its results are invalid and
 * the capacity has been raised for the next call) or CUDA. */
tsp_status tsp_sync(tsp_context* ctx, void* stream, int timeout_ms);

/* Intermediates of the last tsp_fit_motion / tsp_render, for inspection and tests.
 * Call after tsp_sync.  Copies min(bytes, size) bytes to host memory dst and sets
 * *size_out (nullable) to the full size in bytes.  dst may be NULL to query size. */
typedef enum {
    TSP_I_COUNTS = 0,        /* int64[4]: K pairs, NT tiles, pair capacity, overflow */
    TSP_I_RECT = 1,          /* int16[V][n][4]: tile rect x0 y0 x1 y1 (all 0 = culled) */
    TSP_I_DEPTH = 2,         /* uint32[V][n]: bits of the FP32 camera depth          */
    TSP_I_TILES_TOUCHED = 3, /* uint32[V][n]                                         */
    TSP_I_TILE_OFFSETS = 4,  /* uint32[NT+1]: tile t owns pairs [off[t], off[t+1])   */
    TSP_I_PAIRS = 5,         /* uint64[K]: depth_bits << 32 | Gaussian, sorted per tile */
    TSP_I_MOMENTS = 6,       /* float[V][n][16], layout as view_moments              */
    TSP_I_STATS = 7,         /* uint64[8] raster work of the last call when           */
                             /* collect_stats = 1: (pixel, Gaussian) evaluations,     */
                             /* blended contributions, moment additions, list entries;*/
                             /* two-phase kernels also: block hits (entries whose     */
                             /* alpha >= 1/255 ellipse meets an 8x8 block), hits that */
                             /* add a pixel, moment passes, 32-entry walk steps       */
    TSP_I_VIEW_MEANS = 8,    /* float[V][n][4]: mu_2D' (x, y) and its shift from mu_2D */
    TSP_I_VIEW_COV = 9,      /* float[V][n][8]: rows of B with Sigma_2D' = B B^T     */
                             /* (B00 B01 B02 sum-w, B10 B11 B12 0)                     */
    TSP_I_KNN_PATH = 10      /* uint32[2]: neighbour search of the last tsp_knn /     */
                             /* tsp_regularize per candidate set: 0 grid, 1 BVH       */
} tsp_intermediate;
tsp_status tsp_inspect(tsp_context* ctx, int which, void* dst, size_t bytes, size_t* size_out);

/* Device time in milliseconds of the steps of the last call made with
 * stage_timing = 1: [0] a1 projection (with the buffer clears), [1] a2 scan,
 * [2] a2 emit, [3] a3 tile sort, [4] a5 raster-accumulate (or render),
 * [5] a6 per-view solve, [6] a7-a9 multi-view update.  Waits for the call's
 * events.  Writes min(max_n, 7) values; *count (nullable) = 7.
 * Errors: INVALID_ARG (no timed call yet), CUDA. */
tsp_status tsp_stage_times(tsp_context* ctx, float* ms, int max_n, int* count);

/* Per-tile depth sort without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc
 * -- memory-capped tenants of a shared GPU whose budget someone else hands out,
 * hosts whose own allocator owns all device memory, and loops that cannot afford
 * the device-wide synchronization an allocation or a free may bring.
 * keys: device [num_keys] (depth_bits << 32 | Gaussian), sorted ascending in
 * place within each tile t's slice [offsets[t], offsets[t+1]); keys need not be
 * unique (equal keys are equal values, so their order is immaterial); offsets: device
 * [num_tiles + 1], non-decreasing, offsets[num_tiles] = num_keys (slices are
 * clamped to num_keys).  Both on the current CUDA device; keys 8-byte aligned.
 * The merge scratch for long lists lives in a fixed array inside the library
 * (TSP_NOALLOC_SORT_MAX_KEYS keys, 8 MB), held by every GPU that loads the
 * library until the process exits.  The first call on a device looks up that
 * array's device address (with the device current); make that first call before
 * any stream capture.  All calls share the array, so calls that overlap on the
 * GPU race with each other; nothing in it needs clearing between calls.
 * Errors: INVALID_ARG (num_keys > TSP_NOALLOC_SORT_MAX_KEYS, NULL or misaligned
 * pointer), CUDA (lookup or launch failed).  Enqueues on `stream`; no wait. */
#define TSP_NOALLOC_SORT_MAX_KEYS (1u << 20)
tsp_status tsp_sort_tiles_noalloc(uint64_t* keys, const uint32_t* offsets, uint32_t num_tiles,
                                  uint32_t num_keys, void* stream);

/* Workspace allocator hook.  The context's device buffers (sort buffers, moment
 * records, per-view results, staging) come from alloc(bytes, device, user) and
 * go back through release(ptr, bytes, device, user) instead of cudaMalloc and
 * cudaFree: a host whose own allocator owns the device memory (a framework's
 * caching allocator, a tenant with a fixed pool) hands its allocator in here.
 * alloc returns device memory on `device`, 256-byte aligned, or NULL to refuse
 * (the call that needed it then fails with TSP_ERR_OOM, nothing of it enqueued,
 * and the context stays usable).  Both NULL restores cudaMalloc / cudaFree.
 * The call waits for the device, returns the current workspace to the allocator
 * that gave it, and installs the new pair; later calls allocate afresh.  The
 * pointers must stay valid until the context is destroyed or the hook replaced.
 * Errors: INVALID_ARG (ctx NULL, exactly one of alloc / release NULL), CUDA. */
typedef void* (*tsp_alloc_fn)(size_t bytes, int device, void* user);
typedef void (*tsp_free_fn)(void* ptr, size_t bytes, int device, void* user);
tsp_status tsp_set_allocator(tsp_context* ctx, tsp_alloc_fn alloc, tsp_free_fn release, void* user);

/* Device-side start gate of the calls that read caller-owned device tracks
 * (tsp_fit_motion, tsp_fit_motion_batch; not the host-buffer call, which copies
 * its tracks itself).  With a gate set, such a call projects, bins and sorts as
 * usual, then waits on the device -- the host is not involved -- until the
 * 32-bit word at `flag` (device memory of the context's device, 4-byte aligned)
 * is >= `value`, polling with acquire semantics about once a microsecond: a
 * producer that writes the tracks on another stream posts the word after them
 * (with release semantics: a stream-ordered write or a fence before the store).
 * The wait gives up after `timeout_us` microseconds (the GPU's global timer,
 * and a poll count as a second bound); the call then computes nothing from the
 * tracks and writes none of its fitted outputs (means, quats, scales, status,
 * view_affine, view_flags; a requested view_moments copy holds zeros), and
 * tsp_sync reports TSP_ERR_TIMEOUT.  The context stays usable.  flag NULL
 * removes the gate.  The wait counts in the raster stage's time.
 * Errors: INVALID_ARG (ctx NULL, flag misaligned or not device memory,
 * timeout_us outside [1, 1e7]). */
tsp_status tsp_set_track_gate(tsp_context* ctx, const uint32_t* flag, uint32_t value, int64_t timeout_us);

/* Replace the workspace ceiling (options.budget_bytes; 0 = unlimited).  A call
 * whose workspace would grow past it fails with TSP_ERR_BUDGET before any of its
 * work is enqueued (with async_pairs = 0, a pair buffer grown after the count
 * fails the same way, before the scatter).  Held workspace is not shrunk.
 * Errors: INVALID_ARG (ctx NULL, budget_bytes < 0). */
tsp_status tsp_set_budget(tsp_context* ctx, int64_t budget_bytes);

/* Bytes of device workspace the context currently holds. */
tsp_status tsp_workspace_bytes(const tsp_context* ctx, size_t* bytes);

/* Static strings; never NULL. */
const char* tsp_status_string(tsp_status s);
const char* tsp_last_error(const tsp_context* ctx);
int tsp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TSPLAT_H */

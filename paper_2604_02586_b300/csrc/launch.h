// launch.h -- host-side launchers of the libtsplat kernels (one per pipeline step).
#pragma once

#include "common.cuh"

namespace tsp {

// a1: project every (view, Gaussian) of every frame, zero its moment record,
// count tiles.  mode 0 = motion fit, 1 = render (one frame; colour from sh).
cudaError_t launch_preprocess(const ViewSet& vs, const float* sh, int sh_degree, int mode, const Work& w,
                              cudaStream_t st);
// a1 (fit mode): reference displacement of views [v0, v1) -- the track at each
// record's moment origin.  Needs those views' tracks; the other steps of a1-a4 do not.
cudaError_t launch_dref(const ViewSet& vs, const Work& w, int v0, int v1, cudaStream_t st);
cudaError_t launch_track_gate(const uint32_t* flag, uint32_t value, long long timeout_us, const Work& w,
                              cudaStream_t st);
// a2: exclusive scan of the per-tile counts -> tile offsets and the pair count K.
cudaError_t launch_scan(const Work& w, uint32_t NT, cudaStream_t st);
// Exclusive scan of n counts cnt[i * stride] into off[0..n] (off[n] = total);
// span_sum: ceil(n / 1024) + 1 scratch words; status[1..2] receive the total and
// status[0] bit 0 is set if it exceeds cap.
// With enable != nullptr every kernel returns at once when *enable == 0.
cudaError_t launch_scan_u32(const uint32_t* cnt, uint32_t stride, uint32_t n, uint32_t* off,
                            unsigned long long* span_sum, uint32_t cap, uint32_t* status, cudaStream_t st,
                            const uint32_t* enable = nullptr);
// Sort each of nseg segments [off[s], off[s + 1]) of 64-bit keys ascending (keys
// unique within a segment); tmp: as many keys as keys, long_list: nseg words,
// long_count: one word.  With enable != nullptr the kernels return at once when
// *enable == 0.
cudaError_t launch_segment_sort(const uint32_t* off, uint64_t* keys, uint64_t* tmp, uint32_t cap, uint32_t nseg,
                                uint32_t* long_list, uint32_t* long_count, cudaStream_t st,
                                const uint32_t* enable = nullptr);
// a2: emit (depth << 32 | g) into each touched tile's slice.
cudaError_t launch_scatter(const ViewSet& vs, const Work& w, cudaStream_t st);
// a3: sort each tile's slice ascending (depth, then Gaussian index).
cudaError_t launch_tile_sort(const Work& w, uint32_t NT, cudaStream_t st);
// a5: blend and accumulate alpha T weighted track moments per (view, Gaussian), for
// the ntiles tiles starting at tile_base (tiles are numbered view by view).
// variant 0: two-phase, one CTA per tile; 5: two-phase persistent over
// resident_ctas CTAs fed by a device-side queue (w.queue); 1, 2, 4: warp-shuffle
// reduction with that many pixels per thread.
cudaError_t launch_raster_accumulate(const ViewSet& vs, const Work& w, uint32_t tile_base, uint32_t ntiles,
                                     bool stats, int variant, int resident_ctas, cudaStream_t st);
// One-time kernel attributes of the raster step (shared-memory carveout).
cudaError_t raster_prepare();
// Shared-memory carveout of the render adjoint (once per context).
cudaError_t backward_prepare();
// CTAs of the persistent raster that fit on the device at once.
int raster_resident_ctas(int device);
// the render's adjoint: dL/dcolour -> per (view, Gaussian) 2D gradients
// (tile-recomputed blend) -> dL/d(mean, opacity, scales, quaternion, colour
// coefficients) per Gaussian.
cudaError_t launch_render_backward(const ViewSet& vs, const Work& w, uint32_t NT, const RenderGrad& rg,
                                   const float* sh, int sh_degree, size_t records, cudaStream_t st);
// render colour and final transmittance.
cudaError_t launch_raster_render(const ViewSet& vs, const Work& w, uint32_t NT, float* const* rgb,
                                 float* const* final_T, cudaStream_t st);
// a6: per-view discard tests, affine solve, Eq. 2.
cudaError_t launch_view_solve(const ViewSet& vs, const FitParams& fp, const Work& w, const FrameOut& fo,
                              cudaStream_t st);
// a7-a9: triangulation, covariance fit, eigen decomposition and outputs, per frame.
cudaError_t launch_multiview(const ViewSet& vs, const FitParams& fp, const Work& w, const FrameOut& fo,
                             cudaStream_t st);

// Motion regularization (Sec. 4.5).
struct GridParam {                  // uniform grid of one component's members
    float lo[3], inv[3], h[3];      // box corner, cells per unit, cell edge
    int dims[3];
    int ncell;
    float margin;                   // FP32 slack of the cell walls
};
constexpr int kMaxGrids = 3;        // the query order and two candidate sets
struct GridDesc {                   // grid j's members: every point (bits 0) or mask & bits
    int G;
    uint8_t bits[kMaxGrids];
};
// Scratch of up to kMaxGrids grids over the same n points, C = knn_max_cells(n)
// cells each, counting-sorted into one array (grid j's cell c holds
// sorted[cell_off[j C + c], cell_off[j C + c + 1])).
struct KnnWork {
    uint32_t* zero;                 // acc and count, cleared together (zero_bytes)
    size_t zero_bytes;
    uint32_t* acc;                  // [kMaxGrids][8]: bounding box keys, member count
    uint32_t* count;                // [kMaxGrids * C]
    GridParam* gp;                  // [kMaxGrids]
    uint32_t* cell_off;             // [kMaxGrids * C + 1]
    unsigned long long* span_sum;   // [kMaxGrids * C / 1024 + 2]
    uint32_t* status;               // 4 words
    uint2* slot;                    // [kMaxGrids][n] (cell, rank in cell)
    float4* sorted;                 // [kMaxGrids * n] members by cell: x, y, z, index bits
    // BVH fallback of the candidate sets (skewed point sets): Morton buckets,
    // sorted keys, nodes, parents, refit flags, per-set switch
    uint32_t* bvh_zero;             // bcount, flag, skew, use: cleared together
    size_t bvh_zero_bytes;
    uint32_t* bcount;               // [2 * kMortonBuckets]
    uint32_t* flag;                 // [2][n]
    unsigned long long* skew;       // [2] sum over cells of count^2
    uint32_t* use_bvh;              // [2], then [2] = use_bvh[0] | use_bvh[1]
    uint32_t* boff;                 // [2 * kMortonBuckets + 1]
    unsigned long long* bspan;      // [2 * kMortonBuckets / 1024 + 2]
    uint32_t* bstatus;              // 4 words
    uint2* bslot;                   // [2][n]
    uint64_t* keys;                 // [2n] (Morton code << 32 | index), sorted per bucket
    uint64_t* keys_tmp;             // [2n]
    uint32_t* long_list;            // [2 * kMortonBuckets]
    uint32_t* long_count;           // 1 word
    float4* nodes;                  // [2][n][4]: child boxes (lo0 + child0, hi0, lo1 + child1, hi1)
    int32_t* parent;                // [2][2n]: internal node i at [i], leaf k at [n + k]
    uint32_t* err;                  // the context's device status word (kStatusInternal)
};
constexpr int kMortonBuckets = 1 << 16;
struct RegParams {
    int n, V, k, min_views;
    float min_px, frac;
    const float* moments;           // [V][n][16]
    const uint32_t* status;         // [n] TSP_* bits of the fit
    const float4 *mo0, *q0, *s0;    // before
    const float4 *mo1, *q1, *s1;    // fitted
    uint8_t* mask;                  // [n] member / static bits
    float4 *dpos, *dscale, *drot;   // motion components
    float4 *fpos, *fscale, *frot;   // median-filtered components
    int32_t *nbr_pos, *nbr_cov;     // [n][k]
    float4 *mo_out, *q_out, *s_out;
    uint32_t* flags;
    const float4* qorder;           // [n] Gaussians in cell order (index bits in .w)
};
// Cells of the neighbour grid for n points (an upper bound; the grid itself is
// sized on the device).
uint32_t knn_max_cells(int n);
// For every point, its k nearest members of each candidate set j < ncand
// (mask & bits[j] != 0; ncand 1 or 2; k <= TSP_REG_MAX_K) into nbr0 / nbr1
// [n][k], -1 padded.
cudaError_t launch_knn(const float4* mo, const uint8_t* mask, const uint8_t* bits, int ncand, int n, int k,
                       const KnnWork& kw, int32_t* nbr0, int32_t* nbr1, cudaStream_t st);
// Static flags, neighbours of both components, median filter, propagation and
// the new parameters.
cudaError_t launch_regularize(const RegParams& rp, const KnnWork& kw, cudaStream_t st);

}  // namespace tsp

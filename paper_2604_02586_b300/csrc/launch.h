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
// a2: exclusive scan of the per-tile counts -> tile offsets and the pair count K.
cudaError_t launch_scan(const Work& w, uint32_t NT, cudaStream_t st);
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

}  // namespace tsp

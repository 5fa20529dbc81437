// render.cu -- the colour render (Sec. 3.1) of the Gaussians' splats, for the
// render check and the gradient refinement that follows the relocation.
#include "launch.h"

namespace tsp {

namespace {

constexpr uint32_t kFull = 0xffffffffu;

// Colour render (Sec. 3.1), one 128-thread CTA per tile: warp w walks the tile's
// depth-ordered list for its 8x8 block (w & 1, w >> 1) on its own, lane l owning
// pixels (l & 7, (l >> 3) + 4k), k = 0, 1.  Entries are culled per block as in the
// accumulate walk (an entry whose alpha >= 1/255 ellipse misses every pixel centre
// of the block cannot change any of them), so each pixel sees the same Gaussians in
// the same order with the same arithmetic (render_alpha, render_transmit) as a
// pixel-by-pixel walk of the whole list, which the adjoint recomputes.
struct RenderSmem {
    float4 g0[32];
    float4 g1[32];
    float4 c[32];
};

// TW: tile width, 16 (16 x 16 tiles) or 32 (32 x 8), known at compile time.
template <int TW>
__device__ __forceinline__ void render_block(const ViewSet& vs, const Work& w, const RenderOut& ro, uint32_t tile,
                                             int blk, RenderSmem& sm)
{
    const uint32_t beg = min(w.tile_off[tile], w.cap), end = min(w.tile_off[tile + 1], w.cap);
    int v, tx, ty;
    view_of_tile(vs, tile, v, tx, ty);
    const int lane = threadIdx.x & 31;
    constexpr int TH = kTilePx / TW;
    constexpr int nbx = TW / 8;                // 8x8 blocks per tile row
    const int bxo = (blk % nbx) * 8, byo = (blk / nbx) * 8;
    const int W = vs.cam[v].W, H = vs.cam[v].H;
    const size_t vbase = (size_t)vs.vrec[v];
    const float xc = (float)(bxo + (lane & 7)) + 0.5f;
    float yc[2], T[2], cr[2], cg[2], cb[2];
    bool done[2], inside[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int ly = byo + (lane >> 3) + 4 * k;
        inside[k] = tx * TW + bxo + (lane & 7) < W && ty * TH + ly < H;
        yc[k] = (float)ly + 0.5f;
        T[k] = 1.0f;
        cr[k] = cg[k] = cb[k] = 0.f;
        done[k] = !inside[k];
    }
    // list entries carry the block mask: only the hits load their records
    uint32_t e_next = beg + lane < end ? (uint32_t)w.pairs[beg + lane] : 0u;
    for (uint32_t b0 = beg; b0 < end; b0 += 32) {
        if (!__any_sync(kFull, !done[0] || !done[1])) break;
        const uint32_t e = e_next;
        if (b0 + 32 + lane < end) e_next = (uint32_t)w.pairs[b0 + 32 + lane];
        const bool hit = b0 + lane < end && ((e >> blk) & 1u);
        if (hit) {
            const uint32_t g = entry_gauss(e);
            const float4* rc = w.rec + 4 * (vbase + g);
            sm.g0[lane] = tile_local_packed(rc[kRecGeom0], rc[kRecCorner].x, tx, ty, TW, TH);
            sm.g1[lane] = rc[kRecGeom1];
            sm.c[lane] = w.color[vbase + g];
        }
        uint32_t m = __ballot_sync(kFull, hit);
        __syncwarp();
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const float4 g0 = sm.g0[j], g1 = sm.g1[j];
            // render_alpha and render_transmit for the lane's two pixels in packed
            // FP32x2: each component is the same correctly rounded operation, so
            // the values (and the adjoint's recomputed decisions) are unchanged
            const float ex = __fsub_rn(xc, g0.x);
            const float z1 = __fmul_rn(ex, g0.z);
            const float z1s = __fmul_rn(z1, z1);
            const float2 ey = __fadd2_rn(make_float2(yc[0], yc[1]), make_float2(-g0.y, -g0.y));
            const float2 t = __ffma2_rn(make_float2(-g0.w, -g0.w), make_float2(ex, ex), ey);
            const float2 z2 = __fmul2_rn(t, make_float2(g1.x, g1.x));
            const float2 pw = __ffma2_rn(z2, z2, make_float2(z1s, z1s));
            const float2 oG = __fmul2_rn(make_float2(g1.y, g1.y),
                                         make_float2(sfu_exp2_approx(-pw.x), sfu_exp2_approx(-pw.y)));
            const float2 al = make_float2(fminf(kAlphaMax, oG.x), fminf(kAlphaMax, oG.y));
            const float2 Tp = make_float2(T[0], T[1]);
            const float2 Tn = __fmul2_rn(Tp, __fadd2_rn(make_float2(1.0f, 1.0f), make_float2(-al.x, -al.y)));
            const float2 wp = __fmul2_rn(al, Tp);
            float wk[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float alpha = k ? al.y : al.x, tn = k ? Tn.y : Tn.x;
                const bool pass = !done[k] && alpha >= kAlphaMin;
                const bool term = pass && tn < kTMin;
                const bool blend = pass && !term;
                wk[k] = blend ? (k ? wp.y : wp.x) : 0.f;
                T[k] = blend ? tn : T[k];
                done[k] = done[k] || term;
            }
            const float4 c = sm.c[j];
            const float2 w2 = make_float2(wk[0], wk[1]);
            const float2 r2 = __ffma2_rn(w2, make_float2(c.x, c.x), make_float2(cr[0], cr[1]));
            const float2 g2 = __ffma2_rn(w2, make_float2(c.y, c.y), make_float2(cg[0], cg[1]));
            const float2 b2 = __ffma2_rn(w2, make_float2(c.z, c.z), make_float2(cb[0], cb[1]));
            cr[0] = r2.x; cr[1] = r2.y; cg[0] = g2.x; cg[1] = g2.y; cb[0] = b2.x; cb[1] = b2.y;
        }
        __syncwarp();                                  // staging is rewritten next
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (!inside[k]) continue;
        const size_t pix = (size_t)(ty * TH + byo + (lane >> 3) + 4 * k) * W + (tx * TW + bxo + (lane & 7));
        float* o = ro.rgb[v] + 3 * pix;
        o[0] = cr[k]; o[1] = cg[k]; o[2] = cb[k];
        ro.T[v][pix] = T[k];
    }
}

template <int TW>
__global__ void __launch_bounds__(128) k_raster_render(const ViewSet vs, const Work w, const RenderOut ro)
{
    __shared__ RenderSmem sm[4];
    const int warp = threadIdx.x >> 5;
    render_block<TW>(vs, w, ro, blockIdx.x, warp, sm[warp]);
}

}  // namespace

cudaError_t launch_raster_render(const ViewSet& vs, const Work& w, uint32_t NT, float* const* rgb,
                                 float* const* final_T, cudaStream_t st)
{
    if (NT == 0) return cudaSuccess;
    RenderOut ro;
    for (int v = 0; v < vs.V; ++v) { ro.rgb[v] = rgb[v]; ro.T[v] = final_T[v]; }
    if (vs.tw == 32) k_raster_render<32><<<NT, 128, 0, st>>>(vs, w, ro);
    else k_raster_render<16><<<NT, 128, 0, st>>>(vs, w, ro);
    return cudaGetLastError();
}

}  // namespace tsp

// raster.cu -- a5 raster-accumulate (Sec. 4.3.5).
//
// One CTA per 16x16 tile.  The tile's depth-sorted list is walked in batches of
// kBatch Gaussians whose blend parameters are staged in shared memory together
// with a conservative footprint box.  Each warp owns a block of the tile and
// skips every Gaussian whose box misses it (no pixel there can reach
// alpha = 1/255, so nothing changes).  Each
// pixel blends front to back: alpha = min(0.99, o G(x)), Gaussians with
// alpha < 1/255 are skipped, the walk stops before a Gaussian that would bring
// the transmittance below 1e-4, and w = alpha T (Eq. 4's weight).
//
// Moments: every visible pixel adds 16 values per Gaussian.  The 32 lanes of a
// warp are folded with a transposing butterfly (16 shuffles for 16 values, each
// step exchanges half of the values still held), warps are summed through
// shared memory, and one float4 atomic per 4 values goes to global memory, so a
// (tile, Gaussian) pair costs 4 vector atomics whatever the number of pixels.
// Sums are taken about a per-(view, Gaussian) origin (mu_2D clamped to the image)
// and displacement reference (the track at that origin), which keeps FP32 sums
// free of cancellation; a6 undoes both shifts exactly.
#include <algorithm>

#include "launch.h"

namespace tsp {

namespace {

constexpr int kBatch = 64;
constexpr uint32_t kFull = 0xffffffffu;

// 2^x by the SFU's approximate exponential (flush-to-zero; |rel. error| ~ 2^-22).
// x <= 0 here, and a result below 2^-126 (alpha < 1/255 by far) flushes to 0.
__device__ __forceinline__ float sfu_exp2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// kStats = true is a measurement variant: the same walk, plus exact counts of the
// work done (evaluations, blended contributions, moment additions, list entries).
//
// P pixels per thread: warp w covers the 8 x (4P) block (w & 1, w >> 1) of the
// tile; lane l owns pixels (l & 7, (l >> 3) + 4k), k < P.  Per batch, two ballots
// give each warp the 64-bit set of staged Gaussians whose footprint box touches
// its block; the warp walks only that set, in list order.  A Gaussian's sums over
// the warp's pixels are folded once per (warp, Gaussian) hit.
template <int P, bool kStats>
__global__ void __launch_bounds__(kTilePx / P) k_raster_accumulate(const ViewSet vs, const Work w,
                                                                       uint32_t tile_base)
{
    constexpr int kThreads = kTilePx / P;
    constexpr int kNW = kThreads / 32;
    constexpr int BH = 4 * P;
    __shared__ float4 s_g0[kBatch];
    __shared__ float4 s_g1[kBatch];
    __shared__ float4 s_box[kBatch];
    __shared__ float2 s_ref[kBatch];
    __shared__ uint32_t s_id[kBatch];
    __shared__ uint32_t s_mask[kNW][2];
    __shared__ __align__(16) float s_part[kBatch][kNW][16];

    const uint32_t tile = tile_base + blockIdx.x;
    const uint32_t beg = min(w.tile_off[tile], w.cap), end = min(w.tile_off[tile + 1], w.cap);
    if (beg >= end) return;
    int v, tx, ty;
    view_of_tile(vs, tile, v, tx, ty);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bxo = (warp & 1) * 8, byo = (warp >> 1) * BH;
    const int W = vs.cam[v].W, H = vs.cam[v].H;
    const size_t vbase = (size_t)vs.vrec[v];

    float T[P], ddx[P], ddy[P], yc[P];
    bool done[P], vis[P], stat[P];
    const float xc = (float)(bxo + (lane & 7)) + 0.5f;
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const int ly = byo + (lane >> 3) + 4 * k;
        const int px = tx * kTile + bxo + (lane & 7), py = ty * kTile + ly;
        const bool inside = px < W && py < H;
        yc[k] = (float)ly + 0.5f;
        ddx[k] = 0.f; ddy[k] = 0.f; vis[k] = false;
        if (inside) {
            const size_t pix = (size_t)py * W + px;
            const float2 d = vs.disp[v][pix];
            ddx[k] = d.x; ddy[k] = d.y;
            vis[k] = vs.vis[v][pix] != 0;
        }
        // static pixel test |x' - x| < 1 (Sec. 4.5.2), in FP32 as the tracks are FP32
        stat[k] = __fmaf_rn(ddx[k], ddx[k], __fmul_rn(ddy[k], ddy[k])) < 1.0f;
        T[k] = 1.0f;
        done[k] = !inside;
    }
    const float bx0 = (float)bxo + 0.5f, bx1 = bx0 + 7.0f;
    const float by0 = (float)byo + 0.5f, by1 = by0 + (float)(BH - 1);
    unsigned long long n_eval = 0, n_blend = 0, n_add = 0, n_list = 0;

    for (uint32_t b0 = beg; b0 < end; b0 += kBatch) {
        const int nb = (int)min((uint32_t)kBatch, end - b0);
        if (kStats && tid == 0) n_list += nb;
        if (tid < nb) {
            const uint32_t g = (uint32_t)w.pairs[b0 + tid];
            const float4 g0 = tile_local(w.geom0[vbase + g], w.rect[vbase + g], tx, ty, kTile, kTile);
            const float4 g1 = w.geom1[vbase + g];
            s_id[tid] = g;
            s_g0[tid] = g0;
            s_g1[tid] = g1;
            s_box[tid] = footprint_box(g0, g1);
            s_ref[tid] = w.dref[vbase + g];
        }
        __syncthreads();
        bool alive = false;
#pragma unroll
        for (int k = 0; k < P; ++k) alive |= !done[k];
        uint32_t mlo = 0, mhi = 0;
        if (__any_sync(kFull, alive)) {
            bool h0 = false, h1 = false;
            if (lane < nb) {
                const float4 bb = s_box[lane];
                h0 = bb.x <= bx1 && bb.y >= bx0 && bb.z <= by1 && bb.w >= by0;
            }
            if (lane + 32 < nb) {
                const float4 bb = s_box[lane + 32];
                h1 = bb.x <= bx1 && bb.y >= bx0 && bb.z <= by1 && bb.w >= by0;
            }
            mlo = __ballot_sync(kFull, h0);
            mhi = __ballot_sync(kFull, h1);
        }
        if (lane == 0) { s_mask[warp][0] = mlo; s_mask[warp][1] = mhi; }
        unsigned long long m = ((unsigned long long)mhi << 32) | mlo;
        while (m) {
            const int j = __ffsll((long long)m) - 1;
            m &= m - 1;
            const float4 g0 = s_g0[j];
            const float4 g1 = s_g1[j];
            const float2 rf = s_ref[j];
            float val[16];
            int npix = 0, nstat = 0;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const float ex = xc - g0.x, ey = yc[k] - g0.y;
                float wk = 0.f;
                bool add = false;
                if (!done[k]) {
                    const float z1 = ex * g0.z;
                    const float z2 = fmaf(-g0.w, ex, ey) * g1.x;
                    const float pw = fmaf(z2, z2, z1 * z1);
                    const float alpha = fminf(kAlphaMax, g1.y * exp2f(-pw));
                    if (kStats) ++n_eval;
                    if (alpha >= kAlphaMin) {
                        const float Tn = T[k] * (1.0f - alpha);
                        if (Tn < kTMin) {
                            done[k] = true;
                        } else {
                            if (kStats) ++n_blend;
                            if (vis[k]) {
                                wk = alpha * T[k];
                                add = true;
                                if (kStats) ++n_add;
                            }
                            T[k] = Tn;
                        }
                    }
                }
                // coordinates about the moment origin, displacement about the
                // Gaussian's reference track; wk = 0 where nothing is added
                const float mx = ex - g1.z, my = ey - g1.w;
                const float dx = ddx[k] - rf.x, dy = ddy[k] - rf.y;
                const float wx = wk * mx, wy = wk * my;
                const float ws = stat[k] ? wk : 0.f;
                if (k == 0) {
                    val[0] = wk; val[1] = wx; val[2] = wy;
                    val[3] = wx * mx; val[4] = wx * my; val[5] = wy * my;
                    val[6] = wk * dx; val[7] = wk * dy;
                    val[8] = wx * dx; val[9] = wx * dy;
                    val[10] = wy * dx; val[11] = wy * dy;
                    val[12] = ws;
                } else {
                    val[0] += wk; val[1] += wx; val[2] += wy;
                    val[3] = fmaf(wx, mx, val[3]); val[4] = fmaf(wx, my, val[4]); val[5] = fmaf(wy, my, val[5]);
                    val[6] = fmaf(wk, dx, val[6]); val[7] = fmaf(wk, dy, val[7]);
                    val[8] = fmaf(wx, dx, val[8]); val[9] = fmaf(wx, dy, val[9]);
                    val[10] = fmaf(wy, dx, val[10]); val[11] = fmaf(wy, dy, val[11]);
                    val[12] += ws;
                }
                npix += __popc(__ballot_sync(kFull, add));
                nstat += __popc(__ballot_sync(kFull, add && stat[k]));
            }
            val[13] = 0.f; val[14] = 0.f; val[15] = 0.f;
            float r = 0.f;
            if (npix) r = warp_transpose_sum16(val, lane);      // warp-uniform branch
            if ((lane & 1) == 0)
                s_part[j][warp][lane >> 1] = lane == 26 ? (float)npix : lane == 28 ? (float)nstat : r;
        }
        __syncthreads();
        for (int t = tid; t < nb * 4; t += kThreads) {
            const int j = t >> 2, qd = t & 3;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < kNW; ++k) {
                const uint32_t mk = s_mask[k][j >> 5];
                if (mk & (1u << (j & 31))) {
                    const float4 p = *reinterpret_cast<const float4*>(&s_part[j][k][4 * qd]);
                    acc.x += p.x; acc.y += p.y; acc.z += p.z; acc.w += p.w;
                }
            }
            if (acc.x != 0.f || acc.y != 0.f || acc.z != 0.f || acc.w != 0.f)
                atomicAdd(&w.moments[(vbase + s_id[j]) * 4 + qd], acc);
        }
        bool any_alive = false;
#pragma unroll
        for (int k = 0; k < P; ++k) any_alive |= !done[k];
        if (__syncthreads_count(any_alive) == 0) break;
    }
    if (kStats) {
        atomicAdd(&w.stats[0], n_eval);
        atomicAdd(&w.stats[1], n_blend);
        atomicAdd(&w.stats[2], n_add);
        if (tid == 0) atomicAdd(&w.stats[3], n_list);
    }
}


// Two-phase accumulate (the default).  Warp w owns the 8x8 block (w & 1, w >> 1)
// of the tile, lane l the pixels (l & 7, (l >> 3) + 4h), h = 0, 1, and walks the
// tile's depth-ordered list on its own (no block-wide barrier): 32 entries at a
// time, lane l loads entry l, tests whether its alpha >= 1/255 ellipse meets the
// block, and stages the hits in warp-private shared memory.
//   Phase 1 (blend, pixel-parallel): for each hit, every lane blends its two
//   pixels and writes the weight w = alpha T (0 where nothing is added) into a
//   warp-private buffer, one column per pending hit; hits that add no pixel of
//   the block are dropped.
//   Phase 2 (moments, hit-parallel): once 16 hits are pending, lane l sums the
//   13 weighted moments of hit l & 15 over pixel half l >> 4 (32 pixels) from
//   the buffer, two horizontally adjacent pixels at a time in packed FP32x2
//   arithmetic (each moment as an (even pixel, odd pixel) pair, joined at the
//   end; two passes, position then displacement moments, so the pairs of sums
//   fit the 72 registers of 7 CTAs per SM); the halves are joined with one
//   shuffle per value and lanes 0-15 add the result to global memory with 4
//   float4 atomics.
// Buffer layout: the weights of hit c at the pixel pair p (pixels 2p, 2p + 1)
// of half h are the float2 at h * kWHalf + p * kWRow + 2c.  A row stride of 34
// words makes the phase-1 writes (lane l: pair l >> 1, word l & 1) hit 32
// different banks and the phase-2 reads (lanes = hits) 32 consecutive words.
constexpr int kChunk = 16;
constexpr int kWRow = 2 * kChunk + 2;
constexpr int kWHalf = 16 * kWRow;
constexpr int kWWords = 2 * kWHalf;

// Warp-private shared memory of the two-phase walk.
struct WarpSmem {
    float4 g0[32];
    float4 g1[32];
    float4 hd[32];                 // (origin x, origin y, reference x, reference y)
    uint32_t id[32];
    float W[kWWords];
    float4 D[2][16];               // per half and pixel pair: (d_x, d_x', d_y, d_y')
    float2 S[2][16];               // per half and pixel pair: static flags (0 or 1)
};

// One warp, one 8x8 block `blk` of tile `tile`: the two-phase walk above.  Work
// counts (kStats) accumulate in cnt.
// TW: tile width, 16 (16 x 16 tiles) or 32 (32 x 8); a compile-time value so the
// block and pixel coordinates cost no registers.
template <bool kStats, int TW>
__device__ __forceinline__ void accumulate_block(const ViewSet& vs, const Work& w, uint32_t tile, int blk,
                                                 WarpSmem& sm, unsigned long long (&cnt)[3])
{
    const uint32_t beg = min(w.tile_off[tile], w.cap), end = min(w.tile_off[tile + 1], w.cap);
    if (beg >= end) return;
    int v, tx, ty;
    view_of_tile(vs, tile, v, tx, ty);
    const int lane = threadIdx.x & 31;
    constexpr int TH = kTilePx / TW;
    constexpr int nbx = TW / 8;                // 8x8 blocks per tile row: 2 (16 x 16) or 4 (32 x 8)
    const int bxo = (blk % nbx) * 8, byo = (blk / nbx) * 8;
    const int W = vs.cam[v].W, H = vs.cam[v].H;
    const size_t vbase = (size_t)vs.vrec[v];
    float* const Wb = sm.W;

    // T = 0 marks a pixel that is outside the image or has terminated
    float T[2];
    bool vis[2];
    uint32_t stat_mask[2];
    const float xc = (float)(bxo + (lane & 7)) + 0.5f;
    float yc[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int ly = byo + (lane >> 3) + 4 * k;
        const int px = tx * TW + bxo + (lane & 7), py = ty * TH + ly;
        const bool inside = px < W && py < H;
        float ddx = 0.f, ddy = 0.f;
        vis[k] = false;
        if (inside) {
            const size_t pix = (size_t)py * W + px;
            const float2 d = vs.disp[v][pix];
            ddx = d.x; ddy = d.y;
            vis[k] = vs.vis[v][pix] != 0;
        }
        // static pixel test |x' - x| < 1 (Sec. 4.5.2), in FP32 as the tracks are FP32
        const bool stat = __fmaf_rn(ddx, ddx, __fmul_rn(ddy, ddy)) < 1.0f;
        float* const dp = reinterpret_cast<float*>(&sm.D[k][lane >> 1]);
        dp[lane & 1] = ddx;
        dp[2 + (lane & 1)] = ddy;
        reinterpret_cast<float*>(&sm.S[k][lane >> 1])[lane & 1] = stat ? 1.f : 0.f;
        stat_mask[k] = __ballot_sync(kFull, stat);
        yc[k] = (float)ly + 0.5f;
        T[k] = inside ? 1.0f : 0.0f;
    }
    const float bx0 = (float)bxo + 0.5f, bx1 = bx0 + 7.0f;
    const float by0 = (float)byo + 0.5f, by1 = by0 + 7.0f;
    if (kStats && blk == 0 && lane == 0) atomicAdd(&w.stats[3], (unsigned long long)(end - beg));

    // pending hit c is held by lane c: moment record, origin and reference, and the
    // masks of the pixels it added (rows 0-3, 4-7)
    int pend = 0;
    uint32_t h_id = 0, h_m0 = 0, h_m1 = 0;
    float4 h_hd = make_float4(0.f, 0.f, 0.f, 0.f);

    auto phase2 = [&](int npend) {
        __syncwarp();
        const int c = lane & 15, half = lane >> 4;
        const float ox = __shfl_sync(kFull, h_hd.x, c), oy = __shfl_sync(kFull, h_hd.y, c);
        const float rx = __shfl_sync(kFull, h_hd.z, c), ry = __shfl_sync(kFull, h_hd.w, c);
        const float x0 = ((float)bxo + 0.5f) - ox;
        const float y0 = ((float)(byo + 4 * half) + 0.5f) - oy;
        // every moment as an (even pixel, odd pixel) pair: a[q] sums moment q
        // over the pixels 2p and 2p + 1 of every pair p; two passes over the
        // pairs (the position moments, then the displacement moments)
        const float2 z = make_float2(0.f, 0.f);
        float2 a0 = z, a1 = z, a2 = z, a3 = z, a4 = z, a5 = z, a6 = z, a7 = z, a8 = z, a9 = z, a10 = z,
               a11 = z, a12 = z;
        const float* Wh = Wb + half * kWHalf + 2 * c;
        const float4* Dh = sm.D[half];
        const float2* Sh = sm.S[half];
#pragma unroll
        for (int p = 0; p < 16; ++p) {
            const float2 w2 = *reinterpret_cast<const float2*>(Wh + p * kWRow);
            const float2 st2 = Sh[p];
            const int col = 2 * (p & 3);
            const float2 X = make_float2(x0 + (float)col, x0 + (float)(col + 1));
            const float yv = y0 + (float)(p >> 2);
            const float2 Y = make_float2(yv, yv);
            const float2 wX = __fmul2_rn(w2, X), wY = __fmul2_rn(w2, Y);
            a0 = __fadd2_rn(a0, w2);
            a1 = __fadd2_rn(a1, wX);
            a2 = __fadd2_rn(a2, wY);
            a3 = __ffma2_rn(wX, X, a3);
            a4 = __ffma2_rn(wX, Y, a4);
            a5 = __ffma2_rn(wY, Y, a5);
            a12 = __ffma2_rn(w2, st2, a12);
        }
        const float2 nrx = make_float2(-rx, -rx), nry = make_float2(-ry, -ry);
#pragma unroll
        for (int p = 0; p < 16; ++p) {
            const float2 w2 = *reinterpret_cast<const float2*>(Wh + p * kWRow);
            const float4 dd = Dh[p];
            const int col = 2 * (p & 3);
            const float2 X = make_float2(x0 + (float)col, x0 + (float)(col + 1));
            const float yv = y0 + (float)(p >> 2);
            const float2 Y = make_float2(yv, yv);
            const float2 dX = __fadd2_rn(make_float2(dd.x, dd.y), nrx);
            const float2 dY = __fadd2_rn(make_float2(dd.z, dd.w), nry);
            const float2 wX = __fmul2_rn(w2, X), wY = __fmul2_rn(w2, Y);
            a6 = __ffma2_rn(w2, dX, a6);
            a7 = __ffma2_rn(w2, dY, a7);
            a8 = __ffma2_rn(wX, dX, a8);
            a9 = __ffma2_rn(wX, dY, a9);
            a10 = __ffma2_rn(wY, dX, a10);
            a11 = __ffma2_rn(wY, dY, a11);
        }
        float s[13] = {a0.x + a0.y, a1.x + a1.y, a2.x + a2.y, a3.x + a3.y, a4.x + a4.y,
                       a5.x + a5.y, a6.x + a6.y, a7.x + a7.y, a8.x + a8.y, a9.x + a9.y,
                       a10.x + a10.y, a11.x + a11.y, a12.x + a12.y};
#pragma unroll
        for (int q = 0; q < 13; ++q) s[q] += __shfl_down_sync(kFull, s[q], 16);
        if (lane < npend) {
            const float h_np = (float)(__popc(h_m0) + __popc(h_m1));
            const float h_ns = (float)(__popc(h_m0 & stat_mask[0]) + __popc(h_m1 & stat_mask[1]));
            float4* dst = &w.moments[(vbase + h_id) * 4];
            atomicAdd(dst + 0, make_float4(s[0], s[1], s[2], s[3]));
            atomicAdd(dst + 1, make_float4(s[4], s[5], s[6], s[7]));
            atomicAdd(dst + 2, make_float4(s[8], s[9], s[10], s[11]));
            atomicAdd(dst + 3, make_float4(s[12], h_np, h_ns, 0.f));
        }
        __syncwarp();
    };

    uint32_t g_next = beg + lane < end ? (uint32_t)w.pairs[beg + lane] : 0u;
    for (uint32_t b0 = beg; b0 < end; b0 += 32) {
        if (!__any_sync(kFull, T[0] > 0.f || T[1] > 0.f)) break;
        bool hit = false;
        const uint32_t g = g_next;
        if (b0 + 32 + lane < end) g_next = (uint32_t)w.pairs[b0 + 32 + lane];
        if (b0 + lane < end) {
            const float4 g0 = tile_local(w.geom0[vbase + g], w.rect[vbase + g], tx, ty, TW, TH);
            const float4 g1 = w.geom1[vbase + g];
            const float4 bb = footprint_box(g0, g1);
            hit = bb.x <= bx1 && bb.y >= bx0 && bb.z <= by1 && bb.w >= by0;
            if (hit)
                hit = block_min_power(g0, g1.x, bx0, bx1, by0, by1) <=
                      log2f(255.0f * g1.y) * 1.002f + 1e-4f;
            if (hit) {
                const float2 rf = w.dref[vbase + g];
                sm.g0[lane] = g0;
                sm.g1[lane] = g1;
                sm.hd[lane] = make_float4(g0.x + g1.z, g0.y + g1.w, rf.x, rf.y);
                sm.id[lane] = g;
            }
        }
        uint32_t m = __ballot_sync(kFull, hit);
        __syncwarp();
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const float4 g0 = sm.g0[j];
            const float4 g1 = sm.g1[j];
            // both pixels of a lane share the column: ex, z1; the second row is 4 below
            const float ex = xc - g0.x;
            const float z1 = ex * g0.z;
            const float z1s = z1 * z1;
            float z2[2];
            z2[0] = fmaf(-g0.w, ex, yc[0] - g0.y) * g1.x;
            z2[1] = fmaf(4.0f, g1.x, z2[0]);
            // the lane's two pixels in packed FP32x2 where the operation is shared
            const float2 z2p = make_float2(z2[0], z2[1]);
            const float2 pw = __ffma2_rn(z2p, z2p, make_float2(z1s, z1s));
            const float2 oe = __fmul2_rn(make_float2(g1.y, g1.y), make_float2(sfu_exp2(-pw.x), sfu_exp2(-pw.y)));
            const float2 al = make_float2(fminf(kAlphaMax, oe.x), fminf(kAlphaMax, oe.y));
            const float2 Tp = make_float2(T[0], T[1]);
            const float2 Tn = __fmul2_rn(Tp, __fadd2_rn(make_float2(1.0f, 1.0f), make_float2(-al.x, -al.y)));
            const float2 wa = __fmul2_rn(al, Tp);
            bool add[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float alpha = k ? al.y : al.x, tn = k ? Tn.y : Tn.x;
                const bool pass = alpha >= kAlphaMin;
                const bool blend = pass && tn >= kTMin;    // T = 0: Tn = 0, never blends
                add[k] = blend && vis[k];
                Wb[k * kWHalf + (lane >> 1) * kWRow + 2 * pend + (lane & 1)] = add[k] ? (k ? wa.y : wa.x) : 0.f;
                if (kStats) { cnt[0] += T[k] > 0.f; cnt[1] += blend; cnt[2] += add[k]; }
                T[k] = blend ? tn : (pass ? 0.f : T[k]);   // pass without blend: terminated
            }
            const uint32_t a0 = __ballot_sync(kFull, add[0]), a1 = __ballot_sync(kFull, add[1]);
            if ((a0 | a1) == 0u) continue;             // nothing of this block to add
            if (lane == pend) {
                h_id = sm.id[j];
                h_hd = sm.hd[j];
                h_m0 = a0;
                h_m1 = a1;
            }
            if (++pend == kChunk) {
                phase2(kChunk);
                pend = 0;
            }
        }
        __syncwarp();                                  // staging is rewritten next
    }
    if (pend) phase2(pend);
}

// Grid form: one CTA per tile, warp w takes block w.
template <bool kStats, int TW>
__global__ void __launch_bounds__(128, 7) k_raster_accumulate_2p(const ViewSet vs, const Work w,
                                                                          uint32_t tile_base)
{
    __shared__ WarpSmem sm[4];
    const int warp = threadIdx.x >> 5;
    unsigned long long cnt[3] = {0ull, 0ull, 0ull};
    accumulate_block<kStats, TW>(vs, w, tile_base + blockIdx.x, warp, sm[warp], cnt);
    if (kStats) {
        atomicAdd(&w.stats[0], cnt[0]);
        atomicAdd(&w.stats[1], cnt[1]);
        atomicAdd(&w.stats[2], cnt[2]);
    }
}

// Persistent form: a grid sized to the resident CTAs, each warp taking
// (tile, block) items from a device-side queue (one atomic per item, ascending
// tile order) until none are left.  Warps never wait for one another and no
// CTA is launched per tile.
template <bool kStats, int TW>
__global__ void __launch_bounds__(128, 7) k_raster_accumulate_2p_persistent(const ViewSet vs, const Work w,
                                                                                     uint32_t tile_base,
                                                                                     uint32_t ntiles,
                                                                                     uint32_t* queue)
{
    __shared__ WarpSmem sm[4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long cnt[3] = {0ull, 0ull, 0ull};
    const uint32_t items = 4u * ntiles;
    for (;;) {
        uint32_t item = 0u;
        if (lane == 0) item = atomicAdd(queue, 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= items) break;
        accumulate_block<kStats, TW>(vs, w, tile_base + (item >> 2), (int)(item & 3u), sm[warp], cnt);
    }
    if (kStats) {
        atomicAdd(&w.stats[0], cnt[0]);
        atomicAdd(&w.stats[1], cnt[1]);
        atomicAdd(&w.stats[2], cnt[2]);
    }
}

template <bool kStats, int TW>
void launch_2p(const ViewSet& vs, const Work& w, uint32_t tb, uint32_t NT, bool persistent, int resident_ctas,
               cudaStream_t st)
{
    if (!persistent) {
        k_raster_accumulate_2p<kStats, TW><<<NT, 128, 0, st>>>(vs, w, tb);
    } else {
        const uint32_t grid = (uint32_t)std::max<long long>(1, std::min<long long>(resident_ctas, (long long)NT));
        k_raster_accumulate_2p_persistent<kStats, TW><<<grid, 128, 0, st>>>(vs, w, tb, NT, w.queue);
    }
}

}  // namespace

cudaError_t raster_prepare()
{
    // up to seven 27 KB CTAs per SM need the largest shared-memory carveout; set
    // once per context, outside any stream capture
    const void* kerns[] = {(const void*)k_raster_accumulate_2p<false, 16>, (const void*)k_raster_accumulate_2p<true, 16>,
                           (const void*)k_raster_accumulate_2p_persistent<false, 16>,
                           (const void*)k_raster_accumulate_2p_persistent<true, 16>,
                           (const void*)k_raster_accumulate_2p<false, 32>, (const void*)k_raster_accumulate_2p<true, 32>,
                           (const void*)k_raster_accumulate_2p_persistent<false, 32>,
                           (const void*)k_raster_accumulate_2p_persistent<true, 32>};
    for (const void* k : kerns) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                                   (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_raster_accumulate(const ViewSet& vs, const Work& w, uint32_t tile_base, uint32_t ntiles,
                                     bool stats, int variant, int resident_ctas, cudaStream_t st)
{
    if (ntiles == 0 || vs.nmax == 0) return cudaSuccess;
    const uint32_t NT = ntiles, tb = tile_base;
    if (variant == 0 || variant == 5) {
        if (variant == 5) {
            const cudaError_t e = cudaMemsetAsync(w.queue, 0, sizeof(uint32_t), st);
            if (e != cudaSuccess) return e;
        }
        const bool pers = variant == 5;
        if (vs.tw == 32) {
            if (stats) launch_2p<true, 32>(vs, w, tb, NT, pers, resident_ctas, st);
            else launch_2p<false, 32>(vs, w, tb, NT, pers, resident_ctas, st);
        } else {
            if (stats) launch_2p<true, 16>(vs, w, tb, NT, pers, resident_ctas, st);
            else launch_2p<false, 16>(vs, w, tb, NT, pers, resident_ctas, st);
        }
    } else if (vs.tw != kTile || vs.th != kTile) {
        return cudaErrorInvalidValue;           // the warp-shuffle kernels tile 16 x 16 only
    } else if (variant == 1) {
        if (stats) k_raster_accumulate<1, true><<<NT, kTilePx, 0, st>>>(vs, w, tb);
        else k_raster_accumulate<1, false><<<NT, kTilePx, 0, st>>>(vs, w, tb);
    } else if (variant == 4) {
        if (stats) k_raster_accumulate<4, true><<<NT, kTilePx / 4, 0, st>>>(vs, w, tb);
        else k_raster_accumulate<4, false><<<NT, kTilePx / 4, 0, st>>>(vs, w, tb);
    } else {
        if (stats) k_raster_accumulate<2, true><<<NT, kTilePx / 2, 0, st>>>(vs, w, tb);
        else k_raster_accumulate<2, false><<<NT, kTilePx / 2, 0, st>>>(vs, w, tb);
    }
    return cudaGetLastError();
}

int raster_resident_ctas(int device)
{
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_accumulate_2p_persistent<false, 16>, 128, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return 148 * 4;
    }
    return std::max(1, sms * std::max(1, per_sm));
}


}  // namespace tsp

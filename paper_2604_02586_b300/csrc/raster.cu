// raster.cu -- a5 raster-accumulate (Sec. 4.3.5).
//
// Every pixel blends its tile's depth-sorted list front to back:
// alpha = min(0.99, o G(x)), Gaussians with alpha < 1/255 are skipped, the walk
// stops before a Gaussian that would bring the transmittance below 1e-4, and
// each visible pixel adds w = alpha T (Eq. 4's weight) times its moment terms to
// the Gaussian's (view, Gaussian) record: 13 sums and two pixel counts.  Sums
// are taken about a per-(view, Gaussian) origin (mu_2D clamped to the image) and
// displacement reference (the track at that origin), which keeps FP32 sums free
// of cancellation; a6 undoes both shifts exactly.
//
// The default kernel, k_raster_accumulate_2p (and its persistent form), runs
// one warp per 8x8 block of a tile in two phases: a branch-free pixel-parallel
// blend that writes each pending hit's weights into a warp-private buffer, then
// a hit-parallel pass that sums 16 hits' moments in packed FP32x2 and adds them
// with four float4 atomics per hit (see accumulate_block).  The tile-per-CTA
// warp-shuffle kernels k_raster_accumulate<P> (8x4, 8x8, 8x16 warp blocks) are
// the autotuner's alternatives: they fold each hit's 16 values across the warp
// with a transposing butterfly instead of a weight buffer.
#include <algorithm>

#include "launch.h"

namespace tsp {

namespace {

constexpr int kBatch = 64;
constexpr uint32_t kFull = 0xffffffffu;
constexpr float kLog2_255 = 7.99435329f;   // log2(255): alpha >= 1/255 <=> power - log2 o <= this

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
    if (beg >= end || gate_closed(w)) return;
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
            const uint32_t g = entry_gauss((uint32_t)w.pairs[b0 + tid]);
            const float4* rc = w.rec + 4 * (vbase + g);
            const float4 c3 = rc[kRecCorner];
            const float4 g0 = tile_local_packed(rc[kRecGeom0], c3.x, tx, ty, kTile, kTile);
            const float4 g1 = rc[kRecGeom1];
            s_id[tid] = g;
            s_g0[tid] = g0;
            s_g1[tid] = g1;
            s_box[tid] = footprint_box(g0, g1);
            s_ref[tid] = make_float2(c3.z, c3.w);
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
// time, lane l takes entry l (copied into its shared slot by cp.async during the
// step before) and tests the entry's bit for the block (whether its alpha >= 1/255
// ellipse meets the block).  The hits of the step are compacted into warp-private
// staging in list order (their blend factors) and numbered on from the pending
// ones; each hit's moment origin,
// reference track and Gaussian index go to a ring indexed by hit number, where
// they stay until the hit's moments are added.
//   Phase 1 (blend, pixel-parallel): for each hit in order, every lane blends its
//   two pixels and writes w = alpha T (0 where nothing is added) into column
//   `pend` of a warp-private buffer; lane `pend` keeps the ballots of the pixels
//   the hit added.  The loop has no divergent branch: alpha below 1/255 becomes
//   alpha' = 0 (T (1 - 0) = T exactly), and the transmittance test both ends a
//   terminated pixel (T = 0) and zeroes its weight.
//   Phase 2 (moments, hit-parallel): once 16 hits are pending, lane l sums the
//   13 weighted moments of hit l & 15 over pixel half l >> 4 (32 pixels) from
//   the buffer, two horizontally adjacent pixels at a time in packed FP32x2
//   arithmetic (each moment as an (even pixel, odd pixel) pair, joined at the
//   end; two passes, position then displacement moments, so the pairs of sums
//   fit the 72 registers of 7 CTAs per SM); the halves are joined with one
//   shuffle per value and lanes 0-15 add the result to global memory with 4
//   float4 atomics (none for a hit that added no pixel).
// Buffer layout: the weights of hit c at the pixel pair p (pixels 2p, 2p + 1)
// of half h are the float2 at h * kWHalf + p * kWRow + 2c.  A row stride of 34
// words makes the phase-1 writes (lane l: pair l >> 1, word l & 1) hit 32
// different banks and the phase-2 reads (lanes = hits) 32 consecutive words.
constexpr int kChunk = 16;
constexpr int kWRow = 2 * kChunk + 2;
constexpr int kWHalf = 16 * kWRow;
constexpr int kWWords = 2 * kWHalf;
// hits whose moments are pending (< kChunk) plus one walk step's hits (<= 32)
constexpr int kRing = 48;

// Warp-private shared memory of the two-phase walk.
struct WarpSmem {
    float4 g0[32];                 // this step's hits: mean (tile-local), i11, k
    float2 g1[32];                 // this step's hits: i22, log2(opacity)
    float4 hd[kRing];              // by hit number: (origin x, origin y, reference x, reference y)
    uint32_t id[kRing];            // by hit number: Gaussian index
    float W[kWWords];
    float4 D[2][16];               // per half and pixel pair: (d_x, d_x', d_y, d_y')
    float2 S[2][16];               // per half and pixel pair: static flags (0 or 1)
    uint32_t enext[32];            // per lane: the next walk step's list entry (low word)
};

// One warp, one 8x8 block `blk` of tile `tile`: the two-phase walk above.  Work
// counts (kStats) accumulate in cnt: [0] (pixel, Gaussian) evaluations, [1]
// blended contributions, [2] moment additions, [3] block hits (list entries
// whose ellipse meets the block), [4] hits that add a pixel, [5] phase-2 passes,
// [6] 32-entry walk steps.
// TW: tile width, 16 (16 x 16 tiles) or 32 (32 x 8); a compile-time value so the
// block and pixel coordinates cost no registers.
template <bool kStats, int TW>
__device__ __forceinline__ void accumulate_block(const ViewSet& vs, const Work& w, uint32_t tile, int blk,
                                                 WarpSmem& sm, unsigned long long (&cnt)[7])
{
    const uint32_t beg = min(w.tile_off[tile], w.cap), end = min(w.tile_off[tile + 1], w.cap);
    if (beg >= end || gate_closed(w)) return;
    int v, tx, ty;
    view_of_tile(vs, tile, v, tx, ty);
    const int lane = threadIdx.x & 31;
    constexpr int TH = kTilePx / TW;
    constexpr int nbx = TW / 8;                // 8x8 blocks per tile row: 2 (16 x 16) or 4 (32 x 8)
    const int bxo = (blk % nbx) * 8, byo = (blk / nbx) * 8;
    const int W = vs.cam[v].W, H = vs.cam[v].H;
    const size_t vbase = (size_t)vs.vrec[v];
    float* const Wb = sm.W + (lane >> 1) * kWRow + (lane & 1);

    // the lane's two pixels as pairs: transmittance (0 = outside the image or
    // terminated) and visibility (1 or 0)
    float2 T2 = make_float2(0.f, 0.f), vis2 = make_float2(0.f, 0.f);
    uint32_t stat_mask[2];
    const float xc = (float)(bxo + (lane & 7)) + 0.5f;
    const float yc0 = (float)(byo + (lane >> 3)) + 0.5f;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int ly = byo + (lane >> 3) + 4 * k;
        const int px = tx * TW + bxo + (lane & 7), py = ty * TH + ly;
        const bool inside = px < W && py < H;
        float ddx = 0.f, ddy = 0.f, vis = 0.f;
        if (inside) {
            const size_t pix = (size_t)py * W + px;
            const float2 d = vs.disp[v][pix];
            ddx = d.x; ddy = d.y;
            vis = vs.vis[v][pix] != 0 ? 1.f : 0.f;
        }
        // static pixel test |x' - x| < 1 (Sec. 4.5.2), in FP32 as the tracks are FP32
        const bool stat = __fmaf_rn(ddx, ddx, __fmul_rn(ddy, ddy)) < 1.0f;
        float* const dp = reinterpret_cast<float*>(&sm.D[k][lane >> 1]);
        dp[lane & 1] = ddx;
        dp[2 + (lane & 1)] = ddy;
        reinterpret_cast<float*>(&sm.S[k][lane >> 1])[lane & 1] = stat ? 1.f : 0.f;
        stat_mask[k] = __ballot_sync(kFull, stat);
        if (k == 0) { T2.x = inside ? 1.f : 0.f; vis2.x = vis; }
        else { T2.y = inside ? 1.f : 0.f; vis2.y = vis; }
    }
    if (kStats && blk == 0 && lane == 0) atomicAdd(&w.stats[3], (unsigned long long)(end - beg));

    int pend = 0, q0 = 0;                      // pending count and first pending hit number (mod kRing)
    uint32_t h_m0 = 0, h_m1 = 0;

    auto phase2 = [&](int npend) {
        if (kStats && lane == 0) cnt[5] += 1;
        __syncwarp();
        const int c = lane & 15, half = lane >> 4;
        int slot = q0 + c;
        slot = slot >= kRing ? slot - kRing : slot;
        const float4 hd = sm.hd[slot];         // lanes c >= npend read a stale entry and store nothing
        const float x0 = ((float)bxo + 0.5f) - hd.x;
        const float y0 = ((float)(byo + 4 * half) + 0.5f) - hd.y;
        // every moment as an (even pixel, odd pixel) pair: a[q] sums moment q
        // over the pixels 2p and 2p + 1 of every pair p; two passes over the
        // pairs (the position moments, then the displacement moments).  y~ is
        // constant along a row of 4 pairs, so the moments with a y~ factor are
        // formed per row from that row's sums: sum w y~ = sum_rows y~ (sum_row w).
        // (the first row and pair assign instead of adding to zero)
        float2 a0, a1, a2, a3, a4, a5, a6, a7, a8, a9, a10, a11, a12;
        const float* Wh = sm.W + half * kWHalf + 2 * c;
        const float4* Dh = sm.D[half];
        const float2* Sh = sm.S[half];
#pragma unroll
        for (int row = 0; row < 4; ++row) {
            float2 rw, rwx;
#pragma unroll
            for (int cp = 0; cp < 4; ++cp) {
                const int p = 4 * row + cp;
                const float2 w2 = *reinterpret_cast<const float2*>(Wh + p * kWRow);
                const float2 st2 = Sh[p];
                const float2 X = make_float2(x0 + (float)(2 * cp), x0 + (float)(2 * cp + 1));
                const float2 wX = __fmul2_rn(w2, X);
                if (cp == 0) {
                    rw = w2;
                    rwx = wX;
                } else {
                    rw = __fadd2_rn(rw, w2);
                    rwx = __fadd2_rn(rwx, wX);
                }
                if (p == 0) {
                    a3 = __fmul2_rn(wX, X);
                    a12 = __fmul2_rn(w2, st2);
                } else {
                    a3 = __ffma2_rn(wX, X, a3);
                    a12 = __ffma2_rn(w2, st2, a12);
                }
            }
            const float yv = y0 + (float)row;
            const float2 Y = make_float2(yv, yv);
            const float2 rwy = __fmul2_rn(rw, Y);
            if (row == 0) {
                a0 = rw;
                a1 = rwx;
                a2 = rwy;
                a4 = __fmul2_rn(rwx, Y);
                a5 = __fmul2_rn(rwy, Y);
            } else {
                a0 = __fadd2_rn(a0, rw);
                a1 = __fadd2_rn(a1, rwx);
                a2 = __fadd2_rn(a2, rwy);
                a4 = __ffma2_rn(rwx, Y, a4);
                a5 = __ffma2_rn(rwy, Y, a5);
            }
        }
        const float2 nrx = make_float2(-hd.z, -hd.z), nry = make_float2(-hd.w, -hd.w);
#pragma unroll
        for (int row = 0; row < 4; ++row) {
            float2 rdx, rdy;
#pragma unroll
            for (int cp = 0; cp < 4; ++cp) {
                const int p = 4 * row + cp;
                const float2 w2 = *reinterpret_cast<const float2*>(Wh + p * kWRow);
                const float4 dd = Dh[p];
                const float2 X = make_float2(x0 + (float)(2 * cp), x0 + (float)(2 * cp + 1));
                const float2 wdx = __fmul2_rn(w2, __fadd2_rn(make_float2(dd.x, dd.y), nrx));
                const float2 wdy = __fmul2_rn(w2, __fadd2_rn(make_float2(dd.z, dd.w), nry));
                if (cp == 0) {
                    rdx = wdx;
                    rdy = wdy;
                } else {
                    rdx = __fadd2_rn(rdx, wdx);
                    rdy = __fadd2_rn(rdy, wdy);
                }
                if (p == 0) {
                    a8 = __fmul2_rn(X, wdx);
                    a9 = __fmul2_rn(X, wdy);
                } else {
                    a8 = __ffma2_rn(X, wdx, a8);
                    a9 = __ffma2_rn(X, wdy, a9);
                }
            }
            const float yv = y0 + (float)row;
            const float2 Y = make_float2(yv, yv);
            if (row == 0) {
                a6 = rdx;
                a7 = rdy;
                a10 = __fmul2_rn(rdx, Y);
                a11 = __fmul2_rn(rdy, Y);
            } else {
                a6 = __fadd2_rn(a6, rdx);
                a7 = __fadd2_rn(a7, rdy);
                a10 = __ffma2_rn(rdx, Y, a10);
                a11 = __ffma2_rn(rdy, Y, a11);
            }
        }
        // the buffer holds -w: negate while joining the pair halves
        float s[13] = {-a0.x - a0.y, -a1.x - a1.y, -a2.x - a2.y, -a3.x - a3.y, -a4.x - a4.y,
                       -a5.x - a5.y, -a6.x - a6.y, -a7.x - a7.y, -a8.x - a8.y, -a9.x - a9.y,
                       -a10.x - a10.y, -a11.x - a11.y, -a12.x - a12.y};
#pragma unroll
        for (int q = 0; q < 13; ++q) s[q] += __shfl_down_sync(kFull, s[q], 16);
        const uint2 hm = make_uint2(h_m0, h_m1);
        const int np = __popc(hm.x) + __popc(hm.y);
        if (lane < npend && np > 0) {
            const float h_ns = (float)(__popc(hm.x & stat_mask[0]) + __popc(hm.y & stat_mask[1]));
            float4* dst = &w.moments[(vbase + sm.id[slot]) * 4];
            atomicAdd(dst + 0, make_float4(s[0], s[1], s[2], s[3]));
            atomicAdd(dst + 1, make_float4(s[4], s[5], s[6], s[7]));
            atomicAdd(dst + 2, make_float4(s[8], s[9], s[10], s[11]));
            atomicAdd(dst + 3, make_float4(s[12], (float)np, h_ns, 0.f));
        }
        __syncwarp();
        q0 += npend;
        q0 = q0 >= kRing ? q0 - kRing : q0;
    };

    // list entries carry the block mask (bit blk: the entry's ellipse may meet
    // this block); only the hits load their records.  Each lane's entry of the
    // next walk step is copied into its shared slot (cp.async) while this step
    // runs, so that no register holds it through the step's moment passes.
    const uint32_t e_slot = (uint32_t)__cvta_generic_to_shared(&sm.enext[lane]);
    if (beg + lane < end)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(e_slot), "l"(&w.pairs[beg + lane]) : "memory");
    for (uint32_t b0 = beg; b0 < end; b0 += 32) {
        if (!__any_sync(kFull, T2.x > 0.f || T2.y > 0.f)) break;
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        const uint32_t e = sm.enext[lane];        // the low word: Gaussian << 4 | block mask
        if (b0 + 32 + lane < end)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(e_slot), "l"(&w.pairs[b0 + 32 + lane])
                         : "memory");
        const uint32_t g = entry_gauss(e);
        bool hit = b0 + lane < end && ((e >> blk) & 1u);
        if (hit && w.checked && !index_ok(g, (uint32_t)vs.vn[v])) {
            check_failed(w.dstatus, kSiteListEntry);
            hit = false;
        }
        const uint32_t m = __ballot_sync(kFull, hit);
        if (kStats && lane == 0) cnt[6] += 1;
        if (m == 0u) continue;
        const int nh = __popc(m);
        if (hit) {
            const float4* rc = w.rec + 4 * (vbase + g);
            const float4 c3 = rc[kRecCorner];
            const float4 g0 = tile_local_packed(rc[kRecGeom0], c3.x, tx, ty, TW, TH);
            const float4 g1 = rc[kRecGeom1];
            // staged in list order: the hit's rank among this step's hits
            const int r = __popc(m & ((1u << lane) - 1u));
            // hits are numbered on from the pending ones: q0 + pend + r < 2 kRing
            int slot = q0 + pend + r;
            slot = slot >= kRing ? slot - kRing : slot;
            sm.g0[r] = g0;
            // log2(opacity), so that alpha = 2^(log2 o - power)
            sm.g1[r] = make_float2(g1.x, c3.y);
            sm.hd[slot] = make_float4(g0.x + g1.z, g0.y + g1.w, c3.z, c3.w);
            sm.id[slot] = g;
        }
        if (kStats && lane == 0) cnt[3] += nh;
        __syncwarp();
        // phase 1 in runs that end where the pending columns fill up
        for (int i = 0; i < nh;) {
            const int take = min(nh - i, kChunk - pend);
            // unrolled by 4: a hit's transmittance-free part (power, exponential)
            // overlaps the previous hit's blend
#pragma unroll 4
            for (int j = 0; j < take; ++j) {
                const int col = pend + j;
                const float4 h0 = sm.g0[i + j];
                const float2 h1 = sm.g1[i + j];
                // both pixels of a lane share the column: ex, z1; the second row is 4 below
                const float ex = xc - h0.x;
                const float z1 = ex * h0.z;
                const float base = fmaf(z1, z1, -h1.y);          // z1^2 - log2 o
                const float z20 = fmaf(-h0.w, ex, yc0 - h0.y) * h1.x;
                const float2 z2 = make_float2(z20, fmaf(4.0f, h1.x, z20));
                const float2 q = __ffma2_rn(z2, z2, make_float2(base, base));   // power - log2 o
                // alpha = min(0.99, 2^-q) >= 1/255  <=>  q <= log2 255.  The tests
                // yield 1.0 / 0.0 factors, so that the selections run as packed
                // multiplications on the FMA pipe (the compare-and-select pipe is
                // the busier one)
                const float2 pf = make_float2(q.x <= kLog2_255 ? 1.f : 0.f, q.y <= kLog2_255 ? 1.f : 0.f);
                const float e0 = sfu_exp2(-q.x), e1 = sfu_exp2(-q.y);
                // -alpha' with alpha' = alpha where it passes, else 0 (T is then kept exactly)
                const float2 nap = __fmul2_rn(make_float2(fmaxf(-kAlphaMax, -e0), fmaxf(-kAlphaMax, -e1)), pf);
                const float2 Tn = __ffma2_rn(nap, T2, T2);             // T - alpha' T
                const float2 wv = __fmul2_rn(nap, __fmul2_rn(T2, vis2)); // -alpha' T (0 where not visible)
                // T (1 - alpha') < 1e-4: terminated (T = 0 stays 0); its weight and
                // every later one are 0
                const float2 bf = make_float2(Tn.x >= kTMin ? 1.f : 0.f, Tn.y >= kTMin ? 1.f : 0.f);
                if (kStats) {
                    cnt[0] += (T2.x > 0.f) + (T2.y > 0.f);
                    cnt[1] += (bf.x > 0.f && pf.x > 0.f && T2.x > 0.f) + (bf.y > 0.f && pf.y > 0.f && T2.y > 0.f);
                }
                T2 = __fmul2_rn(Tn, bf);
                const float2 wb = __fmul2_rn(wv, bf);
                const float w0 = wb.x, w1 = wb.y;
                Wb[2 * col] = w0;                  // the buffer holds -w
                Wb[kWHalf + 2 * col] = w1;
                const uint32_t m0 = __ballot_sync(kFull, w0 < 0.f), m1 = __ballot_sync(kFull, w1 < 0.f);
                h_m0 = lane == col ? m0 : h_m0;
                h_m1 = lane == col ? m1 : h_m1;
                if (kStats) {
                    cnt[2] += (w0 < 0.f) + (w1 < 0.f);
                    if (lane == 0 && (m0 | m1)) cnt[4] += 1;
                }
            }
            i += take;
            pend += take;
            if (pend == kChunk) {
                phase2(kChunk);
                pend = 0;
            }
        }
        __syncwarp();                                  // staging is rewritten next
    }
    if (pend) phase2(pend);
    asm volatile("cp.async.wait_all;\n" ::: "memory");   // a copy still in flight after an early end
}

// Work counts of one warp into the context's counters (stats[3], the list
// entries, is counted by the walk itself).
__device__ __forceinline__ void add_stats(const Work& w, const unsigned long long (&cnt)[7])
{
    atomicAdd(&w.stats[0], cnt[0]);
    atomicAdd(&w.stats[1], cnt[1]);
    atomicAdd(&w.stats[2], cnt[2]);
#pragma unroll
    for (int k = 3; k < 7; ++k)
        if (cnt[k]) atomicAdd(&w.stats[k + 1], cnt[k]);
}

// Grid form: one CTA per tile, warp w takes block w.
template <bool kStats, int TW>
__global__ void __launch_bounds__(128, 7) k_raster_accumulate_2p(const ViewSet vs, const Work w,
                                                                          uint32_t tile_base)
{
    __shared__ WarpSmem sm[4];
    const int warp = threadIdx.x >> 5;
    unsigned long long cnt[7] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
    accumulate_block<kStats, TW>(vs, w, tile_base + blockIdx.x, warp, sm[warp], cnt);
    if (kStats) add_stats(w, cnt);
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
    unsigned long long cnt[7] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
    const uint32_t items = 4u * ntiles;
    for (;;) {
        uint32_t item = 0u;
        if (lane == 0) item = atomicAdd(queue, 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= items) break;
        accumulate_block<kStats, TW>(vs, w, tile_base + (item >> 2), (int)(item & 3u), sm[warp], cnt);
    }
    if (kStats) add_stats(w, cnt);
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

// binning.cu -- a1 projection, a2 count/scan/emit, a3 per-tile depth sort.
//
// Eq. 1 (Sec. 3.1) projects each 3D Gaussian; the blend visits Gaussians in depth
// order per pixel (Sec. 3.1).  Work is binned by 16x16 tile: each (view, Gaussian)
// lists itself in every tile its 3-sigma rectangle touches, and each tile's list
// is sorted by (FP32 depth bits, Gaussian index).
//
// Design: a counting sort by tile (one atomic per pair to count, a scan, one atomic
// per pair to place) followed by a per-tile sort in shared memory.  Each pair is
// written once and read once by the sort, instead of the 6-8 read/write passes of
// a global radix sort over (view, tile, depth) keys.
#include <algorithm>

#include "launch.h"

namespace tsp {

namespace {

// grid (ceil(nmax/128), F): one thread per Gaussian, its view-dependent colour
// (real SH up to degree 3 along the unit direction camera centre -> mean, + 0.5,
// clamped at 0) in every view of its frame; the coefficients are read once.
__global__ void __launch_bounds__(128) k_colour(const ViewSet vs, const float* __restrict__ sh, int sh_degree,
                                                Work w)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int f = blockIdx.y;
    if (g >= vs.fn[f]) return;
    const int nb = (sh_degree + 1) * (sh_degree + 1);
    float c[16][3];
    const float* s = sh + (size_t)g * nb * 3;
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) c[k][ch] = k < nb ? s[3 * k + ch] : 0.f;
    const float4 m = vs.fmo[f][g];
    for (int v = vs.fview[f]; v < vs.fview[f + 1]; ++v) {
        const DevCam& cm = vs.cam[v];
        // camera centre C = -R^T t
        const float Cx = -(cm.R[0] * cm.t[0] + cm.R[3] * cm.t[1] + cm.R[6] * cm.t[2]);
        const float Cy = -(cm.R[1] * cm.t[0] + cm.R[4] * cm.t[1] + cm.R[7] * cm.t[2]);
        const float Cz = -(cm.R[2] * cm.t[0] + cm.R[5] * cm.t[1] + cm.R[8] * cm.t[2]);
        float dx = m.x - Cx, dy = m.y - Cy, dz = m.z - Cz;
        const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inv; dy *= inv; dz *= inv;
        float Y[16];
        sh_basis16(dx, dy, dz, Y);
        float r = 0.5f, gg = 0.5f, b = 0.5f;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            r += Y[k] * c[k][0];
            gg += Y[k] * c[k][1];
            b += Y[k] * c[k][2];
        }
        w.color[(size_t)vs.vrec[v] + g] = make_float4(fmaxf(r, 0.f), fmaxf(gg, 0.f), fmaxf(b, 0.f), 0.f);
    }
}

// grid (ceil(nmax/256), V): one thread per (view, Gaussian), Gaussian index fastest.
// kMode 0: motion fit (zero the moment record, note the moment origin's pixel);
// kMode 1: render (view-dependent colour; one frame).
// The tile counters are raised once per (record, tile) item.  A warp's items are
// spread evenly over its lanes (a warp scan numbers them; each lane finds the
// owner of its item by a 5-step shuffle search), so the warp issues about
// (its items) / 32 atomic instructions instead of one per tile of its largest
// rectangle.
template <int kMode>
__global__ void __launch_bounds__(256) k_preprocess(const ViewSet vs, const float* __restrict__ sh,
                                                    int sh_degree, Work w)
{
    constexpr int mode = kMode;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    const int lane = threadIdx.x & 31;
    uint32_t cnt = 0u, rxy = 0u, rw = 0u;         // items, rectangle corner and width
    if (g < vs.vn[v]) {
        const size_t i = (size_t)vs.vrec[v] + g;
        const int fr = vs.vframe[v];
        if (mode == 0) {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            w.moments[4 * i] = z; w.moments[4 * i + 1] = z; w.moments[4 * i + 2] = z; w.moments[4 * i + 3] = z;
        }
        const float4 m = vs.fmo[fr][g];
        KeyProj p;
        if (!key_project(vs.cam[v], m, vs.fq[fr][g], vs.fs[fr][g], vs.tiles_x[v], vs.tiles_y[v], vs.tw, vs.th, p)) {
            w.rect[i] = make_short4(0, 0, 0, 0);
            w.touched[i] = 0u;
            w.depth[i] = 0u;
        } else {
            w.rect[i] = make_short4((short)p.x0, (short)p.y0, (short)p.x1, (short)p.y1);
            cnt = (uint32_t)((p.x1 - p.x0) * (p.y1 - p.y0));
            rxy = (uint32_t)p.x0 | ((uint32_t)p.y0 << 16);
            rw = (uint32_t)(p.x1 - p.x0);
            w.touched[i] = cnt;
            w.depth[i] = __float_as_uint(p.pz);
            const float3 f = blend_factor(p);
            // mean relative to the rectangle's corner pixel (x0*tw, y0*th), to ~1e-6 px
            float2 ux, uy;
            mean2d_df(vs.cam[v], m, ux, uy);
            const float rx = __fadd_rn(__fsub_rn(ux.x, (float)(p.x0 * vs.tw)), ux.y);
            const float ry = __fadd_rn(__fsub_rn(uy.x, (float)(p.y0 * vs.th)), uy.y);
            float4* rc = w.rec + 4 * i;
            rc[kRecGeom0] = make_float4(rx, ry, f.x, f.y);
            const float2 dlt = moment_origin_shift(ux, uy, rx, ry, p.x0 * vs.tw, p.y0 * vs.th,
                                                   vs.cam[v].W, vs.cam[v].H);
            rc[kRecGeom1] = make_float4(f.z, m.w, dlt.x, dlt.y);
            rc[kRecCull] = cull_record(f.x, f.y, f.z, m.w);
            rc[kRecCorner] = make_float4(rec_pack_corner(p.x0, p.y0), log2f(m.w), 0.f, 0.f);
            if (mode == 0) {
                // the pixel holding the moment origin; k_dref reads the track there
                const int W = vs.cam[v].W, H = vs.cam[v].H;
                const int ox = min(max((int)floorf(ux.x + ux.y + dlt.x), 0), W - 1);
                const int oy = min(max((int)floorf(uy.x + uy.y + dlt.y), 0), H - 1);
                w.oref[i] = (uint32_t)oy * (uint32_t)W + (uint32_t)ox;
            }
        }
    }
    uint32_t inc = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    const uint32_t exc = inc - cnt;
    const uint32_t base = vs.toff[v];
    const uint32_t tx_n = (uint32_t)vs.tiles_x[v];
    for (uint32_t it0 = 0; it0 < total; it0 += 32) {
        const uint32_t item = it0 + (uint32_t)lane;
        int own = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t e = __shfl_sync(0xffffffffu, exc, own + step);
            if (e <= item) own += step;
        }
        const uint32_t off = item - __shfl_sync(0xffffffffu, exc, own);
        const uint32_t xy = __shfl_sync(0xffffffffu, rxy, own);
        const uint32_t wd = __shfl_sync(0xffffffffu, rw, own);
        if (item < total) {
            const uint32_t dy = wd ? off / wd : 0u, dx = off - dy * wd;
            const uint32_t t = base + ((xy >> 16) + dy) * tx_n + (xy & 0xffffu) + dx;
            atomicAdd(&w.tile_count[(size_t)t * kCounterStride], 1u);
        }
    }
}

// Reference displacement of every (view, Gaussian) record of views v0.. (grid.y
// views): the track at the pixel holding the moment origin.  Separate from the
// preprocess so that tracks may still be in flight while the tiles are binned.
__global__ void __launch_bounds__(256) k_dref(const ViewSet vs, Work w, int v0)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = v0 + (int)blockIdx.y;
    if (g >= vs.vn[v] || gate_closed(w)) return;
    const size_t i = (size_t)vs.vrec[v] + g;
    if (w.touched[i] == 0u) return;
    const uint32_t pix = w.oref[i];
    if (w.checked && !pixel_ok(pix, (uint32_t)vs.cam[v].W, (uint32_t)vs.cam[v].H)) {
        check_failed(w.dstatus, kSiteRefPixel);
        reinterpret_cast<float2*>(w.rec + 4 * i + kRecCorner)[1] = make_float2(0.f, 0.f);
        return;
    }
    reinterpret_cast<float2*>(w.rec + 4 * i + kRecCorner)[1] = vs.disp[v][pix];
}

// Exclusive scan of the NT strided tile counts in three launches: (1) each CTA
// sums a span of kScanSpan tiles (4 independent loads per thread), (2) one CTA
// scans the span sums and writes K and off[NT], (3) each CTA scans its span again
// and adds the span's prefix.
constexpr int kScanThreads = 256;
constexpr int kScanSpan = 4 * kScanThreads;

// Block-wide inclusive scan of one 64-bit value per thread; returns the inclusive
// prefix and leaves the block total in *total.
__device__ __forceinline__ unsigned long long block_scan_incl(unsigned long long x,
                                                              unsigned long long* warp_tot,
                                                              unsigned long long* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long q = lane < nw ? warp_tot[lane] : 0ull;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, q, d);
            if (lane >= d) q += y;
        }
        if (lane < nw) warp_tot[lane] = q;
    }
    __syncthreads();
    const unsigned long long r = x + (wid > 0 ? warp_tot[wid - 1] : 0ull);
    *total = warp_tot[nw - 1];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void load_counts4(const uint32_t* __restrict__ cnt, uint32_t NT, uint32_t i0,
                                             uint32_t stride, uint32_t (&c)[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] = (i0 + k < NT) ? cnt[(size_t)(i0 + k) * stride] : 0u;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ cnt, uint32_t NT,
                                                              uint32_t stride,
                                                              unsigned long long* __restrict__ span_sum,
                                                              const uint32_t* __restrict__ enable)
{
    if (enable && !*enable) return;
    __shared__ unsigned long long warp_tot[32];
    uint32_t c[4];
    load_counts4(cnt, NT, blockIdx.x * kScanSpan + 4 * threadIdx.x, stride, c);
    unsigned long long tot;
    block_scan_incl((unsigned long long)c[0] + c[1] + c[2] + c[3], warp_tot, &tot);
    if (threadIdx.x == 0) span_sum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_spans(unsigned long long* __restrict__ span_sum, uint32_t nspan,
                                                     uint32_t* __restrict__ off, uint32_t NT, uint32_t cap,
                                                     uint32_t* dstatus, const uint32_t* __restrict__ enable)
{
    if (enable && !*enable) return;
    __shared__ unsigned long long warp_tot[32];
    unsigned long long carry = 0;
    for (uint32_t b = 0; b < nspan; b += 1024) {
        const uint32_t i = b + threadIdx.x;
        const unsigned long long x = i < nspan ? span_sum[i] : 0ull;
        unsigned long long tot;
        const unsigned long long incl = block_scan_incl(x, warp_tot, &tot);
        if (i < nspan) span_sum[i] = carry + incl - x;            // exclusive prefix
        carry += tot;
    }
    if (threadIdx.x == 0) {
        off[NT] = (uint32_t)min(carry, 0xffffffffull);
        dstatus[1] = (uint32_t)(carry & 0xffffffffull);
        dstatus[2] = (uint32_t)(carry >> 32);
        if (carry > cap) atomicOr(&dstatus[0], kStatusOverflow);
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* __restrict__ cnt, uint32_t NT,
                                                            uint32_t stride,
                                                            const unsigned long long* __restrict__ span_pre,
                                                            uint32_t* __restrict__ off,
                                                            const uint32_t* __restrict__ enable)
{
    if (enable && !*enable) return;
    __shared__ unsigned long long warp_tot[32];
    const uint32_t i0 = blockIdx.x * kScanSpan + 4 * threadIdx.x;
    uint32_t c[4];
    load_counts4(cnt, NT, i0, stride, c);
    const unsigned long long sum = (unsigned long long)c[0] + c[1] + c[2] + c[3];
    unsigned long long tot;
    unsigned long long run = block_scan_incl(sum, warp_tot, &tot) - sum + span_pre[blockIdx.x];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (i0 + k < NT) {
            off[i0 + k] = (uint32_t)min(run, 0xffffffffull);
            run += c[k];
        }
}

// The 32 records of a warp (one view, consecutive Gaussians) are flattened into
// their (record, tile) items: a warp scan of the tile counts numbers the items,
// lane l takes items l, l + 32, ..., finds the owning record as the last lane
// whose exclusive count is <= the item (a 5-step shuffle search), and 8 items per
// lane have their slot atomics (and their lists' start offsets) in flight before
// any result is used.  Lanes stay
// busy whatever the mix of culled, small and large records.
__global__ void __launch_bounds__(256) k_scatter(const ViewSet vs, Work w)
{
    constexpr int kIlp = 8;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    const int lane = threadIdx.x & 31;
    uint32_t cnt = 0u, rxy = 0u, rzw = 0u, klo = 0u, khi = 0u;
    if (g < vs.vn[v]) {
        const size_t i = (size_t)vs.vrec[v] + g;
        cnt = w.touched[i];
        if (cnt) {
            const short4 r = w.rect[i];
            rxy = (uint32_t)(uint16_t)r.x | ((uint32_t)(uint16_t)r.y << 16);
            rzw = (uint32_t)(uint16_t)r.z | ((uint32_t)(uint16_t)r.w << 16);
            klo = (uint32_t)g;
            khi = w.depth[i];
        }
    }
    uint32_t inc = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    const uint32_t exc = inc - cnt;
    const uint32_t base = vs.toff[v];
    const int tx_n = vs.tiles_x[v];
    for (uint32_t it0 = 0; it0 < total; it0 += 32 * kIlp) {
        uint32_t toff[kIlp], slot[kIlp], k0[kIlp], k1[kIlp], tt[kIlp];
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            const uint32_t item = it0 + (uint32_t)(u * 32 + lane);
            int own = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t e = __shfl_sync(0xffffffffu, exc, own + step);
                if (e <= item) own += step;
            }
            const uint32_t off = item - __shfl_sync(0xffffffffu, exc, own);
            const uint32_t xy = __shfl_sync(0xffffffffu, rxy, own);
            const uint32_t zw = __shfl_sync(0xffffffffu, rzw, own);
            k0[u] = __shfl_sync(0xffffffffu, klo, own);
            k1[u] = __shfl_sync(0xffffffffu, khi, own);
            const uint32_t x0 = xy & 0xffffu, y0 = xy >> 16, rw = (zw & 0xffffu) - x0;
            const uint32_t dy = rw ? off / rw : 0u, dx = off - dy * rw;
            const uint32_t t = base + (y0 + dy) * (uint32_t)tx_n + x0 + dx;
            tt[u] = t;
            // the list's start is fetched, and the entry's block mask formed, while
            // the slot atomic is in flight
            if (item < total) {
                if (w.checked && !index_ok(t, w.nt)) {
                    check_failed(w.dstatus, kSiteScatterTile);
                    tt[u] = 0xffffffffu;
                    continue;
                }
                slot[u] = atomicAdd(&w.tile_fill[(size_t)t * kCounterStride], 1u);
                toff[u] = w.tile_off[t];
                // the entry's low word: Gaussian << 4 | block mask (pair_key), the mean
                // moved to the tile's corner by tile_local's exact integer shift
                const float4* rc = w.rec + 4 * ((size_t)vs.vrec[v] + k0[u]);
                const float2 mu = *reinterpret_cast<const float2*>(rc + kRecGeom0);
                const uint32_t mk = block_hit_mask(mu.x + (float)(-(int)dx * vs.tw), mu.y + (float)(-(int)dy * vs.th),
                                                   rc[kRecCull], vs.tw);
                k0[u] = (k0[u] << 4) | mk;
            }
        }
#pragma unroll
        for (int u = 0; u < kIlp; ++u)
            if (it0 + (uint32_t)(u * 32 + lane) < total) {
                if (w.checked) {
                    if (tt[u] == 0xffffffffu) continue;
                    if (!slot_ok(toff[u], slot[u], w.tile_off[tt[u] + 1])) {
                        check_failed(w.dstatus, kSiteScatterSlot);
                        continue;
                    }
                }
                const uint64_t pos = (uint64_t)toff[u] + slot[u];
                if (pos < w.cap) w.pairs[pos] = ((uint64_t)k1[u] << 32) | k0[u];
            }
    }
}

constexpr int kSortCap = 4096;      // entries sorted in shared memory at once
constexpr int kSortThreads = 256;
// CTAs of the long-list sort: one tile each at a time; enough to fill 148 SMs
// (a dense frame has thousands of lists longer than kWarpSortMax)
constexpr int kLongSortCtas = 148 * 4;

// Bitonic sort of n <= kSortCap keys at src (global) in shared memory, written back.
__device__ void smem_sort(uint64_t* src, uint32_t n, uint64_t* s)
{
    uint32_t P = 2;
    while (P < n) P <<= 1;
    for (uint32_t i = threadIdx.x; i < P; i += kSortThreads) s[i] = i < n ? src[i] : ~0ull;
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < P; i += kSortThreads) {
                const uint32_t l = i ^ j;
                if (l > i) {
                    const uint64_t a = s[i], b = s[l];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) { s[i] = b; s[l] = a; }
                }
            }
            __syncthreads();
        }
    for (uint32_t i = threadIdx.x; i < n; i += kSortThreads) src[i] = s[i];
    __syncthreads();
}

// One warp per tile list of 2 <= n <= 32 * KPL keys, bitonic-sorted in registers:
// lane l holds list positions l * KPL + i, i < KPL, padded with ~0 (keys are
// unique and never ~0).  The network is the bitonic sort in its "flip" form: the
// merge of two sorted runs into one of size k starts by comparing position p
// with its mirror p ^ (k - 1), and every later stage compares p with p ^ j
// (j = k/4, ..., 1); all comparators put the smaller key at the lower position,
// so no stage needs a direction.  Strides below KPL stay inside a lane (fixed
// register pairs); larger ones pair lane l with lane l ^ m through shuffles.
constexpr int kWarpSortMax = 512;

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t x, int m)
{
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)x, m);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(x >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}

// a gets the smaller key, b the larger
__device__ __forceinline__ void cmp_swap(uint64_t& a, uint64_t& b)
{
    const bool sw = b < a;
    const uint64_t lo = sw ? b : a, hi = sw ? a : b;
    a = lo;
    b = hi;
}

// The key this lane keeps of the pair (own x, partner's y): the smaller one at
// the lower position of the pair, the larger one at the upper.
__device__ __forceinline__ uint64_t keep(uint64_t x, uint64_t y, bool lower)
{
    return ((y < x) == lower) ? y : x;
}

// In-lane stage of stride J: pairs (i, i + J) for the i with bit J clear.
template <int KPL, int J>
__device__ __forceinline__ void lane_stage(uint64_t (&x)[KPL])
{
#pragma unroll
    for (int i = 0; i < KPL; ++i)
        if ((i & J) == 0) cmp_swap(x[i], x[i ^ J]);
}

// In-lane stages of strides J, J/2, ..., 1.
template <int KPL, int J>
__device__ __forceinline__ void lane_stages(uint64_t (&x)[KPL])
{
    if constexpr (J >= 1) {
        lane_stage<KPL, J>(x);
        lane_stages<KPL, J / 2>(x);
    }
}

// Sorts each lane's KPL keys: merges of size K = 2, 4, ..., KPL, each a mirror
// stage followed by strides K/4, ..., 1.
template <int KPL, int K>
__device__ __forceinline__ void lane_sort(uint64_t (&x)[KPL])
{
    if constexpr (K <= KPL) {
#pragma unroll
        for (int i = 0; i < KPL; ++i)
            if ((i & (K / 2)) == 0) cmp_swap(x[i], x[i ^ (K - 1)]);
        lane_stages<KPL, K / 4>(x);
        lane_sort<KPL, 2 * K>(x);
    }
}

template <int KPL>
__device__ __forceinline__ void warp_sort_list(uint64_t* __restrict__ keys, uint32_t n, int lane)
{
    uint64_t x[KPL];
#pragma unroll
    for (int i = 0; i < KPL; ++i) {
        const uint32_t e = (uint32_t)(lane * KPL + i);
        x[i] = e < n ? keys[e] : ~0ull;
    }
    lane_sort<KPL, 2>(x);
    // merges across lanes stay rolled: unrolling every list size overflows the
    // instruction cache once warps of one SM sort lists of different sizes
#pragma unroll 1
    for (int kl = 2; kl <= 32; kl <<= 1) {         // merged run = kl lanes
        {
            // mirror stage: lane l with l ^ (kl - 1), element i with KPL - 1 - i
            const int m = kl - 1;
            const bool lower = (lane & (kl >> 1)) == 0;
#pragma unroll
            for (int i = 0; i < KPL / 2; ++i) {
                const uint64_t ya = shfl_xor_u64(x[KPL - 1 - i], m);
                const uint64_t yb = shfl_xor_u64(x[i], m);
                x[i] = keep(x[i], ya, lower);
                x[KPL - 1 - i] = keep(x[KPL - 1 - i], yb, lower);
            }
            if constexpr (KPL == 1) x[0] = keep(x[0], shfl_xor_u64(x[0], m), lower);
        }
#pragma unroll 1
        for (int jl = kl >> 2; jl >= 1; jl >>= 1) {
            const bool lower = (lane & jl) == 0;
#pragma unroll
            for (int i = 0; i < KPL; ++i) x[i] = keep(x[i], shfl_xor_u64(x[i], jl), lower);
        }
        lane_stages<KPL, KPL / 2>(x);
    }
#pragma unroll
    for (int i = 0; i < KPL; ++i) {
        const uint32_t e = (uint32_t)(lane * KPL + i);
        if (e < n) keys[e] = x[i];
    }
}

// Eight tiles per 256-thread CTA, one per warp; tiles whose lists are longer than
// kWarpSortMax are appended to long_list (count in *long_count) for
// k_tile_sort_warp_long (up to kWarpSortLong keys) and k_tile_sort (longer).
__global__ void __launch_bounds__(256) k_tile_sort_warp(const uint32_t* __restrict__ off,
                                                        uint64_t* __restrict__ pairs, uint32_t cap,
                                                        uint32_t NT, uint32_t* __restrict__ long_list,
                                                        uint32_t* __restrict__ long_count,
                                                        const uint32_t* __restrict__ enable,
                                                        uint32_t* __restrict__ check_status)
{
    if (enable && !*enable) return;
    const uint32_t t = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= NT) return;
    if (check_status && !range_ok(off[t], off[t + 1], 0xffffffffu)) {
        if (lane == 0) check_failed(check_status, kSiteTileRange);
        return;
    }
    const uint32_t b = min(off[t], cap), e = min(off[t + 1], cap);
    if (e <= b + 1) return;
    const uint32_t n = e - b;
    uint64_t* keys = pairs + b;
    if (n <= 32) warp_sort_list<1>(keys, n, lane);
    else if (n <= 64) warp_sort_list<2>(keys, n, lane);
    else if (n <= 128) warp_sort_list<4>(keys, n, lane);
    else if (n <= 256) warp_sort_list<8>(keys, n, lane);
    else if (n <= (uint32_t)kWarpSortMax) warp_sort_list<16>(keys, n, lane);
    else if (lane == 0) long_list[atomicAdd(long_count, 1u)] = t;
}

// Listed lists of kWarpSortMax < n <= kWarpSortLong keys: one warp each, 32 keys
// a lane (the same network; 64 registers of keys), the warps of the grid taking
// the listed tiles in turn.
constexpr int kWarpSortLong = 1024;

__global__ void __launch_bounds__(256) k_tile_sort_warp_long(const uint32_t* __restrict__ off,
                                                             uint64_t* __restrict__ pairs, uint32_t cap,
                                                             const uint32_t* __restrict__ long_list,
                                                             const uint32_t* __restrict__ long_count,
                                                             const uint32_t* __restrict__ enable)
{
    if (enable && !*enable) return;
    const uint32_t count = *long_count;
    const int lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t li = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; li < count; li += nw) {
        const uint32_t t = long_list[li];
        const uint32_t b = min(off[t], cap), e = min(off[t + 1], cap);
        if (e - b <= (uint32_t)kWarpSortLong) warp_sort_list<32>(pairs + b, e - b, lane);
    }
}

// Listed lists longer than kWarpSortLong, one CTA at a time per tile.  Up to
// kSortCap keys sort in shared memory; longer lists sort kSortCap-sized runs there
// and then merge runs pairwise in global memory (each key finds its output slot
// by a binary search in the partner run; keys are unique).
__global__ void __launch_bounds__(kSortThreads) k_tile_sort(const uint32_t* __restrict__ off,
                                                            uint64_t* pairs, uint64_t* tmp, uint32_t cap,
                                                            const uint32_t* __restrict__ long_list,
                                                            const uint32_t* __restrict__ long_count,
                                                            const uint32_t* __restrict__ enable)
{
    if (enable && !*enable) return;
    __shared__ uint64_t s[kSortCap];
    const uint32_t count = *long_count;
    for (uint32_t li = blockIdx.x; li < count; li += gridDim.x) {
        const uint32_t t = long_list[li];
        const uint32_t b = min(off[t], cap), e = min(off[t + 1], cap);
        const uint32_t n = e - b;
        if (n <= (uint32_t)kWarpSortLong) continue;          // sorted by k_tile_sort_warp_long
        if (n <= (uint32_t)kSortCap) {
            smem_sort(pairs + b, n, s);
            continue;
        }
        for (uint32_t c = 0; c < n; c += kSortCap) smem_sort(pairs + b + c, min((uint32_t)kSortCap, n - c), s);
        uint64_t* src = pairs + b;
        uint64_t* dst = tmp + b;
        for (uint32_t L = kSortCap; L < n; L <<= 1) {
            for (uint32_t i = threadIdx.x; i < n; i += kSortThreads) {
                const uint32_t run = i / L, start = run * L, partner = run ^ 1u;
                const uint64_t key = src[i];
                const uint64_t ps64 = (uint64_t)partner * L;
                if (ps64 >= n) { dst[i] = key; continue; }
                const uint32_t ps = (uint32_t)ps64, pe = min(ps + L, n);
                uint32_t lo = ps, hi = pe;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (src[mid] < key) lo = mid + 1; else hi = mid;
                }
                const uint32_t pair_start = min(run, partner) * L;
                dst[pair_start + (i - start) + (lo - ps)] = key;
            }
            __syncthreads();
            uint64_t* x = src; src = dst; dst = x;
        }
        if (src != pairs + b)
            for (uint32_t i = threadIdx.x; i < n; i += kSortThreads) pairs[b + i] = src[i];
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_preprocess(const ViewSet& vs, const float* sh, int sh_degree, int mode, const Work& w,
                              cudaStream_t st)
{
    if (vs.nmax == 0 || vs.V == 0) return cudaSuccess;
    dim3 grid((vs.nmax + 255) / 256, vs.V);
    if (mode == 0) {
        k_preprocess<0><<<grid, 256, 0, st>>>(vs, sh, sh_degree, w);
    } else {
        k_preprocess<1><<<grid, 256, 0, st>>>(vs, sh, sh_degree, w);
        k_colour<<<dim3((vs.nmax + 127) / 128, vs.F), 128, 0, st>>>(vs, sh, sh_degree, w);
    }
    return cudaGetLastError();
}

// The track gate: one thread polls the 32-bit word at `flag` until it reaches
// `value` (acquire at GPU scope, so the tracks written before the producer's
// release are visible after), sleeping ~1 us between polls.  The wait is bounded
// twice, by the global timer and by a poll count; when it runs out it sets
// kStatusGate and returns, and the track readers and output writers of the call
// return at once (gate_closed).
__global__ void k_track_gate(const uint32_t* flag, uint32_t value, unsigned long long timeout_ns,
                             uint32_t max_polls, uint32_t* dstatus)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (uint32_t polls = 0;; ++polls) {
        uint32_t cur;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(flag) : "memory");
        if (cur >= value) return;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (polls >= max_polls || t - t0 >= timeout_ns) {
            atomicOr(&dstatus[0], kStatusGate);
            return;
        }
        __nanosleep(1000);
    }
}

cudaError_t launch_track_gate(const uint32_t* flag, uint32_t value, long long timeout_us, const Work& w,
                              cudaStream_t st)
{
    const unsigned long long ns = (unsigned long long)timeout_us * 1000ull;
    const uint32_t polls = (uint32_t)std::min<long long>(4 * timeout_us + 1000, 0x7fffffffLL);
    k_track_gate<<<1, 32, 0, st>>>(flag, value, ns, polls, w.dstatus);
    return cudaGetLastError();
}

cudaError_t launch_dref(const ViewSet& vs, const Work& w, int v0, int v1, cudaStream_t st)
{
    if (vs.nmax == 0 || v1 <= v0) return cudaSuccess;
    dim3 grid((vs.nmax + 255) / 256, v1 - v0);
    k_dref<<<grid, 256, 0, st>>>(vs, w, v0);
    return cudaGetLastError();
}

cudaError_t launch_scan(const Work& w, uint32_t NT, cudaStream_t st)
{
    return launch_scan_u32(w.tile_count, kCounterStride, NT, w.tile_off, w.span_sum, w.cap, w.dstatus, st);
}

cudaError_t launch_scan_u32(const uint32_t* cnt, uint32_t stride, uint32_t n, uint32_t* off,
                            unsigned long long* span_sum, uint32_t cap, uint32_t* status, cudaStream_t st,
                            const uint32_t* enable)
{
    const uint32_t nspan = (n + kScanSpan - 1) / kScanSpan;
    if (nspan > 0) k_scan_reduce<<<nspan, kScanThreads, 0, st>>>(cnt, n, stride, span_sum, enable);
    k_scan_spans<<<1, 1024, 0, st>>>(span_sum, nspan, off, n, cap, status, enable);
    if (nspan > 0) k_scan_down<<<nspan, kScanThreads, 0, st>>>(cnt, n, stride, span_sum, off, enable);
    return cudaGetLastError();
}

cudaError_t launch_segment_sort(const uint32_t* off, uint64_t* keys, uint64_t* tmp, uint32_t cap, uint32_t nseg,
                                uint32_t* long_list, uint32_t* long_count, cudaStream_t st, const uint32_t* enable)
{
    if (nseg == 0) return cudaSuccess;
    const cudaError_t e = cudaMemsetAsync(long_count, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    k_tile_sort_warp<<<(nseg + 7) / 8, 256, 0, st>>>(off, keys, cap, nseg, long_list, long_count, enable,
                                                     nullptr);
    k_tile_sort_warp_long<<<kLongSortCtas, 256, 0, st>>>(off, keys, cap, long_list, long_count, enable);
    k_tile_sort<<<kLongSortCtas, kSortThreads, 0, st>>>(off, keys, tmp, cap, long_list, long_count, enable);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const ViewSet& vs, const Work& w, cudaStream_t st)
{
    if (vs.nmax == 0 || vs.V == 0) return cudaSuccess;
    dim3 grid((vs.nmax + 255) / 256, vs.V);
    k_scatter<<<grid, 256, 0, st>>>(vs, w);
    return cudaGetLastError();
}

cudaError_t launch_tile_sort(const Work& w, uint32_t NT, cudaStream_t st)
{
    if (NT == 0) return cudaSuccess;
    // tile_fill is free once the pairs are scattered: it holds the long-list tiles
    k_tile_sort_warp<<<(NT + 7) / 8, 256, 0, st>>>(w.tile_off, w.pairs, w.cap, NT, w.tile_fill, &w.dstatus[3],
                                                   nullptr, w.checked ? w.dstatus : nullptr);
    k_tile_sort_warp_long<<<kLongSortCtas, 256, 0, st>>>(w.tile_off, w.pairs, w.cap, w.tile_fill, &w.dstatus[3],
                                                         nullptr);
    k_tile_sort<<<kLongSortCtas, kSortThreads, 0, st>>>(w.tile_off, w.pairs, w.pairs_tmp, w.cap, w.tile_fill,
                                              &w.dstatus[3], nullptr);
    return cudaGetLastError();
}

}  // namespace tsp

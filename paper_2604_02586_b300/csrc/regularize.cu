// regularize.cu -- motion regularization (Sec. 4.5): static detection from the
// PWI-LS pixel counters, exact K-nearest neighbours on a uniform grid, median
// filtering of the motion components and propagation to the Gaussians that
// have none.
//
// Neighbours.  The members of a component (Gaussians with a solved position, or
// with a solved covariance) are counting-sorted into a uniform grid whose box and
// cell count are chosen on the device from the members' bounding box and number
// (about two members per cell), so nothing waits on the host.  Each query walks
// shells of cells around its own cell (shell r = the cells at Chebyshev distance
// r); within a shell the cells of one (z, y) row that lie in the shell are
// contiguous in the sorted order, so a row is one range.  The walk stops once the
// k-th best distance is below the distance from the query to the nearest cell
// not yet visited, less a margin that covers the FP32 rounding of the cell
// assignment; so the k nearest found are the exact k nearest under the pinned
// FP32 distance and (distance, index) order.
//
// Skewed point sets.  A uniform grid sized by the members' box and count fails
// when the density varies by orders of magnitude (dense surfaces with a sparse
// far field of floaters, tight clusters): the dense regions crowd few cells.
// When the grid's occupancy statistic (sum over cells of count^2 / members) is
// far above a Poisson grid's, the set is searched with a bounding-volume
// hierarchy instead: members sorted by 30-bit Morton code (bucketed by the top
// 16 bits, buckets sorted by (code, index)), a binary radix tree built from the
// sorted keys (Karras 2012, "Maximizing parallelism in the construction of BVHs,
// octrees, and k-d trees"), child boxes refitted bottom-up, and a depth-first
// walk, nearer child first, that skips a subtree whose box distance exceeds the
// current k-th.  The box distance is computed with the same FP32 operations as
// the point distance from per-axis gaps that no member's offset can undercut,
// so by monotone rounding it is a lower bound of every member's FP32 distance:
// the pruning is exact.  The switch is taken on the device; both paths are
// always launched and the unused one returns at once.
#include <cfloat>
#include <cmath>

#include "launch.h"

namespace tsp {
namespace {

constexpr int kRegThreads = 256;
constexpr int kMembersPerCell = 3;       // grid density: members per cell on average
// BVH when sum(count^2) / members exceeds this (a Poisson grid gives about
// kMembersPerCell + 1)
constexpr float kSkewLimit = 16.0f;

__device__ __forceinline__ uint32_t ordered_key(float f)
{
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float key_value(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// The pinned FP32 squared distance: ((dx*dx + dy*dy) + dz*dz), each operation
// rounded on its own.
__device__ __forceinline__ float dist2(float qx, float qy, float qz, float4 p)
{
    const float dx = __fsub_rn(qx, p.x), dy = __fsub_rn(qy, p.y), dz = __fsub_rn(qz, p.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Grid j's members: every point (bits 0) or those with mask & bits != 0.
__device__ __forceinline__ bool member(const uint8_t* mask, uint8_t bits, int g)
{
    return bits == 0 || (mask[g] & bits) != 0;
}

// acc[8 j + 0..2] ~key(min), [8 j + 3..5] key(max), [8 j + 6] member count of
// grid j; all start at 0.
__global__ void __launch_bounds__(kRegThreads) k_grid_bounds(const float4* __restrict__ mo,
                                                            const uint8_t* __restrict__ mask, GridDesc gd, int n,
                                                            uint32_t* __restrict__ acc)
{
    __shared__ uint32_t s[kMaxGrids][7][kRegThreads / 32];
    uint32_t v[kMaxGrids][7];
#pragma unroll
    for (int j = 0; j < kMaxGrids; ++j)
#pragma unroll
        for (int i = 0; i < 7; ++i) v[j][i] = 0;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const float4 p = mo[g];
        const uint32_t k[3] = {ordered_key(p.x), ordered_key(p.y), ordered_key(p.z)};
#pragma unroll
        for (int j = 0; j < kMaxGrids; ++j) {
            if (j >= gd.G || !member(mask, gd.bits[j], g)) continue;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                v[j][i] = max(v[j][i], ~k[i]);
                v[j][3 + i] = max(v[j][3 + i], k[i]);
            }
            v[j][6] += 1;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kMaxGrids; ++j)
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            uint32_t x = v[j][i];
            for (int o = 16; o > 0; o >>= 1) {
                const uint32_t y = __shfl_xor_sync(0xffffffffu, x, o);
                x = i == 6 ? x + y : max(x, y);
            }
            if (lane == 0) s[j][i][wid] = x;
        }
    __syncthreads();
    if (threadIdx.x < 7 * gd.G) {
        const int j = threadIdx.x / 7, i = threadIdx.x % 7;
        uint32_t x = 0;
        for (int w = 0; w < kRegThreads / 32; ++w) x = i == 6 ? x + s[j][i][w] : max(x, s[j][i][w]);
        if (i == 6) {
            if (x) atomicAdd(&acc[8 * j + 6], x);
        } else {
            atomicMax(&acc[8 * j + i], x);
        }
    }
}

// Thread j: grid j over its members' box with about kMembersPerCell members per
// cell and at most max_cells cells.
__global__ void k_grid_setup(const uint32_t* __restrict__ acc_all, int G, uint32_t max_cells,
                             GridParam* __restrict__ gp_all)
{
    const int j = threadIdx.x;
    if (j >= G) return;
    const uint32_t* acc = acc_all + 8 * j;
    GridParam* gp = gp_all + j;
    const uint32_t m = acc[6];
    float lo[3], ext[3], E = 0.0f, amax = 0.0f;
    for (int i = 0; i < 3; ++i) {
        if (m == 0) {
            lo[i] = 0.0f;
            ext[i] = 1.0f;
        } else {
            lo[i] = key_value(~acc[i]);
            const float hi = key_value(acc[3 + i]);
            ext[i] = hi - lo[i];
            amax = fmaxf(amax, fmaxf(fabsf(lo[i]), fabsf(hi)));
        }
        if (!(ext[i] < 1e30f)) ext[i] = 1.0f;
        E = fmaxf(E, ext[i]);
    }
    if (!(E > 0.0f)) E = 1.0f;
    for (int i = 0; i < 3; ++i) ext[i] = fmaxf(ext[i], 1e-3f * E);
    float target = fmaxf(1.0f, floorf((float)m / kMembersPerCell));
    if (target > (float)max_cells) target = (float)max_cells;
    // cubic cells; an axis shorter than one cell gets one cell and the others
    // share the count
    int d[3] = {0, 0, 0};
    for (int round = 0; round < 3; ++round) {
        float vol = 1.0f;
        int free_axes = 0;
        for (int i = 0; i < 3; ++i)
            if (d[i] == 0) {
                vol *= ext[i];
                ++free_axes;
            }
        if (free_axes == 0) break;
        const float h = free_axes == 3 ? cbrtf(vol / target) : (free_axes == 2 ? sqrtf(vol / target) : vol / target);
        bool fixed = false;
        for (int i = 0; i < 3; ++i)
            if (d[i] == 0 && ext[i] < h) {
                d[i] = 1;
                fixed = true;
            }
        if (!fixed) {
            for (int i = 0; i < 3; ++i)
                if (d[i] == 0) d[i] = (int)fminf(fmaxf(floorf(ext[i] / h), 1.0f), 1048576.0f);
            break;
        }
    }
    for (int i = 0; i < 3; ++i) d[i] = d[i] > 0 ? d[i] : 1;
    while ((unsigned long long)d[0] * d[1] * d[2] > max_cells) {
        const int a = d[0] >= d[1] && d[0] >= d[2] ? 0 : (d[1] >= d[2] ? 1 : 2);
        d[a] -= 1;
    }
    for (int i = 0; i < 3; ++i) {
        gp->lo[i] = lo[i];
        gp->inv[i] = d[i] / ext[i];
        gp->h[i] = ext[i] / d[i];
        gp->dims[i] = d[i];
    }
    gp->ncell = d[0] * d[1] * d[2];
    // covers the FP32 rounding of (x - lo) * inv and of the cell walls
    gp->margin = 1e-5f * E + 1e-6f * amax;
}

__device__ __forceinline__ int cell_axis(float x, float lo, float inv, int dim)
{
    const float f = fminf(fmaxf((x - lo) * inv, 0.0f), (float)(dim - 1));
    return (int)f;
}

__device__ __forceinline__ void cell_of(const GridParam& gp, float x, float y, float z, int& cx, int& cy, int& cz)
{
    cx = cell_axis(x, gp.lo[0], gp.inv[0], gp.dims[0]);
    cy = cell_axis(y, gp.lo[1], gp.inv[1], gp.dims[1]);
    cz = cell_axis(z, gp.lo[2], gp.inv[2], gp.dims[2]);
}

// count[j C + cell] of every grid; slot[j n + g] = (cell, rank within the cell)
__global__ void __launch_bounds__(kRegThreads) k_grid_count(const float4* __restrict__ mo,
                                                           const uint8_t* __restrict__ mask, GridDesc gd, int n,
                                                           const GridParam* __restrict__ gpp, uint32_t C,
                                                           uint32_t* __restrict__ count, uint2* __restrict__ slot)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const float4 p = mo[g];
#pragma unroll
    for (int j = 0; j < kMaxGrids; ++j) {
        if (j >= gd.G || !member(mask, gd.bits[j], g)) continue;
        const GridParam& gp = gpp[j];
        int cx, cy, cz;
        cell_of(gp, p.x, p.y, p.z, cx, cy, cz);
        const uint32_t c = ((uint32_t)cz * gp.dims[1] + cy) * gp.dims[0] + cx;
        slot[(size_t)j * n + g] = make_uint2(c, atomicAdd(&count[(size_t)j * C + c], 1u));
    }
}

__global__ void __launch_bounds__(kRegThreads) k_grid_scatter(const float4* __restrict__ mo,
                                                             const uint8_t* __restrict__ mask, GridDesc gd, int n,
                                                             const uint2* __restrict__ slot, uint32_t C,
                                                             const uint32_t* __restrict__ cell_off,
                                                             float4* __restrict__ sorted)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const float4 p = mo[g];
    const float4 e = make_float4(p.x, p.y, p.z, __int_as_float(g));
#pragma unroll
    for (int j = 0; j < kMaxGrids; ++j) {
        if (j >= gd.G || !member(mask, gd.bits[j], g)) continue;
        const uint2 s = slot[(size_t)j * n + g];
        sorted[cell_off[(size_t)j * C + s.x] + s.y] = e;
    }
}

// (d, i) before (bd, bi)?
__device__ __forceinline__ bool closer(float d, int i, float bd, int bi) { return d < bd || (d == bd && i < bi); }

// Insert (d, i) into the sorted list (bd, bi) if it is closer than its last entry.
template <int KMAX>
__device__ __forceinline__ void insert(float (&bd)[KMAX], int (&bi)[KMAX], float d, int i)
{
    if (!closer(d, i, bd[KMAX - 1], bi[KMAX - 1])) return;
    bool c[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX - 1; ++j) c[j] = closer(d, i, bd[j], bi[j]);
    c[KMAX - 1] = true;
#pragma unroll
    for (int j = KMAX - 1; j > 0; --j) {
        bd[j] = c[j - 1] ? bd[j - 1] : (c[j] ? d : bd[j]);
        bi[j] = c[j - 1] ? bi[j - 1] : (c[j] ? i : bi[j]);
    }
    bd[0] = c[0] ? d : bd[0];
    bi[0] = c[0] ? i : bi[0];
}

// Squared distance from q to the cells [x0, x1] x {y} x {z}, each axis' gap
// shrunk by the margin: a lower bound on the FP32 distance of every member there.
__device__ __forceinline__ float seg_bound2(const GridParam& gp, float qx, float qy, float qz, int x0, int x1, int y,
                                            int z)
{
    const float gx = fmaxf(fmaxf(gp.lo[0] + (float)x0 * gp.h[0] - qx, qx - (gp.lo[0] + (float)(x1 + 1) * gp.h[0])) -
                               gp.margin, 0.0f);
    const float gy = fmaxf(fmaxf(gp.lo[1] + (float)y * gp.h[1] - qy, qy - (gp.lo[1] + (float)(y + 1) * gp.h[1])) -
                               gp.margin, 0.0f);
    const float gz = fmaxf(fmaxf(gp.lo[2] + (float)z * gp.h[2] - qz, qz - (gp.lo[2] + (float)(z + 1) * gp.h[2])) -
                               gp.margin, 0.0f);
    return gx * gx + gy * gy + gz * gz;
}

struct KnnQuery {
    float x, y, z;
    int self;
    int k;
};

// Scan the members of cells [x0, x1] x {y} x {z} unless all of them are farther
// than the current k-th (then none can enter the list: the bound is below every
// member's FP32 distance by more than its rounding, so "farther" is strict).
template <int KMAX>
__device__ __forceinline__ void scan_seg(const GridParam& gp, const uint32_t* __restrict__ co,
                                         const float4* __restrict__ sorted, const KnnQuery& q, int x0, int x1, int y,
                                         int z, float (&bd)[KMAX], int (&bi)[KMAX])
{
    float kth = INFINITY;
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
        if (j == q.k - 1) kth = bd[j];
    if (kth < INFINITY && seg_bound2(gp, q.x, q.y, q.z, x0, x1, y, z) * (1.0f - 1e-6f) >= kth) return;
    const uint32_t row = ((uint32_t)z * gp.dims[1] + y) * gp.dims[0];
    const uint32_t a = co[row + x0], b = co[row + x1 + 1];
    for (uint32_t j = a; j < b; ++j) {
        const float4 p = sorted[j];
        const int idx = __float_as_int(p.w);
        if (idx == q.self) continue;
        insert<KMAX>(bd, bi, dist2(q.x, q.y, q.z, p), idx);
    }
}

// (dz, dy) of the nine rows of the 3 x 3 x 3 block, nearest first: the query's
// own row, the four rows sharing a face with it, the four diagonal rows.
__constant__ int8_t kBlockRows[9][2] = {{0, 0}, {-1, 0}, {1, 0}, {0, -1}, {0, 1}, {-1, -1}, {-1, 1}, {1, -1}, {1, 1}};

// Block (x, y): queries [x * blockDim, ...) in the cell order of grid 0 (every
// point), their k nearest members of candidate grid y + 1 (k <= KMAX), -1 padded.
template <int KMAX>
__global__ void __launch_bounds__(kRegThreads) k_knn(int n, int k, const GridParam* __restrict__ gpp, uint32_t C,
                                                    const uint32_t* __restrict__ cell_off,
                                                    const float4* __restrict__ sorted, int32_t* __restrict__ nbr0,
                                                    int32_t* __restrict__ nbr1, const uint32_t* __restrict__ use_bvh)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n || use_bvh[blockIdx.y]) return;
    const int grid = blockIdx.y + 1;
    const GridParam gp = gpp[grid];
    const uint32_t* __restrict__ co = cell_off + (size_t)grid * C;
    int32_t* __restrict__ nbr = blockIdx.y == 0 ? nbr0 : nbr1;
    const float4 qp = sorted[t];
    const KnnQuery q{qp.x, qp.y, qp.z, __float_as_int(qp.w), k};
    int c[3];
    cell_of(gp, q.x, q.y, q.z, c[0], c[1], c[2]);
    const float qc[3] = {q.x, q.y, q.z};
    float bd[KMAX];
    int bi[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        bd[j] = INFINITY;
        bi[j] = INT_MAX;
    }
    int rmax = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) rmax = max(rmax, max(c[i], gp.dims[i] - 1 - c[i]));
    const int d0 = gp.dims[0], d1 = gp.dims[1], d2 = gp.dims[2];
    {
        const int x0 = max(c[0] - 1, 0), x1 = min(c[0] + 1, d0 - 1);
        for (int r = 0; r < 9; ++r) {
            const int z = c[2] + kBlockRows[r][0], y = c[1] + kBlockRows[r][1];
            if (z < 0 || z >= d2 || y < 0 || y >= d1) continue;
            scan_seg<KMAX>(gp, co, sorted, q, x0, x1, y, z, bd, bi);
        }
    }
    for (int r = 1;; ++r) {
        // distance to the nearest cell not yet visited
        float b = INFINITY;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (c[i] - r > 0) b = fminf(b, qc[i] - (gp.lo[i] + (float)(c[i] - r) * gp.h[i]));
            if (c[i] + r < gp.dims[i] - 1) b = fminf(b, gp.lo[i] + (float)(c[i] + r + 1) * gp.h[i] - qc[i]);
        }
        float kth = INFINITY;
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
            if (j == k - 1) kth = bd[j];
        b -= gp.margin;
        if (r >= rmax || (b > 0.0f && kth < b * b * (1.0f - 1e-6f))) break;
        const int s = r + 1;
        const int z0 = max(c[2] - s, 0), z1 = min(c[2] + s, d2 - 1);
        const int y0 = max(c[1] - s, 0), y1 = min(c[1] + s, d1 - 1);
        const int x0 = max(c[0] - s, 0), x1 = min(c[0] + s, d0 - 1);
        for (int z = z0; z <= z1; ++z) {
            for (int y = y0; y <= y1; ++y) {
                if (abs(z - c[2]) == s || abs(y - c[1]) == s) {
                    scan_seg<KMAX>(gp, co, sorted, q, x0, x1, y, z, bd, bi);
                } else {
                    if (c[0] - s >= 0) scan_seg<KMAX>(gp, co, sorted, q, c[0] - s, c[0] - s, y, z, bd, bi);
                    if (c[0] + s < d0) scan_seg<KMAX>(gp, co, sorted, q, c[0] + s, c[0] + s, y, z, bd, bi);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
        if (j < k) nbr[(size_t)q.self * k + j] = bi[j] == INT_MAX ? -1 : bi[j];
}

// ----------------------------------------------------------------- BVH fallback

constexpr int kBvhStack = 64;          // > tree depth: unique 64-bit keys give at most 64 levels

// Sum over the cells of candidate grid y + 1 of count^2.
__global__ void __launch_bounds__(kRegThreads) k_grid_skew(const uint32_t* __restrict__ count, uint32_t C,
                                                          unsigned long long* __restrict__ skew)
{
    __shared__ unsigned long long s[kRegThreads / 32];
    const uint32_t* c = count + (size_t)(blockIdx.y + 1) * C;
    unsigned long long v = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x)
        v += (unsigned long long)c[i] * c[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kRegThreads / 32; ++w) t += s[w];
        if (t) atomicAdd(&skew[blockIdx.y], t);
    }
}

// use_bvh[c] for each candidate set, use_bvh[2] = any of them.
__global__ void k_bvh_decide(const uint32_t* __restrict__ acc, const unsigned long long* __restrict__ skew, int ncand,
                             uint32_t* __restrict__ use_bvh)
{
    if (threadIdx.x != 0) return;
    uint32_t any = 0u;
    for (int c = 0; c < ncand; ++c) {
        const uint32_t m = acc[8 * (c + 1) + 6];
        const uint32_t u = (m > 1u && (float)skew[c] > kSkewLimit * (float)m) ? 1u : 0u;
        use_bvh[c] = u;
        any |= u;
    }
    use_bvh[2] = any;
}

// Spread the low 10 bits of x to every third bit.
__device__ __forceinline__ uint32_t spread3(uint32_t x)
{
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__device__ __forceinline__ uint32_t morton30(float4 p, const uint32_t* acc)
{
    const float c[3] = {p.x, p.y, p.z};
    uint32_t code = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float lo = key_value(~acc[i]), hi = key_value(acc[3 + i]);
        const float ext = hi - lo;
        const float inv = ext > 0.f ? 1024.0f / ext : 0.f;
        const uint32_t qi = (uint32_t)fminf(fmaxf((c[i] - lo) * inv, 0.f), 1023.f);
        code |= spread3(qi) << (2 - i);
    }
    return code;
}

// Members of candidate set y: bucket by the top 16 bits of the Morton code.
__global__ void __launch_bounds__(kRegThreads) k_bvh_codes(const float4* __restrict__ mo,
                                                          const uint8_t* __restrict__ mask, GridDesc gd, int n,
                                                          const uint32_t* __restrict__ acc,
                                                          const uint32_t* __restrict__ use_bvh,
                                                          uint32_t* __restrict__ bcount, uint2* __restrict__ bslot)
{
    const int c = blockIdx.y;
    if (!use_bvh[c]) return;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        if (!member(mask, gd.bits[c + 1], g)) continue;
        const uint32_t code = morton30(mo[g], acc + 8 * (c + 1));
        const uint32_t b = (uint32_t)c * kMortonBuckets + (code >> 14);      // top 16 of 30 bits
        bslot[(size_t)c * n + g] = make_uint2(b, atomicAdd(&bcount[b], 1u));
    }
}

__global__ void __launch_bounds__(kRegThreads) k_bvh_scatter(const float4* __restrict__ mo,
                                                            const uint8_t* __restrict__ mask, GridDesc gd, int n,
                                                            const uint32_t* __restrict__ acc,
                                                            const uint32_t* __restrict__ use_bvh,
                                                            const uint2* __restrict__ bslot,
                                                            const uint32_t* __restrict__ boff,
                                                            uint64_t* __restrict__ keys)
{
    const int c = blockIdx.y;
    if (!use_bvh[c]) return;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        if (!member(mask, gd.bits[c + 1], g)) continue;
        const uint32_t code = morton30(mo[g], acc + 8 * (c + 1));
        const uint2 s = bslot[(size_t)c * n + g];
        keys[boff[s.x] + s.y] = ((uint64_t)code << 32) | (uint32_t)g;
    }
}

// Common-prefix length of sorted keys i and j (-1 outside [0, m)); keys are unique.
__device__ __forceinline__ int bvh_delta(const uint64_t* __restrict__ keys, long long m, long long i, long long j)
{
    if (j < 0 || j >= m) return -1;
    return __clzll((long long)(keys[i] ^ keys[j]));
}

// Karras' construction of internal node i of a binary radix tree over m sorted keys.
// Child encoding: >= 0 an internal node, < 0 the member with index -(c + 1).
__device__ __forceinline__ void bvh_node(const uint64_t* __restrict__ keys, long long m, long long i, int n,
                                              float4* __restrict__ nodes, int32_t* __restrict__ parent)
{
    const int d = bvh_delta(keys, m, i, i + 1) > bvh_delta(keys, m, i, i - 1) ? 1 : -1;
    const int dmin = bvh_delta(keys, m, i, i - d);
    long long lmax = 2;
    while (bvh_delta(keys, m, i, i + lmax * d) > dmin) lmax <<= 1;
    long long l = 0;
    for (long long t = lmax >> 1; t >= 1; t >>= 1)
        if (bvh_delta(keys, m, i, i + (l + t) * d) > dmin) l += t;
    const long long j = i + l * d;
    const int dnode = bvh_delta(keys, m, i, j);
    long long s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (bvh_delta(keys, m, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const long long gam = i + s * d + (d < 0 ? -1 : 0);
    const long long lo = i < j ? i : j, hi = i < j ? j : i;
    int c0, c1;
    if (lo == gam) {
        c0 = -(int)(uint32_t)(keys[gam] & 0xffffffffu) - 1;
        parent[n + gam] = (int)i;
    } else {
        c0 = (int)gam;
        parent[gam] = (int)i;
    }
    if (hi == gam + 1) {
        c1 = -(int)(uint32_t)(keys[gam + 1] & 0xffffffffu) - 1;
        parent[n + gam + 1] = (int)i;
    } else {
        c1 = (int)(gam + 1);
        parent[gam + 1] = (int)i;
    }
    nodes[4 * i + 0].w = __int_as_float(c0);
    nodes[4 * i + 2].w = __int_as_float(c1);
    if (i == 0) parent[0] = -1;
}

__global__ void __launch_bounds__(kRegThreads) k_bvh_build(int n, const uint32_t* __restrict__ acc,
                                                          const uint32_t* __restrict__ use_bvh,
                                                          const uint32_t* __restrict__ boff,
                                                          const uint64_t* __restrict__ keys_all,
                                                          float4* __restrict__ nodes_all,
                                                          int32_t* __restrict__ parent_all)
{
    const int c = blockIdx.y;
    if (!use_bvh[c]) return;
    const long long m = acc[8 * (c + 1) + 6];
    const uint64_t* keys = keys_all + boff[(size_t)c * kMortonBuckets];
    float4* nodes = nodes_all + (size_t)c * n * 4;
    int32_t* parent = parent_all + (size_t)c * 2 * n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m - 1;
         i += (long long)gridDim.x * blockDim.x)
        bvh_node(keys, m, i, n, nodes, parent);
}


__device__ __forceinline__ void child_box(const float4* __restrict__ nodes, const float4* __restrict__ mo, int ch,
                                          float3& lo, float3& hi)
{
    if (ch < 0) {
        const float4 p = mo[-(ch + 1)];
        lo = make_float3(p.x, p.y, p.z);
        hi = lo;
    } else {
        const float4 a = __ldcg(nodes + 4 * ch), b = __ldcg(nodes + 4 * ch + 1);
        const float4 e = __ldcg(nodes + 4 * ch + 2), f = __ldcg(nodes + 4 * ch + 3);
        lo = make_float3(fminf(a.x, e.x), fminf(a.y, e.y), fminf(a.z, e.z));
        hi = make_float3(fmaxf(b.x, f.x), fmaxf(b.y, f.y), fmaxf(b.z, f.z));
    }
}

// From leaf k upwards: the second child to finish a node computes its child boxes.
__device__ __forceinline__ void bvh_refit_leaf(int n, const float4* __restrict__ mo, float4* __restrict__ nodes,
                                               const int32_t* __restrict__ parent, uint32_t* __restrict__ flag,
                                               uint32_t* __restrict__ status, long long k)
{
    int node = parent[n + k];
    for (int level = 0; node >= 0; ++level) {
        if (level > kBvhStack) {                   // deeper than any valid tree: report, stop
            atomicOr(status, kStatusInternal);
            return;
        }
        __threadfence();
        if (atomicAdd(&flag[node], 1u) == 0u) return;       // the other child is not done yet
        __threadfence();
        const int c0 = __float_as_int(__ldcg(nodes + 4 * node).w), c1 = __float_as_int(__ldcg(nodes + 4 * node + 2).w);
        float3 lo0, hi0, lo1, hi1;
        child_box(nodes, mo, c0, lo0, hi0);
        child_box(nodes, mo, c1, lo1, hi1);
        __stcg(nodes + 4 * node + 0, make_float4(lo0.x, lo0.y, lo0.z, __int_as_float(c0)));
        __stcg(nodes + 4 * node + 1, make_float4(hi0.x, hi0.y, hi0.z, 0.f));
        __stcg(nodes + 4 * node + 2, make_float4(lo1.x, lo1.y, lo1.z, __int_as_float(c1)));
        __stcg(nodes + 4 * node + 3, make_float4(hi1.x, hi1.y, hi1.z, 0.f));
        node = parent[node];
    }
}

// Bottom-up boxes: the second child to finish a node computes its child boxes.
__global__ void __launch_bounds__(kRegThreads) k_bvh_refit(int n, const float4* __restrict__ mo,
                                                          const uint32_t* __restrict__ acc,
                                                          const uint32_t* __restrict__ use_bvh,
                                                          float4* __restrict__ nodes_all,
                                                          const int32_t* __restrict__ parent_all,
                                                          uint32_t* __restrict__ flag_all, uint32_t* __restrict__ status)
{
    const int c = blockIdx.y;
    if (!use_bvh[c]) return;
    const long long m = acc[8 * (c + 1) + 6];
    float4* nodes = nodes_all + (size_t)c * n * 4;
    const int32_t* parent = parent_all + (size_t)c * 2 * n;
    uint32_t* flag = flag_all + (size_t)c * n;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (long long)gridDim.x * blockDim.x)
        bvh_refit_leaf(n, mo, nodes, parent, flag, status, k);
}

// Lower bound of the pinned FP32 distance from q to any point of the box [lo, hi]:
// the same operations on per-axis gaps, which no member's |offset| undercuts.
__device__ __forceinline__ float box_dist2(float qx, float qy, float qz, float4 lo, float4 hi)
{
    const float gx = fmaxf(fmaxf(__fsub_rn(lo.x, qx), __fsub_rn(qx, hi.x)), 0.f);
    const float gy = fmaxf(fmaxf(__fsub_rn(lo.y, qy), __fsub_rn(qy, hi.y)), 0.f);
    const float gz = fmaxf(fmaxf(__fsub_rn(lo.z, qz), __fsub_rn(qz, hi.z)), 0.f);
    return __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
}

// Query qp (position, index bits): its k nearest members by the BVH of m >= 2
// members.
template <int KMAX>
__device__ __forceinline__ void knn_bvh_query(float4 qp, int k, long long m, const float4* __restrict__ nodes,
                                              int32_t* __restrict__ nbr, uint32_t* __restrict__ status)
{
    const float qx = qp.x, qy = qp.y, qz = qp.z;
    const int self = __float_as_int(qp.w);
    float bd[KMAX];
    int bi[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        bd[j] = INFINITY;
        bi[j] = INT_MAX;
    }
    int stk[kBvhStack];
    float stkd[kBvhStack];
    int sp = 0;
    int cur = 0;                                   // the root (members >= 2)
    const long long max_visits = 2 * m + 8;        // each internal node at most once
    for (long long visit = 0;; ++visit) {
        if (visit > max_visits) {
            atomicOr(status, kStatusInternal);
            break;
        }
        float kth = INFINITY;
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
            if (j == k - 1) kth = bd[j];
        const float4 a = __ldg(nodes + 4 * cur), b = __ldg(nodes + 4 * cur + 1);
        const float4 e = __ldg(nodes + 4 * cur + 2), f = __ldg(nodes + 4 * cur + 3);
        const int c0 = __float_as_int(a.w), c1 = __float_as_int(e.w);
        const float d0 = box_dist2(qx, qy, qz, a, b), d1 = box_dist2(qx, qy, qz, e, f);
        // a member child is its own box: its box distance is its distance
        if (c0 < 0 && -(c0 + 1) != self) insert<KMAX>(bd, bi, d0, -(c0 + 1));
        if (c1 < 0 && -(c1 + 1) != self) insert<KMAX>(bd, bi, d1, -(c1 + 1));
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
            if (j == k - 1) kth = bd[j];
        const bool v0 = c0 >= 0 && d0 <= kth, v1 = c1 >= 0 && d1 <= kth;
        if (v0 && v1) {
            const bool first0 = d0 <= d1;
            if (sp < kBvhStack) {
                stk[sp] = first0 ? c1 : c0;
                stkd[sp] = first0 ? d1 : d0;
                ++sp;
            } else {
                atomicOr(status, kStatusInternal);   // cannot happen for trees of depth < 64
            }
            cur = first0 ? c0 : c1;
            continue;
        }
        if (v0) { cur = c0; continue; }
        if (v1) { cur = c1; continue; }
        bool found = false;
        while (sp > 0) {
            --sp;
            if (stkd[sp] <= kth) {
                cur = stk[sp];
                found = true;
                break;
            }
        }
        if (!found) break;
    }
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
        if (j < k) nbr[(size_t)self * k + j] = bi[j] == INT_MAX ? -1 : bi[j];
}

// Queries in the cell order of grid 0; k nearest members of set y by the BVH.
template <int KMAX>
__global__ void __launch_bounds__(kRegThreads) k_knn_bvh(int n, int k, const uint32_t* __restrict__ acc,
                                                        const uint32_t* __restrict__ use_bvh,
                                                        const float4* __restrict__ sorted,
                                                        const float4* __restrict__ nodes_all,
                                                        int32_t* __restrict__ nbr0, int32_t* __restrict__ nbr1,
                                                        uint32_t* __restrict__ status)
{
    const int c = blockIdx.y;
    if (!use_bvh[c]) return;
    const long long m = acc[8 * (c + 1) + 6];
    const float4* __restrict__ nodes = nodes_all + (size_t)c * n * 4;
    int32_t* __restrict__ nbr = c == 0 ? nbr0 : nbr1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        knn_bvh_query<KMAX>(sorted[t], k, m, nodes, nbr, status);
}

// ----------------------------------------------------------------- rotations

struct M3 {
    float a[3][3];
};

__device__ __forceinline__ M3 rot_of_quat(float4 q)
{
    const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
    M3 R;
    R.a[0][0] = 1.f - 2.f * (y * y + z * z); R.a[0][1] = 2.f * (x * y - w * z); R.a[0][2] = 2.f * (x * z + w * y);
    R.a[1][0] = 2.f * (x * y + w * z); R.a[1][1] = 1.f - 2.f * (x * x + z * z); R.a[1][2] = 2.f * (y * z - w * x);
    R.a[2][0] = 2.f * (x * z - w * y); R.a[2][1] = 2.f * (y * z + w * x); R.a[2][2] = 1.f - 2.f * (x * x + y * y);
    return R;
}

// dR = Rz(ez) Ry(ey) Rx(ex): dR20 = -sin ey, dR21 = cos ey sin ex, dR22 = cos ey cos ex,
// dR10 = sin ez cos ey, dR00 = cos ez cos ey.
__device__ __forceinline__ float3 euler_of(const M3& D)
{
    const float sb = fminf(fmaxf(-D.a[2][0], -1.0f), 1.0f);
    return make_float3(atan2f(D.a[2][1], D.a[2][2]), asinf(sb), atan2f(D.a[1][0], D.a[0][0]));
}

__device__ __forceinline__ M3 rot_of_euler(float3 e)
{
    float sa, ca, sb, cb, sc, cc;
    sincosf(e.x, &sa, &ca);
    sincosf(e.y, &sb, &cb);
    sincosf(e.z, &sc, &cc);
    M3 R;
    R.a[0][0] = cc * cb; R.a[0][1] = cc * sb * sa - sc * ca; R.a[0][2] = cc * sb * ca + sc * sa;
    R.a[1][0] = sc * cb; R.a[1][1] = sc * sb * sa + cc * ca; R.a[1][2] = sc * sb * ca - cc * sa;
    R.a[2][0] = -sb;     R.a[2][1] = cb * sa;                R.a[2][2] = cb * ca;
    return R;
}

// unit quaternion (w, x, y, z) of a rotation matrix; the branch is the largest of
// 1 + trace and 1 + 2 R_kk - trace
__device__ __forceinline__ float4 quat_of_rot(const M3& R)
{
    const float tr = R.a[0][0] + R.a[1][1] + R.a[2][2];
    float4 q;
    if (tr >= R.a[0][0] && tr >= R.a[1][1] && tr >= R.a[2][2]) {
        const float h = 2.f * sqrtf(1.f + tr), ih = 1.f / h;
        q = make_float4(0.25f * h, (R.a[2][1] - R.a[1][2]) * ih, (R.a[0][2] - R.a[2][0]) * ih,
                        (R.a[1][0] - R.a[0][1]) * ih);
    } else if (R.a[0][0] >= R.a[1][1] && R.a[0][0] >= R.a[2][2]) {
        const float h = 2.f * sqrtf(1.f + R.a[0][0] - R.a[1][1] - R.a[2][2]), ih = 1.f / h;
        q = make_float4((R.a[2][1] - R.a[1][2]) * ih, 0.25f * h, (R.a[0][1] + R.a[1][0]) * ih,
                        (R.a[0][2] + R.a[2][0]) * ih);
    } else if (R.a[1][1] >= R.a[2][2]) {
        const float h = 2.f * sqrtf(1.f - R.a[0][0] + R.a[1][1] - R.a[2][2]), ih = 1.f / h;
        q = make_float4((R.a[0][2] - R.a[2][0]) * ih, (R.a[0][1] + R.a[1][0]) * ih, 0.25f * h,
                        (R.a[1][2] + R.a[2][1]) * ih);
    } else {
        const float h = 2.f * sqrtf(1.f - R.a[0][0] - R.a[1][1] + R.a[2][2]), ih = 1.f / h;
        q = make_float4((R.a[1][0] - R.a[0][1]) * ih, (R.a[0][2] + R.a[2][0]) * ih, (R.a[1][2] + R.a[2][1]) * ih,
                        0.25f * h);
    }
    const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    return make_float4(q.x * inv, q.y * inv, q.z * inv, q.w * inv);
}

// --------------------------------------------------------------- the three passes

constexpr uint8_t kPosMember = 1, kCovMember = 2, kStatic = 4;

// Static flags, component membership and the motion components.
__global__ void __launch_bounds__(kRegThreads) k_reg_prepare(RegParams rp)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= rp.n) return;
    // slots 12-15 of each view's record (pixels in .y, static pixels in .z),
    // eight views' loads in flight at a time
    int views = 0;
    const float4* rec = reinterpret_cast<const float4*>(rp.moments) + (size_t)g * 4 + 3;
    const size_t vstride = (size_t)rp.n * 4;
    for (int v0 = 0; v0 < rp.V; v0 += 8) {
        float4 c[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) c[j] = v0 + j < rp.V ? __ldcs(rec + (size_t)(v0 + j) * vstride) : float4{};
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (v0 + j < rp.V && c[j].y > rp.min_px && c[j].z > __fmul_rn(rp.frac, c[j].y)) ++views;
    }
    const bool is_static = views >= rp.min_views;
    const uint32_t st = rp.status[g];
    uint8_t m = is_static ? kStatic : 0;
    if (!is_static && (st & TSP_POS_OK)) m |= kPosMember;
    if (!is_static && (st & TSP_COV_OK)) m |= kCovMember;
    rp.mask[g] = m;
    const float4 a = rp.mo0[g], b = rp.mo1[g];
    rp.dpos[g] = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, 0.f);
    const float4 sa = rp.s0[g], sb = rp.s1[g];
    rp.dscale[g] = make_float4(sb.x - sa.x, sb.y - sa.y, sb.z - sa.z, 0.f);
    const M3 Ra = rot_of_quat(rp.q0[g]), Rb = rot_of_quat(rp.q1[g]);
    M3 D;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            D.a[i][j] = Rb.a[i][0] * Ra.a[j][0] + Rb.a[i][1] * Ra.a[j][1] + Rb.a[i][2] * Ra.a[j][2];
    const float3 e = euler_of(D);
    rp.drot[g] = make_float4(e.x, e.y, e.z, 0.f);
}

// Median of the first cnt of v[0..S) (the rest +inf), by an odd-even transposition
// network over all S slots.
template <int S>
__device__ __forceinline__ float median_sorted(float (&v)[S], int cnt)
{
#pragma unroll
    for (int pass = 0; pass < S; ++pass) {
#pragma unroll
        for (int i = pass & 1; i + 1 < S; i += 2) {
            const float a = fminf(v[i], v[i + 1]), b = fmaxf(v[i], v[i + 1]);
            v[i] = a;
            v[i + 1] = b;
        }
    }
    const int i0 = (cnt - 1) >> 1, i1 = cnt >> 1;
    float lo = 0.f, hi = 0.f;
#pragma unroll
    for (int i = 0; i < S; ++i) {
        if (i == i0) lo = v[i];
        if (i == i1) hi = v[i];
    }
    return (cnt & 1) ? lo : 0.5f * (lo + hi);
}

__device__ __forceinline__ void order2(float& a, float& b)
{
    const float lo = fminf(a, b), hi = fmaxf(a, b);
    a = lo;
    b = hi;
}

__device__ __forceinline__ float median3(float a, float b, float c)
{
    return fmaxf(fminf(a, b), fminf(fmaxf(a, b), c));
}

// Median of exactly nine values: sort each of the three triples; the median of the
// nine is the median of (largest of the three minima, median of the three
// medians, smallest of the three maxima).
__device__ __forceinline__ float median9(float (&v)[9])
{
#pragma unroll
    for (int t = 0; t < 9; t += 3) {
        order2(v[t], v[t + 1]);
        order2(v[t + 1], v[t + 2]);
        order2(v[t], v[t + 1]);
    }
    const float lo = fmaxf(fmaxf(v[0], v[3]), v[6]);
    const float mid = median3(v[1], v[4], v[7]);
    const float hi = fminf(fminf(v[2], v[5]), v[8]);
    return median3(lo, mid, hi);
}

template <int S>
__device__ __forceinline__ float median_of(float (&v)[S], int cnt)
{
    if constexpr (S == 9) {
        if (cnt == 9) return median9(v);
    }
    return median_sorted<S>(v, cnt);
}

template <int KMAX>
__device__ __forceinline__ int neighbours(const int32_t* __restrict__ nbr, int k, int g, int (&nb)[KMAX])
{
    int m = 0;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        nb[j] = j < k ? nbr[(size_t)g * k + j] : -1;
        if (nb[j] >= 0) m = j + 1;
    }
    return m;
}

// Coordinate-wise median of src over g and its m neighbours, into dst[g].
template <int KMAX>
__device__ __forceinline__ void median_filter(const float4* __restrict__ src, float4* __restrict__ dst, int g,
                                              const int (&nb)[KMAX], int m)
{
    float4 x[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
        x[j] = j < m ? src[nb[j]] : make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
    const float4 self = src[g];
    float v[KMAX + 1];
    float out[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[0] = c == 0 ? self.x : (c == 1 ? self.y : self.z);
#pragma unroll
        for (int j = 0; j < KMAX; ++j) v[j + 1] = c == 0 ? x[j].x : (c == 1 ? x[j].y : x[j].z);
        out[c] = median_of<KMAX + 1>(v, m + 1);
    }
    dst[g] = make_float4(out[0], out[1], out[2], 0.f);
}

// Pass 1: every Gaussian with a component takes the median over itself and its
// neighbours with the component.  Threads take the Gaussians in cell order, so a
// warp's neighbours overlap.
template <int KMAX>
__global__ void __launch_bounds__(kRegThreads) k_reg_median(RegParams rp)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rp.n) return;
    const int g = __float_as_int(rp.qorder[t].w);
    const uint8_t m8 = rp.mask[g];
    int nb[KMAX];
    if (m8 & kPosMember) {
        const int m = neighbours<KMAX>(rp.nbr_pos, rp.k, g, nb);
        median_filter<KMAX>(rp.dpos, rp.fpos, g, nb, m);
    }
    if (m8 & kCovMember) {
        const int m = neighbours<KMAX>(rp.nbr_cov, rp.k, g, nb);
        median_filter<KMAX>(rp.dscale, rp.fscale, g, nb, m);
        median_filter<KMAX>(rp.drot, rp.frot, g, nb, m);
    }
}

// Pass 2: propagation of the filtered components and the new parameters.
template <int KMAX>
__global__ void __launch_bounds__(kRegThreads) k_reg_apply(RegParams rp)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rp.n) return;
    const int g = __float_as_int(rp.qorder[t].w);
    const uint8_t m8 = rp.mask[g];
    uint32_t fl = (m8 & kStatic) ? TSP_REG_STATIC : 0u;
    float4 dp = make_float4(0.f, 0.f, 0.f, 0.f), ds = dp, dr = dp;
    int nb[KMAX];
    if (!(m8 & kStatic)) {
        if (m8 & kPosMember) {
            dp = rp.fpos[g];
            fl |= TSP_REG_POS_MEDIAN;
        } else {
            const int m = neighbours<KMAX>(rp.nbr_pos, rp.k, g, nb);
            if (m > 0) {
#pragma unroll
                for (int j = 0; j < KMAX; ++j)
                    if (j < m) {
                        const float4 f = rp.fpos[nb[j]];
                        dp.x += f.x; dp.y += f.y; dp.z += f.z;
                    }
                const float im = 1.0f / (float)m;
                dp = make_float4(dp.x * im, dp.y * im, dp.z * im, 0.f);
                fl |= TSP_REG_POS_PROPAGATED;
            }
        }
        if (m8 & kCovMember) {
            ds = rp.fscale[g];
            dr = rp.frot[g];
            fl |= TSP_REG_COV_MEDIAN;
        } else {
            const int m = neighbours<KMAX>(rp.nbr_cov, rp.k, g, nb);
            if (m > 0) {
#pragma unroll
                for (int j = 0; j < KMAX; ++j)
                    if (j < m) {
                        const float4 a = rp.fscale[nb[j]], b = rp.frot[nb[j]];
                        ds.x += a.x; ds.y += a.y; ds.z += a.z;
                        dr.x += b.x; dr.y += b.y; dr.z += b.z;
                    }
                const float im = 1.0f / (float)m;
                ds = make_float4(ds.x * im, ds.y * im, ds.z * im, 0.f);
                dr = make_float4(dr.x * im, dr.y * im, dr.z * im, 0.f);
                fl |= TSP_REG_COV_PROPAGATED;
            }
        }
    }
    const float4 a = rp.mo0[g];
    rp.mo_out[g] = make_float4(a.x + dp.x, a.y + dp.y, a.z + dp.z, a.w);
    const float4 s = rp.s0[g];
    rp.s_out[g] = make_float4(s.x + ds.x, s.y + ds.y, s.z + ds.z, s.w);
    const float4 q0 = rp.q0[g];
    const M3 Ra = rot_of_quat(q0), E = rot_of_euler(make_float3(dr.x, dr.y, dr.z));
    M3 Rn;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Rn.a[i][j] = E.a[i][0] * Ra.a[0][j] + E.a[i][1] * Ra.a[1][j] + E.a[i][2] * Ra.a[2][j];
    float4 qn = quat_of_rot(Rn);
    if (qn.x * q0.x + qn.y * q0.y + qn.z * q0.z + qn.w * q0.w < 0.f) qn = make_float4(-qn.x, -qn.y, -qn.z, -qn.w);
    rp.q_out[g] = qn;
    rp.flags[g] = fl;
}

inline int blocks(int n) { return (n + kRegThreads - 1) / kRegThreads; }

}  // namespace

uint32_t knn_max_cells(int n) { return n / kMembersPerCell > 1 ? (uint32_t)(n / kMembersPerCell) : 1u; }

cudaError_t launch_knn(const float4* mo, const uint8_t* mask, const uint8_t* bits, int ncand, int n, int k,
                       const KnnWork& kw, int32_t* nbr0, int32_t* nbr1, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const uint32_t C = knn_max_cells(n);
    GridDesc gd{};
    gd.G = ncand + 1;
    gd.bits[0] = 0;                                   // grid 0: every point, the query order
    for (int j = 0; j < ncand; ++j) gd.bits[j + 1] = bits[j];
    cudaError_t e;
    if ((e = cudaMemsetAsync(kw.zero, 0, kw.zero_bytes, st))) return e;
    k_grid_bounds<<<min(blocks(n), 4 * 148), kRegThreads, 0, st>>>(mo, mask, gd, n, kw.acc);
    k_grid_setup<<<1, 32, 0, st>>>(kw.acc, gd.G, C, kw.gp);
    k_grid_count<<<blocks(n), kRegThreads, 0, st>>>(mo, mask, gd, n, kw.gp, C, kw.count, kw.slot);
    if ((e = launch_scan_u32(kw.count, 1, (uint32_t)gd.G * C, kw.cell_off, kw.span_sum,
                             (uint32_t)gd.G * (uint32_t)n, kw.status, st)))
        return e;
    k_grid_scatter<<<blocks(n), kRegThreads, 0, st>>>(mo, mask, gd, n, kw.slot, C, kw.cell_off, kw.sorted);
    // grid or BVH per candidate set, decided on the device
    if ((e = cudaMemsetAsync(kw.bvh_zero, 0, kw.bvh_zero_bytes, st))) return e;
    k_grid_skew<<<dim3(min((int)((C + kRegThreads - 1) / kRegThreads), 4 * 148), ncand), kRegThreads, 0, st>>>(
        kw.count, C, kw.skew);
    k_bvh_decide<<<1, 32, 0, st>>>(kw.acc, kw.skew, ncand, kw.use_bvh);
    const dim3 grid(blocks(n), ncand);
    if (k <= 8)
        k_knn<8><<<grid, kRegThreads, 0, st>>>(n, k, kw.gp, C, kw.cell_off, kw.sorted, nbr0, nbr1, kw.use_bvh);
    else
        k_knn<16><<<grid, kRegThreads, 0, st>>>(n, k, kw.gp, C, kw.cell_off, kw.sorted, nbr0, nbr1, kw.use_bvh);
    // the BVH path: small grid-stride grids, every kernel returns at once unless a
    // set needs it (use_bvh[2] gates the generic scan and sort)
    const dim3 bgrid(min(blocks(n), 8 * 148), ncand);
    const uint32_t* any = kw.use_bvh + 2;
    k_bvh_codes<<<bgrid, kRegThreads, 0, st>>>(mo, mask, gd, n, kw.acc, kw.use_bvh, kw.bcount, kw.bslot);
    const uint32_t nb = (uint32_t)ncand * kMortonBuckets;
    if ((e = launch_scan_u32(kw.bcount, 1, nb, kw.boff, kw.bspan, (uint32_t)ncand * (uint32_t)n, kw.bstatus, st,
                             any)))
        return e;
    k_bvh_scatter<<<bgrid, kRegThreads, 0, st>>>(mo, mask, gd, n, kw.acc, kw.use_bvh, kw.bslot, kw.boff, kw.keys);
    if ((e = launch_segment_sort(kw.boff, kw.keys, kw.keys_tmp, (uint32_t)ncand * (uint32_t)n, nb, kw.long_list,
                                 kw.long_count, st, any)))
        return e;
    k_bvh_build<<<bgrid, kRegThreads, 0, st>>>(n, kw.acc, kw.use_bvh, kw.boff, kw.keys, kw.nodes, kw.parent);
    k_bvh_refit<<<bgrid, kRegThreads, 0, st>>>(n, mo, kw.acc, kw.use_bvh, kw.nodes, kw.parent, kw.flag, kw.err);
    if (k <= 8)
        k_knn_bvh<8><<<bgrid, kRegThreads, 0, st>>>(n, k, kw.acc, kw.use_bvh, kw.sorted, kw.nodes, nbr0, nbr1,
                                                    kw.err);
    else
        k_knn_bvh<16><<<bgrid, kRegThreads, 0, st>>>(n, k, kw.acc, kw.use_bvh, kw.sorted, kw.nodes, nbr0, nbr1,
                                                     kw.err);
    return cudaGetLastError();
}

cudaError_t launch_regularize(const RegParams& rp, const KnnWork& kw, cudaStream_t st)
{
    if (rp.n <= 0) return cudaSuccess;
    k_reg_prepare<<<blocks(rp.n), kRegThreads, 0, st>>>(rp);
    cudaError_t e;
    const uint8_t bits[2] = {kPosMember, kCovMember};
    if ((e = launch_knn(rp.mo0, rp.mask, bits, 2, rp.n, rp.k, kw, rp.nbr_pos, rp.nbr_cov, st))) return e;
    RegParams r2 = rp;
    r2.qorder = kw.sorted;                             // grid 0: every Gaussian in cell order
    if (rp.k <= 8) {
        k_reg_median<8><<<blocks(rp.n), kRegThreads, 0, st>>>(r2);
        k_reg_apply<8><<<blocks(rp.n), kRegThreads, 0, st>>>(r2);
    } else {
        k_reg_median<16><<<blocks(rp.n), kRegThreads, 0, st>>>(r2);
        k_reg_apply<16><<<blocks(rp.n), kRegThreads, 0, st>>>(r2);
    }
    return cudaGetLastError();
}

}  // namespace tsp

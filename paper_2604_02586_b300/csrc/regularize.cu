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
#include <cfloat>
#include <cmath>

#include "launch.h"

namespace tsp {
namespace {

constexpr int kRegThreads = 256;

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

__device__ __forceinline__ bool member(const uint8_t* mask, uint8_t bit, int g) { return (mask[g] & bit) != 0; }

// acc: [0..2] ~key(min), [3..5] key(max), [6] member count; all start at 0.
__global__ void __launch_bounds__(kRegThreads) k_grid_bounds(const float4* __restrict__ mo,
                                                            const uint8_t* __restrict__ mask, uint8_t bit, int n,
                                                            uint32_t* __restrict__ acc)
{
    __shared__ uint32_t s[7][kRegThreads / 32];
    uint32_t v[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        if (!member(mask, bit, g)) continue;
        const float4 p = mo[g];
        const float c[3] = {p.x, p.y, p.z};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const uint32_t k = ordered_key(c[i]);
            v[i] = max(v[i], ~k);
            v[3 + i] = max(v[3 + i], k);
        }
        v[6] += 1;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        uint32_t x = v[i];
        for (int o = 16; o > 0; o >>= 1) {
            const uint32_t y = __shfl_xor_sync(0xffffffffu, x, o);
            x = i == 6 ? x + y : max(x, y);
        }
        if (lane == 0) s[i][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        const int i = threadIdx.x;
        uint32_t x = 0;
        for (int w = 0; w < kRegThreads / 32; ++w) x = i == 6 ? x + s[i][w] : max(x, s[i][w]);
        if (i == 6) {
            if (x) atomicAdd(&acc[6], x);
        } else {
            atomicMax(&acc[i], x);
        }
    }
}

// One thread: the grid over the members' box with about two members per cell and
// at most max_cells cells.
__global__ void k_grid_setup(const uint32_t* __restrict__ acc, uint32_t max_cells, GridParam* __restrict__ gp)
{
    if (threadIdx.x != 0) return;
    const uint32_t m = acc[6];
    double lo[3], ext[3], E = 0.0, amax = 0.0;
    for (int i = 0; i < 3; ++i) {
        if (m == 0) {
            lo[i] = 0.0;
            ext[i] = 1.0;
        } else {
            lo[i] = key_value(~acc[i]);
            const double hi = key_value(acc[3 + i]);
            ext[i] = hi - lo[i];
            amax = fmax(amax, fmax(fabs(lo[i]), fabs(hi)));
        }
        if (!(ext[i] < 1e30)) ext[i] = 1.0;
        E = fmax(E, ext[i]);
    }
    if (!(E > 0.0)) E = 1.0;
    for (int i = 0; i < 3; ++i) ext[i] = fmax(ext[i], 1e-3 * E);
    double target = fmax(1.0, floor(m / 2.0));
    if (target > max_cells) target = max_cells;
    // cubic cells; an axis shorter than one cell gets one cell and the others
    // share the count
    int d[3] = {0, 0, 0};
    for (int round = 0; round < 3; ++round) {
        double vol = 1.0;
        int free_axes = 0;
        for (int i = 0; i < 3; ++i)
            if (d[i] == 0) {
                vol *= ext[i];
                ++free_axes;
            }
        if (free_axes == 0) break;
        const double h = pow(vol / target, 1.0 / free_axes);
        bool fixed = false;
        for (int i = 0; i < 3; ++i)
            if (d[i] == 0 && ext[i] < h) {
                d[i] = 1;
                fixed = true;
            }
        if (!fixed) {
            for (int i = 0; i < 3; ++i)
                if (d[i] == 0) d[i] = (int)fmin(fmax(floor(ext[i] / h), 1.0), 1048576.0);
            break;
        }
    }
    for (int i = 0; i < 3; ++i) d[i] = d[i] > 0 ? d[i] : 1;
    while ((unsigned long long)d[0] * d[1] * d[2] > max_cells) {
        int j = d[0] >= d[1] && d[0] >= d[2] ? 0 : (d[1] >= d[2] ? 1 : 2);
        d[j] -= 1;
    }
    for (int i = 0; i < 3; ++i) {
        gp->lo[i] = (float)lo[i];
        gp->inv[i] = (float)(d[i] / ext[i]);
        gp->h[i] = (float)(ext[i] / d[i]);
        gp->dims[i] = d[i];
    }
    gp->ncell = d[0] * d[1] * d[2];
    // covers the FP32 rounding of (x - lo) * inv and of the cell walls
    gp->margin = (float)(1e-5 * E + 1e-6 * amax);
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

__global__ void __launch_bounds__(kRegThreads) k_grid_count(const float4* __restrict__ mo,
                                                           const uint8_t* __restrict__ mask, uint8_t bit, int n,
                                                           const GridParam* __restrict__ gpp,
                                                           uint32_t* __restrict__ count, uint2* __restrict__ slot)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n || !member(mask, bit, g)) return;
    const GridParam gp = *gpp;
    const float4 p = mo[g];
    int cx, cy, cz;
    cell_of(gp, p.x, p.y, p.z, cx, cy, cz);
    const uint32_t c = ((uint32_t)cz * gp.dims[1] + cy) * gp.dims[0] + cx;
    slot[g] = make_uint2(c, atomicAdd(&count[c], 1u));
}

__global__ void __launch_bounds__(kRegThreads) k_grid_scatter(const float4* __restrict__ mo,
                                                             const uint8_t* __restrict__ mask, uint8_t bit, int n,
                                                             const uint2* __restrict__ slot,
                                                             const uint32_t* __restrict__ cell_off,
                                                             float4* __restrict__ sorted)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n || !member(mask, bit, g)) return;
    const uint2 s = slot[g];
    const float4 p = mo[g];
    sorted[cell_off[s.x] + s.y] = make_float4(p.x, p.y, p.z, __int_as_float(g));
}

// (d, i) before (bd, bi)?
__device__ __forceinline__ bool closer(float d, int i, float bd, int bi) { return d < bd || (d == bd && i < bi); }

template <int KMAX>
__device__ __forceinline__ void insert(float (&bd)[KMAX], int (&bi)[KMAX], float d, int i)
{
    if (!closer(d, i, bd[KMAX - 1], bi[KMAX - 1])) return;
#pragma unroll
    for (int j = KMAX - 1; j > 0; --j) {
        const bool before_prev = closer(d, i, bd[j - 1], bi[j - 1]);
        const bool before_this = closer(d, i, bd[j], bi[j]);
        const float nd = before_prev ? bd[j - 1] : (before_this ? d : bd[j]);
        const int ni = before_prev ? bi[j - 1] : (before_this ? i : bi[j]);
        bd[j] = nd;
        bi[j] = ni;
    }
    if (closer(d, i, bd[0], bi[0])) {
        bd[0] = d;
        bi[0] = i;
    }
}

template <int KMAX>
__device__ __forceinline__ void scan_range(const float4* __restrict__ sorted, uint32_t a, uint32_t b, int self,
                                           float qx, float qy, float qz, float (&bd)[KMAX], int (&bi)[KMAX])
{
    for (uint32_t j = a; j < b; ++j) {
        const float4 p = sorted[j];
        const int idx = __float_as_int(p.w);
        if (idx == self) continue;
        insert<KMAX>(bd, bi, dist2(qx, qy, qz, p), idx);
    }
}

// One thread per query: its k nearest members (k <= KMAX), -1 padded.
template <int KMAX>
__global__ void __launch_bounds__(kRegThreads) k_knn(const float4* __restrict__ mo, int n, int k,
                                                    const GridParam* __restrict__ gpp,
                                                    const uint32_t* __restrict__ cell_off,
                                                    const float4* __restrict__ sorted, int32_t* __restrict__ nbr)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const GridParam gp = *gpp;
    const float4 q = mo[g];
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
    for (int r = 0; r <= rmax; ++r) {
        const int z0 = max(c[2] - r, 0), z1 = min(c[2] + r, d2 - 1);
        const int y0 = max(c[1] - r, 0), y1 = min(c[1] + r, d1 - 1);
        const int x0 = max(c[0] - r, 0), x1 = min(c[0] + r, d0 - 1);
        for (int z = z0; z <= z1; ++z) {
            for (int y = y0; y <= y1; ++y) {
                const uint32_t row = ((uint32_t)z * d1 + y) * d0;
                if (abs(z - c[2]) == r || abs(y - c[1]) == r) {
                    scan_range<KMAX>(sorted, cell_off[row + x0], cell_off[row + x1 + 1], g, q.x, q.y, q.z, bd, bi);
                } else {
                    if (c[0] - r >= 0)
                        scan_range<KMAX>(sorted, cell_off[row + c[0] - r], cell_off[row + c[0] - r + 1], g, q.x,
                                         q.y, q.z, bd, bi);
                    if (r > 0 && c[0] + r < d0)
                        scan_range<KMAX>(sorted, cell_off[row + c[0] + r], cell_off[row + c[0] + r + 1], g, q.x,
                                         q.y, q.z, bd, bi);
                }
            }
        }
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
        if (b > 0.0f && kth < b * b * (1.0f - 1e-6f)) break;
    }
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
        if (j < k) nbr[(size_t)g * k + j] = bi[j] == INT_MAX ? -1 : bi[j];
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
    int views = 0;
    for (int v = 0; v < rp.V; ++v) {
        const float* rec = rp.moments + ((size_t)v * rp.n + g) * 16;
        const float npix = rec[13], nstat = rec[14];
        if (npix > rp.min_px && nstat > __fmul_rn(rp.frac, npix)) ++views;
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
__device__ __forceinline__ float median_of(float (&v)[S], int cnt)
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

// Pass 1: every Gaussian with a component takes the median over itself and its
// neighbours with the component.
template <int KMAX>
__global__ void __launch_bounds__(kRegThreads) k_reg_median(RegParams rp)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= rp.n) return;
    const uint8_t m8 = rp.mask[g];
    int nb[KMAX];
    for (int part = 0; part < 2; ++part) {
        if (!(m8 & (part == 0 ? kPosMember : kCovMember))) continue;
        const int m = neighbours<KMAX>(part == 0 ? rp.nbr_pos : rp.nbr_cov, rp.k, g, nb);
        const int dim = part == 0 ? 3 : 6;
        for (int c = 0; c < dim; ++c) {
            const float* src = reinterpret_cast<const float*>(part == 0 ? rp.dpos : (c < 3 ? rp.dscale : rp.drot));
            const int cc = c % 3;
            float v[KMAX + 1];
            v[0] = src[4 * (size_t)g + cc];
#pragma unroll
            for (int j = 0; j < KMAX; ++j) v[j + 1] = j < m ? src[4 * (size_t)nb[j] + cc] : INFINITY;
            float* dst = reinterpret_cast<float*>(part == 0 ? rp.fpos : (c < 3 ? rp.fscale : rp.frot));
            dst[4 * (size_t)g + cc] = median_of<KMAX + 1>(v, m + 1);
        }
    }
}

// Pass 2: propagation of the filtered components and the new parameters.
template <int KMAX>
__global__ void __launch_bounds__(kRegThreads) k_reg_apply(RegParams rp)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= rp.n) return;
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

uint32_t knn_max_cells(int n) { return n / 2 > 1 ? (uint32_t)(n / 2) : 1u; }

cudaError_t launch_knn(const float4* mo, const uint8_t* mask, uint8_t bit, int n, int k, const KnnWork& kw,
                       int32_t* nbr, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const uint32_t C = knn_max_cells(n);
    cudaError_t e;
    if ((e = cudaMemsetAsync(kw.acc, 0, 8 * sizeof(uint32_t), st))) return e;
    if ((e = cudaMemsetAsync(kw.count, 0, ((size_t)C + 1) * sizeof(uint32_t), st))) return e;
    k_grid_bounds<<<min(blocks(n), 4 * 148), kRegThreads, 0, st>>>(mo, mask, bit, n, kw.acc);
    k_grid_setup<<<1, 32, 0, st>>>(kw.acc, C, kw.gp);
    k_grid_count<<<blocks(n), kRegThreads, 0, st>>>(mo, mask, bit, n, kw.gp, kw.count, kw.slot);
    if ((e = launch_scan_u32(kw.count, 1, C, kw.cell_off, kw.span_sum, (uint32_t)n, kw.status, st))) return e;
    k_grid_scatter<<<blocks(n), kRegThreads, 0, st>>>(mo, mask, bit, n, kw.slot, kw.cell_off, kw.sorted);
    if (k <= 8)
        k_knn<8><<<blocks(n), kRegThreads, 0, st>>>(mo, n, k, kw.gp, kw.cell_off, kw.sorted, nbr);
    else
        k_knn<16><<<blocks(n), kRegThreads, 0, st>>>(mo, n, k, kw.gp, kw.cell_off, kw.sorted, nbr);
    return cudaGetLastError();
}

cudaError_t launch_regularize(const RegParams& rp, const KnnWork& kw, cudaStream_t st)
{
    if (rp.n <= 0) return cudaSuccess;
    k_reg_prepare<<<blocks(rp.n), kRegThreads, 0, st>>>(rp);
    cudaError_t e;
    if ((e = launch_knn(rp.mo0, rp.mask, kPosMember, rp.n, rp.k, kw, rp.nbr_pos, st))) return e;
    if ((e = launch_knn(rp.mo0, rp.mask, kCovMember, rp.n, rp.k, kw, rp.nbr_cov, st))) return e;
    if (rp.k <= 8) {
        k_reg_median<8><<<blocks(rp.n), kRegThreads, 0, st>>>(rp);
        k_reg_apply<8><<<blocks(rp.n), kRegThreads, 0, st>>>(rp);
    } else {
        k_reg_median<16><<<blocks(rp.n), kRegThreads, 0, st>>>(rp);
        k_reg_apply<16><<<blocks(rp.n), kRegThreads, 0, st>>>(rp);
    }
    return cudaGetLastError();
}

}  // namespace tsp

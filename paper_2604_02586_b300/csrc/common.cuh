// common.cuh -- types and device helpers shared by the libtsplat kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tsplat.h"
#include "checks.h"

namespace tsp {

constexpr int kTile = 16;                 // default raster tile edge (pixels); the
                                          // warp-shuffle variants support only 16 x 16
constexpr int kTilePx = kTile * kTile;    // pixels (and shuffle-variant threads) per tile
// Per-tile atomic counters sit 128 bytes apart: one L2 line (one slice) each, so
// the atomics of neighbouring hot tiles do not queue behind one another.
constexpr int kCounterStride = 32;
constexpr int kMaxViews = TSP_MAX_BATCH_VIEWS;   // view slots of one launch, all frames
constexpr int kMaxFrames = TSP_MAX_FRAMES;

struct DevCam {
    int W, H;
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
};

// Everything a kernel needs to know about the frames and views of one launch.
// Passed by value as a kernel parameter (about 16 KB, under the 32 KB limit), so
// no host->device copy is needed.  Views of all frames are numbered together;
// view v belongs to frame vframe[v], whose vn[v] Gaussians have their records
// (view, Gaussian) at vrec[v] + g.
struct ViewSet {
    int V;                                // view slots (all frames)
    int F;                                // frames
    int nmax;                             // largest Gaussian count of a frame
    int tw, th;                           // raster tile: 16 x 16 or 32 x 8 pixels (four 8x8 blocks)
    DevCam cam[kMaxViews];
    int tiles_x[kMaxViews];
    int tiles_y[kMaxViews];
    uint32_t toff[kMaxViews + 1];         // first global tile id of each view
    const float2* disp[kMaxViews];
    const uint8_t* vis[kMaxViews];
    int vframe[kMaxViews];
    int vn[kMaxViews];
    unsigned long long vrec[kMaxViews];
    int fview[kMaxFrames + 1];            // first view of each frame
    int fn[kMaxFrames];                   // Gaussians of each frame
    const float4* fmo[kMaxFrames];        // means + opacity, quaternions, scales
    const float4* fq[kMaxFrames];
    const float4* fs[kMaxFrames];
};

// Per-frame outputs of the motion fit (optional members may be null).
struct FrameOut {
    float4* means[kMaxFrames];
    float4* quats[kMaxFrames];
    float4* scales[kMaxFrames];
    uint32_t* status[kMaxFrames];
    float* view_affine[kMaxFrames];       // [views of the frame][n][6]
    uint32_t* view_flags[kMaxFrames];     // [views of the frame][n]
};

// Per-view output images of the colour render.
struct RenderOut {
    float* rgb[kMaxViews];
    float* T[kMaxViews];
};

// Workspace pointers (device), owned by the context.  Per-record arrays hold one
// entry per (view, Gaussian) of every frame ([R] below, R = sum of views x n).
struct Work {
    short4* rect;          // [R] tile rect x0 y0 x1 y1
    uint32_t* depth;       // [R] FP32 depth bits
    uint32_t* touched;     // [R]
    float4* rec;           // [R * 4] blend records (kRec*: one 64-byte block per record)
    uint32_t* oref;        // [R] pixel index of the moment origin (fit mode)
    float4* color;         // [R] render colour
    float4* moments;       // [R*4] 16 floats per (view, Gaussian)
    float4* vres0;         // [R] mu'_x, mu'_y, shift c_x, c_y
    float4* vres1;         // [R] B00, B01, B02, sum w   (Sigma_2D' = B B^T, B = A V)
    float4* vres3;         // [R] B10, B11, B12, 0
    uint2* vres2;          // [R] view flags, pixels
    uint32_t* tile_count;  // [NT * kCounterStride], tile t at t * kCounterStride
    uint32_t* tile_fill;   // [NT * kCounterStride] likewise; after the scatter: long-list tiles
    uint32_t* tile_off;    // [NT+1]
    uint64_t* pairs;       // [cap]
    uint64_t* pairs_tmp;   // [cap]
    uint32_t cap;
    uint32_t nt;           // tiles of the call
    uint32_t checked;      // 1: checked mode (bounds checks into dstatus)
    uint32_t gated;        // 1: a track gate precedes the track readers (tsp_set_track_gate)
    uint32_t* dstatus;     // [8]: 0 flags (bit 0 overflow, bit 1 internal, bit 2 check),
                           //      1 K (low 32 bits), 2 K high, 3 number of tiles whose
                           //      lists need the long-list sort, 4 first failed check
                           //      site, 5 failed checks
    unsigned long long* stats;  // [4] raster work counters (collect_stats only)
    unsigned long long* span_sum; // [ceil(NT / 1024)] tile-count scan scratch
    uint32_t* queue;       // [1] work-queue head of the persistent raster
};

// Inputs and outputs of the render backward.
constexpr int kGradStride = 12;   // floats per (view, Gaussian) 2D-gradient record (9 used)
struct RenderGrad {
    const float* rgb[kMaxViews];  // forward colour [H][W][3]
    const float* grad[kMaxViews]; // dL/dcolour [H][W][3]
    float* acc;                   // [R][kGradStride]: d mu_2D (2), d Q (00, 01, 11), d opacity, d colour (3)
    float4* g_means;              // [n] (dL/dmean xyz, dL/dopacity)
    float4* g_scales;             // [n] (dL/dscale xyz, 0)
    float4* g_quats;              // [n] dL/d(raw quaternion)
    float* g_sh;                  // [n][(deg+1)^2][3]
};

struct FitParams {
    float det_min, sumw_min_view, lam_min_px2, sumw_min_total, cov_rcond_min;
    int min_px_view, min_views, min_px_total;
};

constexpr uint32_t kStatusOverflow = 1u;
constexpr uint32_t kStatusInternal = 2u;   // a bounded device loop gave up (reported by tsp_sync)
constexpr uint32_t kStatusChecked = 4u;    // checked mode: an index left its buffer (reported by tsp_sync)
constexpr uint32_t kStatusGate = 8u;       // the track gate's wait ran out (reported by tsp_sync)

// A call whose track gate timed out computes nothing from the tracks on: the
// track readers and the output writers return at once.
__device__ __forceinline__ bool gate_closed(const Work& w)
{
    return w.gated && (w.dstatus[0] & kStatusGate) != 0u;
}

// Checked mode: record a failed bounds check (the caller skips the access).
__device__ __forceinline__ void check_failed(uint32_t* dstatus, uint32_t site)
{
    atomicOr(&dstatus[0], kStatusChecked);
    atomicCAS(&dstatus[4], 0u, site);
    atomicAdd(&dstatus[5], 1u);
}

// --------------------------------------------------------------------------
// Key path: culling, depth key and tile rectangle in FP32 with a fixed order of
// correctly rounded operations (every op spelled with an _rn intrinsic, so the
// compiler cannot contract or reorder).  The same sequence also yields the 2D
// covariance factor V = J W R(q) S (Eq. 1) used for blending and for Eq. 2.
// --------------------------------------------------------------------------
struct KeyProj {
    float mx, my;          // mu_2D
    float pz;              // camera depth
    float V0[3], V1[3];    // rows of J W R(q) S: Sigma_2D = V V^T (undilated)
    float a, b, c;         // undilated Sigma_2D entries
    int x0, y0, x1, y1;    // tile rectangle
};

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float ff(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float fd(float a, float b) { return __fdiv_rn(a, b); }

// Returns false if the Gaussian is culled or touches no tile in this view.
__device__ __forceinline__ bool key_project(const DevCam& c, float4 m, float4 q, float4 s,
                                            int tiles_x, int tiles_y, int tw, int th, KeyProj& o)
{
    const float* R = c.R;
    const float px = ff(R[0], m.x, ff(R[1], m.y, ff(R[2], m.z, c.t[0])));
    const float py = ff(R[3], m.x, ff(R[4], m.y, ff(R[5], m.z, c.t[1])));
    const float pz = ff(R[6], m.x, ff(R[7], m.y, ff(R[8], m.z, c.t[2])));
    if (!(pz > 0.2f)) return false;
    const float iz = fd(1.0f, pz);
    const float un = fm(px, iz), vn = fm(py, iz);
    const float limx = fm(1.3f, fd(fm(0.5f, __int2float_rn(c.W)), c.fx));
    const float limy = fm(1.3f, fd(fm(0.5f, __int2float_rn(c.H)), c.fy));
    if (!(fabsf(un) <= limx) || !(fabsf(vn) <= limy)) return false;
    o.mx = ff(c.fx, un, c.cx);
    o.my = ff(c.fy, vn, c.cy);
    o.pz = pz;

    const float n2 = ff(q.x, q.x, ff(q.y, q.y, ff(q.z, q.z, fm(q.w, q.w))));
    if (!(n2 > 0.0f)) return false;
    const float inv = fd(1.0f, __fsqrt_rn(n2));
    const float w = fm(q.x, inv), x = fm(q.y, inv), y = fm(q.z, inv), z = fm(q.w, inv);
    const float xx = fm(x, x), yy = fm(y, y), zz = fm(z, z);
    const float xy = fm(x, y), xz = fm(x, z), yz = fm(y, z);
    const float wx = fm(w, x), wy = fm(w, y), wz = fm(w, z);
    float Q[3][3];
    Q[0][0] = fs(1.0f, fm(2.0f, fa(yy, zz)));
    Q[0][1] = fm(2.0f, fs(xy, wz));
    Q[0][2] = fm(2.0f, fa(xz, wy));
    Q[1][0] = fm(2.0f, fa(xy, wz));
    Q[1][1] = fs(1.0f, fm(2.0f, fa(xx, zz)));
    Q[1][2] = fm(2.0f, fs(yz, wx));
    Q[2][0] = fm(2.0f, fs(xz, wy));
    Q[2][1] = fm(2.0f, fa(yz, wx));
    Q[2][2] = fs(1.0f, fm(2.0f, fa(xx, yy)));
    const float sc[3] = {s.x, s.y, s.z};
    float M[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[i][j] = fm(Q[i][j], sc[j]);

    const float j00 = fm(c.fx, iz), j02 = -fm(fm(c.fx, un), iz);
    const float j11 = fm(c.fy, iz), j12 = -fm(fm(c.fy, vn), iz);
    float T0[3], T1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T0[j] = ff(j00, R[j], fm(j02, R[6 + j]));
        T1[j] = ff(j11, R[3 + j], fm(j12, R[6 + j]));
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        o.V0[j] = ff(T0[0], M[0][j], ff(T0[1], M[1][j], fm(T0[2], M[2][j])));
        o.V1[j] = ff(T1[0], M[0][j], ff(T1[1], M[1][j], fm(T1[2], M[2][j])));
    }
    o.a = ff(o.V0[0], o.V0[0], ff(o.V0[1], o.V0[1], fm(o.V0[2], o.V0[2])));
    o.b = ff(o.V0[0], o.V1[0], ff(o.V0[1], o.V1[1], fm(o.V0[2], o.V1[2])));
    o.c = ff(o.V1[0], o.V1[0], ff(o.V1[1], o.V1[1], fm(o.V1[2], o.V1[2])));
    const float ad = fa(o.a, 0.3f), cd = fa(o.c, 0.3f);
    const float det = ff(ad, cd, -fm(o.b, o.b));
    if (!(det > 0.0f)) return false;
    const float mid = fm(0.5f, fa(ad, cd));
    const float disc = fmaxf(0.1f, ff(mid, mid, -det));
    const float lam = fa(mid, __fsqrt_rn(disc));
    const float r = ceilf(fm(3.0f, __fsqrt_rn(lam)));
    const float ftw = (float)tw, fth = (float)th;
    const float gx = __int2float_rn(tiles_x), gy = __int2float_rn(tiles_y);
    const float fx0 = fminf(fmaxf(floorf(fd(fs(o.mx, r), ftw)), 0.0f), gx);
    const float fx1 = fminf(fmaxf(fa(floorf(fd(fa(o.mx, r), ftw)), 1.0f), 0.0f), gx);
    const float fy0 = fminf(fmaxf(floorf(fd(fs(o.my, r), fth)), 0.0f), gy);
    const float fy1 = fminf(fmaxf(fa(floorf(fd(fa(o.my, r), fth)), 1.0f), 0.0f), gy);
    o.x0 = (int)fx0; o.x1 = (int)fx1; o.y0 = (int)fy0; o.y1 = (int)fy1;
    return o.x1 > o.x0 && o.y1 > o.y0;
}

// --------------------------------------------------------------------------
// Double-float arithmetic (Dekker / Knuth error-free transformations: TwoSum,
// TwoProd via FMA) for the projected mean.  An FP32 pixel coordinate near 1000
// carries ~6e-5 px of rounding, which moves alpha = o exp(-q/2) by ~1e-3 at the
// edge of a 0.6 px footprint; a (hi, lo) pair keeps the mean to ~1e-9 px.
// --------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// mu_2D of the mean m in camera c as (hi, lo) pairs: u = ux.x + ux.y.
__device__ __forceinline__ void mean2d_df(const DevCam& c, float4 m, float2& ux, float2& uy)
{
    const float* R = c.R;
    float ph[3], pl[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float p0, e0, p1, e1, p2, e2, s, f1, f2, f3;
        two_prod(R[3 * k], m.x, p0, e0);
        two_prod(R[3 * k + 1], m.y, p1, e1);
        two_prod(R[3 * k + 2], m.z, p2, e2);
        two_sum(p0, p1, s, f1);
        two_sum(s, p2, s, f2);
        two_sum(s, c.t[k], s, f3);
        const float lo = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, f1)), __fadd_rn(f2, f3));
        fast_two_sum(s, lo, ph[k], pl[k]);
    }
    const float f[2] = {c.fx, c.fy}, cc[2] = {c.cx, c.cy};
    float2 out[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        // q = p_k / p_z in double-float
        const float q1 = __fdiv_rn(ph[k], ph[2]);
        const float r = __fsub_rn(__fadd_rn(__fmaf_rn(-q1, ph[2], ph[k]), pl[k]), __fmul_rn(q1, pl[2]));
        const float q2 = __fdiv_rn(r, ph[2]);
        float qh, ql;
        fast_two_sum(q1, q2, qh, ql);
        // u = f q + c
        float a, ae, sm, se;
        two_prod(f[k], qh, a, ae);
        ae = __fmaf_rn(f[k], ql, ae);
        two_sum(a, cc[k], sm, se);
        float uh, ul;
        fast_two_sum(sm, __fadd_rn(se, ae), uh, ul);
        out[k] = make_float2(uh, ul);
    }
    ux = out[0];
    uy = out[1];
}

// Origin of a (view, Gaussian)'s moment sums: mu_2D clamped to the image
// rectangle [0, W] x [0, H].  Returns delta = origin - mu_2D.  When the centre
// lies off-image, only a sliver at the border is visible; sums taken about the
// far-away centre would lose 2-3 digits to cancellation in FP32.  The shift is
// formed from (rx, ry), the mean relative to the corner pixel (cx, cy) of its
// tile rectangle -- the value the raster stages -- so that a clamped origin
// lands on the border to a unit in the last place of the off-image distance,
// not of |mu_2D|.
__device__ __forceinline__ float2 moment_origin_shift(float2 ux, float2 uy, float rx, float ry, int cx, int cy,
                                                      int W, int H)
{
    const float x = ux.x + ux.y, y = uy.x + uy.y;
    const float dx = x < 0.f ? __fsub_rn((float)(0 - cx), rx) : (x > (float)W ? __fsub_rn((float)(W - cx), rx) : 0.f);
    const float dy = y < 0.f ? __fsub_rn((float)(0 - cy), ry) : (y > (float)H ? __fsub_rn((float)(H - cy), ry) : 0.f);
    return make_float2(dx, dy);
}

// sqrt(log2(e) / 2): with this factor folded into the Cholesky factor, the blend
// evaluates G = exp(-q/2) as exp2(-(z1^2 + z2^2)).
constexpr float kHalfLog2eSqrt = 0.84932180028801904f;

// Blend parameters in factor form.  The dilated covariance is the Gram matrix of
// the columns (V0, sqrt(0.3), 0) and (V1, 0, sqrt(0.3)); a Gram-Schmidt step on
// them gives its Cholesky factor L = [[l11, 0], [l21, l22]] without forming
// a c - b^2, which keeps thin Gaussians accurate.  Returns (i11, k, i22) with
// z1 = dx i11, z2 = (dy - k dx) i22.
__device__ __forceinline__ float3 blend_factor(const KeyProj& p)
{
    const float s3 = 0.54772255750516611f;   // sqrt(0.3)
    const float ad = p.a + 0.3f;
    const float l11 = sqrtf(ad);
    const float l21 = p.b / l11;
    const float f = l21 / l11;
    const float r0 = p.V1[0] - f * p.V0[0];
    const float r1 = p.V1[1] - f * p.V0[1];
    const float r2 = p.V1[2] - f * p.V0[2];
    const float r3 = -f * s3;
    const float l22sq = r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3 + 0.3f;
    const float l22 = sqrtf(l22sq);
    return make_float3(kHalfLog2eSqrt / l11, f, kHalfLog2eSqrt / l22);
}

// Real spherical harmonics (Condon-Shortley phase) up to degree 3 at the unit
// direction (x, y, z): k0 = 1/(2 sqrt(pi)), k1 = sqrt(3/(4 pi)), k2a = sqrt(15/pi)/2,
// k2b = sqrt(5/pi)/4, k2c = sqrt(15/pi)/4, k3a = sqrt(35/(2 pi))/4,
// k3b = sqrt(105/pi)/2, k3c = sqrt(21/(2 pi))/4, k3d = sqrt(7/pi)/4, k3e = sqrt(105/pi)/4.
// With dY, also each function's gradient with respect to (x, y, z), the functions
// read as polynomials (their restriction to the sphere is the basis).
constexpr float kSH0 = 0.28209479177387814f, kSH1 = 0.4886025119029199f;
constexpr float kSH2a = 1.0925484305920792f, kSH2b = 0.31539156525252005f, kSH2c = 0.5462742152960396f;
constexpr float kSH3a = 0.5900435899266435f, kSH3b = 2.890611442640554f, kSH3c = 0.4570457994644658f;
constexpr float kSH3d = 0.3731763325901154f, kSH3e = 1.445305721320277f;

__device__ __forceinline__ void sh_basis16(float x, float y, float z, float (&Y)[16])
{
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = kSH0;
    Y[1] = -kSH1 * y; Y[2] = kSH1 * z; Y[3] = -kSH1 * x;
    Y[4] = kSH2a * x * y; Y[5] = -kSH2a * y * z; Y[6] = kSH2b * (2.f * zz - xx - yy);
    Y[7] = -kSH2a * x * z; Y[8] = kSH2c * (xx - yy);
    Y[9] = -kSH3a * y * (3.f * xx - yy); Y[10] = kSH3b * x * y * z;
    Y[11] = -kSH3c * y * (4.f * zz - xx - yy); Y[12] = kSH3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -kSH3c * x * (4.f * zz - xx - yy); Y[14] = kSH3e * z * (xx - yy);
    Y[15] = -kSH3a * x * (xx - 3.f * yy);
}

__device__ __forceinline__ void sh_basis16_grad(float x, float y, float z, float (&dY)[16][3])
{
    const float xx = x * x, yy = y * y, zz = z * z;
    const float g[16][3] = {
        {0.f, 0.f, 0.f},
        {0.f, -kSH1, 0.f}, {0.f, 0.f, kSH1}, {-kSH1, 0.f, 0.f},
        {kSH2a * y, kSH2a * x, 0.f}, {0.f, -kSH2a * z, -kSH2a * y},
        {-2.f * kSH2b * x, -2.f * kSH2b * y, 4.f * kSH2b * z},
        {-kSH2a * z, 0.f, -kSH2a * x}, {2.f * kSH2c * x, -2.f * kSH2c * y, 0.f},
        {-6.f * kSH3a * x * y, -3.f * kSH3a * (xx - yy), 0.f},
        {kSH3b * y * z, kSH3b * x * z, kSH3b * x * y},
        {2.f * kSH3c * x * y, -kSH3c * (4.f * zz - xx - 3.f * yy), -8.f * kSH3c * y * z},
        {-6.f * kSH3d * x * z, -6.f * kSH3d * y * z, kSH3d * (6.f * zz - 3.f * xx - 3.f * yy)},
        {-kSH3c * (4.f * zz - 3.f * xx - yy), 2.f * kSH3c * x * y, -8.f * kSH3c * x * z},
        {2.f * kSH3e * x * z, -2.f * kSH3e * y * z, kSH3e * (xx - yy)},
        {-3.f * kSH3a * (xx - yy), 6.f * kSH3a * x * y, 0.f}};
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) dY[k][i] = g[k][i];
}

// Blend record with its mean moved from the Gaussian's rectangle corner to this
// tile's corner (an exact integer shift, so the staged mean keeps its precision).
// Blend record of a (view, Gaussian), four float4 in one 64-byte block, so that
// a tile-list entry costs two 32-byte sectors of one cache line:
//   [kRecGeom0] mean - rectangle corner pixel (x, y), i11, k (blend factor form)
//   [kRecGeom1] i22, opacity, moment origin - mean (x, y)
//   [kRecCull]  culling constants (cull_record)
//   [kRecCorner] rectangle corner tile (x0, y0) as two 16-bit integers in the
//               bits of .x, log2(opacity) in .y, reference displacement
//               (.z, .w): the track at the moment origin (fit mode)
constexpr int kRecGeom0 = 0, kRecGeom1 = 1, kRecCull = 2, kRecCorner = 3;

__device__ __forceinline__ float rec_pack_corner(int x0, int y0)
{
    return __uint_as_float((uint32_t)(uint16_t)x0 | ((uint32_t)(uint16_t)y0 << 16));
}

// geom0 moved to tile (tx, ty)'s local frame from the packed corner
__device__ __forceinline__ float4 tile_local_packed(float4 g0, float corner, int tx, int ty, int tw, int th)
{
    const uint32_t c = __float_as_uint(corner);
    g0.x += (float)(((int)(c & 0xffffu) - tx) * tw);
    g0.y += (float)(((int)(c >> 16) - ty) * th);
    return g0;
}

__device__ __forceinline__ float4 tile_local(float4 g0, short4 r, int tx, int ty, int tw, int th)
{
    g0.x += (float)((r.x - tx) * tw);
    g0.y += (float)((r.y - ty) * th);
    return g0;
}

// Tile-local box outside which alpha = min(0.99, o exp2(-p)) < 1/255 for sure:
// p <= log2(255 o) is the ellipse z1^2 + z2^2 <= pm, whose extents follow from
// the factor (i11, k, i22); the 0.1 % widening covers FP32 rounding of p.
// Gaussians that cannot reach 1/255 anywhere get an empty box.
__device__ __forceinline__ float4 footprint_box(float4 g0, float4 g1)
{
    const float pm = log2f(255.0f * g1.y);
    if (!(pm > 0.0f)) return make_float4(1e30f, -1e30f, 1e30f, -1e30f);
    const float sp = sqrtf(pm) * 1.001f;
    const float ix = 1.0f / g0.z, iy = 1.0f / g1.x;
    const float hx = sp * ix + 1e-3f;
    const float hy = sp * sqrtf(g0.w * g0.w * ix * ix + iy * iy) + 1e-3f;
    return make_float4(g0.x - hx, g0.x + hx, g0.y - hy, g0.y + hy);
}

// Pixel of thread tid inside its 16x16 tile: warp w -> block (w & 1, w >> 1) of
// 8x4 pixels, lane l -> (l & 7, l >> 3) inside it.
__device__ __forceinline__ void pixel_of(int tid, int& lx, int& ly)
{
    const int warp = tid >> 5, lane = tid & 31;
    lx = (warp & 1) * 8 + (lane & 7);
    ly = (warp >> 1) * 4 + (lane >> 3);
}

// Sum of v[k] over the warp for k = lane >> 1, returned in every lane.
__device__ __forceinline__ float warp_transpose_sum16(float (&v)[16], int lane)
{
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool up = lane & 16;
        const float send = up ? v[i] : v[i + 8];
        const float keep = up ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool up = lane & 8;
        const float send = up ? v[i] : v[i + 4];
        const float keep = up ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool up = lane & 4;
        const float send = up ? v[i] : v[i + 2];
        const float keep = up ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool up = lane & 2;
        const float send = up ? v[0] : v[1];
        const float keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Blend constants (3DGS conventions): alpha = min(0.99, o G), contributions below
// 1/255 are skipped, the walk stops before a Gaussian that would take T below 1e-4.
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// Colour-render blend of one (pixel, Gaussian): alpha = min(0.99, o 2^-p) with
// p = z1^2 + z2^2 in the factor form of the staged record (tile-local mean g0.xy,
// i11 = g0.z, k = g0.w, i22 = g1.x, opacity g1.y) at the tile-local pixel centre
// (xc, yc), and the transmittance after it.  Every operation is a fixed
// instruction (correctly rounded intrinsics and the SFU's 2^x, relative error
// ~2^-22), so the forward render and its backward, which recomputes the blend tile
// by tile, take bit-identical decisions.
__device__ __forceinline__ float sfu_exp2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float render_alpha(float4 g0, float4 g1, float xc, float yc)
{
    const float ex = __fsub_rn(xc, g0.x), ey = __fsub_rn(yc, g0.y);
    const float z1 = __fmul_rn(ex, g0.z);
    const float z2 = __fmul_rn(__fmaf_rn(-g0.w, ex, ey), g1.x);
    const float pw = __fmaf_rn(z2, z2, __fmul_rn(z1, z1));
    return fminf(kAlphaMax, __fmul_rn(g1.y, sfu_exp2_approx(-pw)));
}

// render_alpha that also returns G = exp2(-power) (the same operations, so alpha
// is bit-identical).
__device__ __forceinline__ float render_alpha_g(float4 g0, float4 g1, float xc, float yc, float& G)
{
    const float ex = __fsub_rn(xc, g0.x), ey = __fsub_rn(yc, g0.y);
    const float z1 = __fmul_rn(ex, g0.z);
    const float z2 = __fmul_rn(__fmaf_rn(-g0.w, ex, ey), g1.x);
    const float pw = __fmaf_rn(z2, z2, __fmul_rn(z1, z1));
    G = sfu_exp2_approx(-pw);
    return fminf(kAlphaMax, __fmul_rn(g1.y, G));
}

// Culling constants of a record, formed once in the projection: the
// alpha >= 1/255 region of a Gaussian is the ellipse p = z1^2 + z2^2 <= log2(255 o)
// (z1 = ex i11, z2 = (ey - k ex) i22, (ex, ey) = pixel centre - mean).  Cut at a
// height ey, it is the interval c1 ey +- w0 sqrt(1 - (ey / hy)^2) with
//     A = i11^2 + k^2 i22^2,  c1 = k i22^2 / A,  w0 = sqrt(pm / A),
//     hy = sqrt(pm A) / (i11 i22)  (the half-height),
// and its rightmost point sits at ey_r = hy tau / sqrt(1 + tau^2), tau = c1 hy / w0
// (the leftmost at -ey_r).  The record holds (hy, c1, w0, ey_r) for the threshold
// raised by 0.2 % + 1e-4 and w0, hy widened by 0.1 % + 1e-3 px, so that FP32
// rounding never drops a pixel the blend keeps.  hy < 0: alpha >= 1/255 nowhere.
__device__ __forceinline__ float4 cull_record(float i11, float k, float i22, float opacity)
{
    const float pm = log2f(255.0f * opacity);
    if (!(pm > 0.0f)) return make_float4(-1e30f, 0.f, 0.f, 0.f);
    const float pw = pm * 1.002f + 1e-4f;
    const float i22s = i22 * i22;
    const float A = fmaf(i11, i11, k * k * i22s);
    const float c1 = k * i22s / A;
    const float w0 = sqrtf(pw / A) * 1.001f + 1e-3f;
    const float hy = sqrtf(pw * A) / (i11 * i22) * 1.001f + 1e-3f;
    const float tau = c1 * hy / w0;
    return make_float4(hy, c1, w0, hy * tau / sqrtf(fmaf(tau, tau, 1.0f)));
}

// x-interval [xl, xr] (relative to the mean) of the record's ellipse within the
// horizontal strip [sy0, sy1] (relative to the mean); false if they do not meet.
// The upper boundary c1 ey + w0 sqrt(1 - (ey/hy)^2) is concave, so its largest
// value over the strip is at ey_r clamped to the strip (the lower boundary's
// smallest at -ey_r); 1e-3 px of slack covers the rounding of the evaluation.
__device__ __forceinline__ bool strip_extent(float4 cr, float sy0, float sy1, float& xl, float& xr)
{
    const float hy = cr.x, c1 = cr.y, w0 = cr.z, eyr = cr.w;
    if (!(sy0 <= hy && sy1 >= -hy)) return false;
    const float lo = fmaxf(sy0, -hy), hi = fminf(sy1, hy);
    const float yr = fminf(fmaxf(eyr, lo), hi), yl = fminf(fmaxf(-eyr, lo), hi);
    // the SFU's reciprocal and square root (relative error ~2^-22): the interval
    // ends move by ~1e-6 of the ellipse's extent, far inside its 0.1 % widening
    float ihy, sr, sl;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ihy) : "f"(hy));
    const float tr = yr * ihy, tl = yl * ihy;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sr) : "f"(fmaxf(0.f, fmaf(-tr, tr, 1.0f))));
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sl) : "f"(fmaxf(0.f, fmaf(-tl, tl, 1.0f))));
    xr = fmaf(c1, yr, w0 * sr) + 1e-3f;
    xl = fmaf(c1, yl, -w0 * sl) - 1e-3f;
    return true;
}

// Tile-list entry (a 64-bit sort key): FP32 depth bits << 32 | Gaussian index << 4
// | block mask.  Keys order by (depth, index) -- the mask sits below the index
// and (depth, index) is unique -- and the low word gives the walks both the
// Gaussian (index < 2^28) and, in bit b, whether its alpha >= 1/255 ellipse
// can meet the tile's 8x8 block b (block b at ((b % (tw / 8)) * 8, (b / (tw / 8)) * 8)
// in the tile: four blocks for 16 x 16 and 32 x 8 tiles).
constexpr uint32_t kMaxGaussians = 1u << 28;
__device__ __forceinline__ uint64_t pair_key(uint32_t depth_bits, uint32_t g, uint32_t mask)
{
    return ((uint64_t)depth_bits << 32) | (g << 4) | mask;
}
__device__ __forceinline__ uint32_t entry_gauss(uint32_t lo) { return lo >> 4; }

// Block mask of a record in one tile: (mx, my) its mean in the tile's frame, cr
// its culling constants.  Bit b is set when the ellipse meets block b's pixel
// centres [bx + 0.5, bx + 7.5] x [by + 0.5, by + 7.5]: per 8-pixel row of blocks,
// the ellipse's x-interval in that strip against each block's columns.
__device__ __forceinline__ uint32_t block_hit_mask(float mx, float my, float4 cr, int tw)
{
    const int nbx = tw >> 3, nby = 4 / nbx;
    uint32_t m = 0u;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if (r >= nby) break;
        const float sy0 = ((float)(8 * r) + 0.5f) - my;
        float xl, xr;
        if (!strip_extent(cr, sy0, sy0 + 7.0f, xl, xr)) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (c >= nbx) break;
            const float bx0 = ((float)(8 * c) + 0.5f) - mx;
            if (xl <= bx0 + 7.0f && xr >= bx0) m |= 1u << (r * nbx + c);
        }
    }
    return m;
}

__device__ __forceinline__ float render_transmit(float T, float alpha)
{
    return __fmul_rn(T, __fsub_rn(1.0f, alpha));
}

__device__ __forceinline__ void view_of_tile(const ViewSet& vs, uint32_t tile, int& v, int& tx, int& ty)
{
    int lo = 0, hi = vs.V - 1;                 // last view whose first tile is <= tile
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (vs.toff[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    v = lo;
    const uint32_t local = tile - vs.toff[v];
    tx = (int)(local % (uint32_t)vs.tiles_x[v]);
    ty = (int)(local / (uint32_t)vs.tiles_x[v]);
}

}  // namespace tsp

// backward.cu -- the adjoint of the colour render (the blend of Sec. 3.1), for
// the gradient refinement that follows the track-guided relocation.
//
// For a loss L with dL/dC given at every pixel, C = sum_i c_i alpha_i T_i over the
// Gaussians of the pixel's tile list in depth order, with the blend's decisions
// (footprint box, alpha >= 1/255, the transmittance cut-off, the clamps of alpha at
// 0.99 and of the colour at 0) held fixed:
//   dL/dc_i     = alpha_i T_i dL/dC
//   dL/dalpha_i = dL/dC . (c_i T_i - (C - P_i) / (1 - alpha_i)),  P_i = sum_{j<=i} c_j alpha_j T_j
// (the colour behind i scales with 1 - alpha_i).  alpha = o G, G = exp(-d^T Q d / 2)
// with d = pixel centre - mu_2D and Q the inverse of the dilated Sigma_2D.
//
// k_render_backward recomputes each tile's blend front to back from the tile
// lists (no per-pixel lists are stored; the forward colour C is an input) with the
// forward render's walk: warp w takes the 8x8 block (w & 1, w >> 1), lane l its
// pixels (l & 7, (l >> 3) + 4k), entries culled by the exact ellipse-block test,
// the same arithmetic and decisions per pixel.  Two phases, as in the moment
// accumulation:
//   phase 1 (pixel-parallel), per hit: h = G dL/dalpha (0 where alpha is clamped)
//   and the weight alpha T of each pixel into a warp-private buffer;
//   phase 2 (hit-parallel), per 8 pending hits: the block sums S0 = sum h,
//   S1, S2 = sum h (x~, y~), S3, S4, S5 = sum h (x~^2, x~ y~, y~^2) with
//   (x~, y~) = pixel centre - mu_2D, and sum alpha T dL/dC per channel.  With
//   G = 2^-p, p = z1^2 + z2^2, z1 = x~ i11, z2 = (y~ - k x~) i22, the per-(view,
//   Gaussian) quantities are dL/dmu_2D = o ln2 dp/d(x~, y~) applied to (S1, S2),
//   dL/dQ = -o/2 (S3, 2 S4, S5) and dL/do = S0; 3 float4 atomics per (block, hit).
// The colour term of dL/dalpha uses the running scalar Q = dL/dC . P, so a pixel
// keeps 4 numbers of state.  k_render_backward_project then carries them, one thread
// per Gaussian over its views, through Q = inverse(Sigma_2D + 0.3 I),
// Sigma_2D = (J W) Sigma_3D (J W)^T, the perspective map, the colour basis along
// the viewing direction and Sigma_3D = R(q) diag(s^2) R(q)^T.
#include "launch.h"

namespace tsp {

namespace {

constexpr float kLn2 = 0.69314718055994531f;
constexpr uint32_t kFull = 0xffffffffu;


constexpr int kBChunk = 8;                       // pending hits per phase 2
constexpr int kBRow = 2 * kBChunk + 2;           // words per pixel: (h, w) per hit, padded
constexpr int kBQuarter = 16 * kBRow + 16;       // 16 pixels; = 16 (mod 32) words
constexpr int kBWords = 4 * kBQuarter;

struct BwdSmem {
    float4 g0[32];
    float4 g1[32];
    float4 c[32];
    uint32_t id[32];
    float4 pg0[kBChunk];                         // pending hits: blend parameters, record
    float4 pg1[kBChunk];
    uint32_t pid[kBChunk];
    float HW[kBWords];                           // (h, w) of pixel 16 q + j, hit c at q kBQuarter + j kBRow + 2c
    float4 gC[64];                               // dL/dC of each pixel
};

// TW: tile width, 16 (16 x 16 tiles) or 32 (32 x 8), known at compile time.
template <int TW>
__device__ __forceinline__ void backward_block(const ViewSet& vs, const Work& w, const RenderGrad& rg, uint32_t tile,
                                               int blk, BwdSmem& sm)
{
    const uint32_t beg = min(w.tile_off[tile], w.cap), end = min(w.tile_off[tile + 1], w.cap);
    if (beg >= end) return;
    int v, tx, ty;
    view_of_tile(vs, tile, v, tx, ty);
    const int lane = threadIdx.x & 31;
    constexpr int TH = kTilePx / TW;
    constexpr int nbx = TW / 8;                // 8x8 blocks per tile row
    const int bxo = (blk % nbx) * 8, byo = (blk / nbx) * 8;
    const int W = vs.cam[v].W, H = vs.cam[v].H;
    const size_t vbase = (size_t)vs.vrec[v];
    const float xc = (float)(bxo + (lane & 7)) + 0.5f;
    float yc[2], T[2], D[2], Q[2], gc[2][3];
    bool done[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int ly = byo + (lane >> 3) + 4 * k;
        const int px = tx * TW + bxo + (lane & 7), py = ty * TH + ly;
        const bool inside = px < W && py < H;
        float cf[3] = {0.f, 0.f, 0.f};
        gc[k][0] = gc[k][1] = gc[k][2] = 0.f;
        if (inside) {
            const size_t pix = 3 * ((size_t)py * W + px);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                cf[ch] = rg.rgb[v][pix + ch];
                gc[k][ch] = rg.grad[v][pix + ch];
            }
        }
        sm.gC[lane + 32 * k] = make_float4(gc[k][0], gc[k][1], gc[k][2], 0.f);
        D[k] = gc[k][0] * cf[0] + gc[k][1] * cf[1] + gc[k][2] * cf[2];   // dL/dC . C
        Q[k] = 0.f;                                                     // dL/dC . P
        yc[k] = (float)ly + 0.5f;
        T[k] = 1.0f;
        done[k] = !inside;
    }
    // column 0 of pixel p = lane (+ 32: two quarters further) in the (h, w) buffer
    const int hofs = (lane >> 4) * kBQuarter + (lane & 15) * kBRow;
    int pend = 0;

    auto phase2 = [&](int npend) {
        __syncwarp();
        const int c = lane & 7, q = lane >> 3;
        const float4 p0 = sm.pg0[c];
        float s[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) s[m] = 0.f;
        const float* hq = sm.HW + q * kBQuarter + 2 * c;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int p = 16 * q + j;
            const float2 hw = *reinterpret_cast<const float2*>(hq + j * kBRow);
            const float X = (float)(bxo + (p & 7)) + 0.5f - p0.x;
            const float Y = (float)(byo + (p >> 3)) + 0.5f - p0.y;
            const float4 g = sm.gC[p];
            const float hx = hw.x * X, hy = hw.x * Y;
            s[0] += hw.x;
            s[1] += hx;
            s[2] += hy;
            s[3] = fmaf(hx, X, s[3]);
            s[4] = fmaf(hx, Y, s[4]);
            s[5] = fmaf(hy, Y, s[5]);
            s[6] = fmaf(hw.y, g.x, s[6]);
            s[7] = fmaf(hw.y, g.y, s[7]);
            s[8] = fmaf(hw.y, g.z, s[8]);
        }
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            s[m] += __shfl_xor_sync(kFull, s[m], 8);
            s[m] += __shfl_xor_sync(kFull, s[m], 16);
        }
        if (q == 0 && c < npend) {
            const float4 p1 = sm.pg1[c];
            const float o = p1.y, i22s = p1.x * p1.x;
            // dp/d(x~, y~) = 2 (A x~ + B y~, B x~ + Cc y~)
            const float A = fmaf(p0.z, p0.z, p0.w * p0.w * i22s), B = -p0.w * i22s, Cc = i22s;
            const float f = 2.f * o * kLn2;
            float* dst = rg.acc + (vbase + sm.pid[c]) * kGradStride;
            atomicAdd(reinterpret_cast<float4*>(dst),
                      make_float4(f * fmaf(A, s[1], B * s[2]), f * fmaf(B, s[1], Cc * s[2]), -0.5f * o * s[3],
                                  -o * s[4]));
            atomicAdd(reinterpret_cast<float4*>(dst + 4), make_float4(-0.5f * o * s[5], s[0], s[6], s[7]));
            atomicAdd(dst + 8, s[8]);
        }
        __syncwarp();
    };

    for (uint32_t b0 = beg; b0 < end; b0 += 32) {
        if (!__any_sync(kFull, !done[0] || !done[1])) break;
        // list entries carry the block mask: only the hits load their records
        const uint32_t e = b0 + lane < end ? (uint32_t)w.pairs[b0 + lane] : 0u;
        const bool hit = b0 + lane < end && ((e >> blk) & 1u);
        if (hit) {
            const uint32_t g = entry_gauss(e);
            const float4* rc = w.rec + 4 * (vbase + g);
            sm.g0[lane] = tile_local_packed(rc[kRecGeom0], rc[kRecCorner].x, tx, ty, TW, TH);
            sm.g1[lane] = rc[kRecGeom1];
            sm.c[lane] = w.color[vbase + g];
            sm.id[lane] = g;
        }
        uint32_t m = __ballot_sync(kFull, hit);
        __syncwarp();
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const float4 g0 = sm.g0[j], g1 = sm.g1[j], c = sm.c[j];
            // render_alpha_g / render_transmit of the lane's two pixels in packed
            // FP32x2 (each component the same correctly rounded operation)
            const float ex = __fsub_rn(xc, g0.x);
            const float z1 = __fmul_rn(ex, g0.z);
            const float z1s = __fmul_rn(z1, z1);
            const float2 ey = __fadd2_rn(make_float2(yc[0], yc[1]), make_float2(-g0.y, -g0.y));
            const float2 t = __ffma2_rn(make_float2(-g0.w, -g0.w), make_float2(ex, ex), ey);
            const float2 z2 = __fmul2_rn(t, make_float2(g1.x, g1.x));
            const float2 pw = __ffma2_rn(z2, z2, make_float2(z1s, z1s));
            const float2 G = make_float2(sfu_exp2_approx(-pw.x), sfu_exp2_approx(-pw.y));
            const float2 oG = __fmul2_rn(make_float2(g1.y, g1.y), G);
            const float2 al = make_float2(fminf(kAlphaMax, oG.x), fminf(kAlphaMax, oG.y));
            const float2 Tp = make_float2(T[0], T[1]);
            const float2 om = __fadd2_rn(make_float2(1.0f, 1.0f), make_float2(-al.x, -al.y));
            const float2 Tn = __fmul2_rn(Tp, om);
            const float2 wp = __fmul2_rn(al, Tp);
            bool add[2];
            float wk[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float alpha = k ? al.y : al.x, tn = k ? Tn.y : Tn.x;
                const bool pass = !done[k] && alpha >= kAlphaMin;
                const bool term = pass && tn < kTMin;
                add[k] = pass && !term;
                wk[k] = add[k] ? (k ? wp.y : wp.x) : 0.f;
                done[k] = done[k] || term;
            }
            // dL/dC . c, the running dL/dC . P (this Gaussian included) and dL/dalpha
            const float2 w2 = make_float2(wk[0], wk[1]);
            const float2 gcc = __ffma2_rn(make_float2(gc[0][0], gc[1][0]), make_float2(c.x, c.x),
                                          __ffma2_rn(make_float2(gc[0][1], gc[1][1]), make_float2(c.y, c.y),
                                                     __fmul2_rn(make_float2(gc[0][2], gc[1][2]),
                                                                make_float2(c.z, c.z))));
            const float2 Q2 = __ffma2_rn(w2, gcc, make_float2(Q[0], Q[1]));
            float hv[2], wv[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float q = k ? Q2.y : Q2.x;
                if (add[k]) {
                    Q[k] = q;
                    const float ga = fmaf(k ? gcc.y : gcc.x, T[k], -__fdividef(D[k] - q, k ? om.y : om.x));
                    const float Gk = k ? G.y : G.x;
                    hv[k] = (k ? oG.y : oG.x) < kAlphaMax ? ga * Gk : 0.f;   // alpha = o G, not clamped
                    T[k] = k ? Tn.y : Tn.x;
                } else {
                    hv[k] = 0.f;
                }
                wv[k] = wk[k];
            }
            if (!__any_sync(kFull, add[0] || add[1])) continue;               // nothing of this block
#pragma unroll
            for (int k = 0; k < 2; ++k)
                *reinterpret_cast<float2*>(&sm.HW[hofs + 2 * k * kBQuarter + 2 * pend]) = make_float2(hv[k], wv[k]);
            if (lane == 0) {
                sm.pg0[pend] = g0;
                sm.pg1[pend] = g1;
                sm.pid[pend] = sm.id[j];
            }
            if (++pend == kBChunk) {
                phase2(kBChunk);
                pend = 0;
            }
        }
        __syncwarp();                                   // staging is rewritten next
    }
    if (pend) phase2(pend);
}

// 7 CTAs per SM: 72 registers, and 7 x 31.4 KB of shared memory with the
// largest carveout (set once per context by backward_prepare)
template <int TW>
__global__ void __launch_bounds__(128, 7) k_render_backward(const ViewSet vs, const Work w, const RenderGrad rg)
{
    __shared__ BwdSmem sm[4];
    const int warp = threadIdx.x >> 5;
    backward_block<TW>(vs, w, rg, blockIdx.x, warp, sm[warp]);
}

// grid (ceil(nmax / 128), F): one thread per Gaussian of frame blockIdx.y.
__global__ void __launch_bounds__(128) k_render_backward_project(const ViewSet vs, const Work w,
                                                                 const RenderGrad rg, const float* __restrict__ sh,
                                                                 int sh_degree)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int f = blockIdx.y;
    if (g >= vs.fn[f]) return;
    const int nb = (sh_degree + 1) * (sh_degree + 1);
    const float4 mo = vs.fmo[f][g], qi = vs.fq[f][g], si = vs.fs[f][g];
    const float X[3] = {mo.x, mo.y, mo.z};
    const float qnorm = sqrtf(qi.x * qi.x + qi.y * qi.y + qi.z * qi.z + qi.w * qi.w);
    const float qw = qi.x / qnorm, qx = qi.y / qnorm, qy = qi.z / qnorm, qz = qi.w / qnorm;
    const float R[3][3] = {
        {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
        {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
        {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)}};
    const float sv[3] = {si.x, si.y, si.z};
    float S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            S[i][j] = R[i][0] * sv[0] * sv[0] * R[j][0] + R[i][1] * sv[1] * sv[1] * R[j][1] +
                      R[i][2] * sv[2] * sv[2] * R[j][2];
    const float* shg = sh + (size_t)g * nb * 3;
    float gX[3] = {0.f, 0.f, 0.f}, gS[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float go = 0.f, gsh[16][3];
#pragma unroll
    for (int k = 0; k < 16; ++k) gsh[k][0] = gsh[k][1] = gsh[k][2] = 0.f;
    for (int v = vs.fview[f]; v < vs.fview[f + 1]; ++v) {
        const size_t rec = (size_t)vs.vrec[v] + g;
        if (w.touched[rec] == 0u) continue;
        const float* a = rg.acc + rec * kGradStride;
        const float gmx = a[0], gmy = a[1], q00 = a[2], q01 = a[3], q11 = a[4];
        const float gc[3] = {a[6], a[7], a[8]};
        go += a[5];
        const DevCam& c = vs.cam[v];
        float p[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) p[i] = c.R[3 * i] * X[0] + c.R[3 * i + 1] * X[1] + c.R[3 * i + 2] * X[2] + c.t[i];
        const float iz = 1.f / p[2], iz2 = iz * iz, iz3 = iz2 * iz;
        const float J[2][3] = {{c.fx * iz, 0.f, -c.fx * p[0] * iz2}, {0.f, c.fy * iz, -c.fy * p[1] * iz2}};
        float T[2][3], TS[2][3];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int j = 0; j < 3; ++j) T[u][j] = J[u][0] * c.R[j] + J[u][1] * c.R[3 + j] + J[u][2] * c.R[6 + j];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int j = 0; j < 3; ++j) TS[u][j] = T[u][0] * S[0][j] + T[u][1] * S[1][j] + T[u][2] * S[2][j];
        // Q = inverse of the dilated Sigma_2D [[a, b], [b, d]]
        const float sa = TS[0][0] * T[0][0] + TS[0][1] * T[0][1] + TS[0][2] * T[0][2] + 0.3f;
        const float sb = TS[0][0] * T[1][0] + TS[0][1] * T[1][1] + TS[0][2] * T[1][2];
        const float sd = TS[1][0] * T[1][0] + TS[1][1] * T[1][1] + TS[1][2] * T[1][2] + 0.3f;
        const float det = sa * sd - sb * sb, id = 1.f / det, id2 = id * id;
        const float ga = q00 * (-sd * sd * id2) + q01 * (sb * sd * id2) + q11 * (id - sa * sd * id2);
        const float gd = q00 * (id - sa * sd * id2) + q01 * (sa * sb * id2) + q11 * (-sa * sa * id2);
        const float gb = q00 * (2.f * sb * sd * id2) + q01 * (-id - 2.f * sb * sb * id2) + q11 * (2.f * sa * sb * id2);
        const float G2[2][2] = {{ga, 0.5f * gb}, {0.5f * gb, gd}};
        // Sigma_2D = T S T^T
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                gS[i][j] += T[0][i] * (G2[0][0] * T[0][j] + G2[0][1] * T[1][j]) +
                            T[1][i] * (G2[1][0] * T[0][j] + G2[1][1] * T[1][j]);
        float gT[2][3], gJ[2][3];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int j = 0; j < 3; ++j) gT[u][j] = 2.f * (G2[u][0] * TS[0][j] + G2[u][1] * TS[1][j]);
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                gJ[u][k] = gT[u][0] * c.R[3 * k] + gT[u][1] * c.R[3 * k + 1] + gT[u][2] * c.R[3 * k + 2];
        // the perspective map: mu_2D and J at the camera-space point p
        float gp[3];
        gp[0] = gJ[0][2] * (-c.fx * iz2) + gmx * c.fx * iz;
        gp[1] = gJ[1][2] * (-c.fy * iz2) + gmy * c.fy * iz;
        gp[2] = gJ[0][0] * (-c.fx * iz2) + gJ[0][2] * (2.f * c.fx * p[0] * iz3) + gJ[1][1] * (-c.fy * iz2) +
                gJ[1][2] * (2.f * c.fy * p[1] * iz3) - gmx * c.fx * p[0] * iz2 - gmy * c.fy * p[1] * iz2;
#pragma unroll
        for (int j = 0; j < 3; ++j) gX[j] += c.R[j] * gp[0] + c.R[3 + j] * gp[1] + c.R[6 + j] * gp[2];
        // colour along the direction from the camera centre C = -R^T t
        float dir[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            dir[i] = X[i] + (c.R[i] * c.t[0] + c.R[3 + i] * c.t[1] + c.R[6 + i] * c.t[2]);
        const float dist = sqrtf(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
#pragma unroll
        for (int i = 0; i < 3; ++i) dir[i] /= dist;
        float Y[16], dY[16][3];
        sh_basis16(dir[0], dir[1], dir[2], Y);
        sh_basis16_grad(dir[0], dir[1], dir[2], dY);
        float gY[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) gY[k] = 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float raw = 0.5f;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (k < nb) raw = fmaf(Y[k], shg[3 * k + ch], raw);
            if (!(raw > 0.f)) continue;                       // clamped at 0
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (k < nb) {
                    gsh[k][ch] = fmaf(Y[k], gc[ch], gsh[k][ch]);
                    gY[k] = fmaf(shg[3 * k + ch], gc[ch], gY[k]);
                }
        }
        float gdir[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int i = 0; i < 3; ++i) gdir[i] = fmaf(gY[k], dY[k][i], gdir[i]);
        const float dd = dir[0] * gdir[0] + dir[1] * gdir[1] + dir[2] * gdir[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) gX[i] += (gdir[i] - dir[i] * dd) / dist;
    }
    // Sigma_3D = R D R^T, D = diag(s^2)
    float gs[3], gR[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) acc += R[i][k] * gS[i][j] * R[j][k];
        gs[k] = 2.f * sv[k] * acc;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            gR[i][k] = 2.f * (gS[i][0] * R[0][k] + gS[i][1] * R[1][k] + gS[i][2] * R[2][k]) * sv[k] * sv[k];
    const float dRw[3][3] = {{0.f, -2.f * qz, 2.f * qy}, {2.f * qz, 0.f, -2.f * qx}, {-2.f * qy, 2.f * qx, 0.f}};
    const float dRx[3][3] = {{0.f, 2.f * qy, 2.f * qz}, {2.f * qy, -4.f * qx, -2.f * qw}, {2.f * qz, 2.f * qw, -4.f * qx}};
    const float dRy[3][3] = {{-4.f * qy, 2.f * qx, 2.f * qw}, {2.f * qx, 0.f, 2.f * qz}, {-2.f * qw, 2.f * qz, -4.f * qy}};
    const float dRz[3][3] = {{-4.f * qz, -2.f * qw, 2.f * qx}, {2.f * qw, -4.f * qz, 2.f * qy}, {2.f * qx, 2.f * qy, 0.f}};
    float gh[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            gh[0] += gR[i][j] * dRw[i][j];
            gh[1] += gR[i][j] * dRx[i][j];
            gh[2] += gR[i][j] * dRy[i][j];
            gh[3] += gR[i][j] * dRz[i][j];
        }
    const float hq = gh[0] * qw + gh[1] * qx + gh[2] * qy + gh[3] * qz;
    rg.g_means[g] = make_float4(gX[0], gX[1], gX[2], go);
    rg.g_scales[g] = make_float4(gs[0], gs[1], gs[2], 0.f);
    rg.g_quats[g] = make_float4((gh[0] - qw * hq) / qnorm, (gh[1] - qx * hq) / qnorm, (gh[2] - qy * hq) / qnorm,
                                (gh[3] - qz * hq) / qnorm);
    float* out = rg.g_sh + (size_t)g * nb * 3;
#pragma unroll
    for (int k = 0; k < 16; ++k)
        if (k < nb) {
            out[3 * k] = gsh[k][0];
            out[3 * k + 1] = gsh[k][1];
            out[3 * k + 2] = gsh[k][2];
        }
}

}  // namespace

cudaError_t backward_prepare()
{
    const cudaError_t e = cudaFuncSetAttribute((const void*)k_render_backward<16>,
                                               cudaFuncAttributePreferredSharedMemoryCarveout,
                                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void*)k_render_backward<32>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

cudaError_t launch_render_backward(const ViewSet& vs, const Work& w, uint32_t NT, const RenderGrad& rg,
                                   const float* sh, int sh_degree, size_t records, cudaStream_t st)
{
    if (vs.nmax == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(rg.acc, 0, records * kGradStride * sizeof(float), st);
    if (e != cudaSuccess) return e;
    if (NT > 0 && vs.tw == 32) k_render_backward<32><<<NT, 128, 0, st>>>(vs, w, rg);
    else if (NT > 0) k_render_backward<16><<<NT, 128, 0, st>>>(vs, w, rg);
    dim3 grid((vs.nmax + 127) / 128, vs.F);
    k_render_backward_project<<<grid, 128, 0, st>>>(vs, w, rg, sh, sh_degree);
    return cudaGetLastError();
}

}  // namespace tsp

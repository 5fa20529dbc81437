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
// lists (no per-pixel lists are stored; the forward colour C is an input), with
// the same layout, staging and decisions as the forward render kernel, and folds
// each (8x4 warp block, Gaussian) contribution to the 9 per-(view, Gaussian)
// quantities (d mu_2D, d Q, d opacity, d colour) with one transposing butterfly
// before its atomics.  k_render_backward_project then carries them, one thread
// per Gaussian over its views, through Q = inverse(Sigma_2D + 0.3 I),
// Sigma_2D = (J W) Sigma_3D (J W)^T, the perspective map, the colour basis along
// the viewing direction and Sigma_3D = R(q) diag(s^2) R(q)^T.
#include "launch.h"

namespace tsp {

namespace {

constexpr int kBBatch = 64;
constexpr float kLn2 = 0.69314718055994531f;

__global__ void __launch_bounds__(kTilePx) k_render_backward(const ViewSet vs, const Work w,
                                                             const RenderGrad rg)
{
    __shared__ float4 s_g0[kBBatch];
    __shared__ float4 s_g1[kBBatch];
    __shared__ float4 s_box[kBBatch];
    __shared__ float4 s_c[kBBatch];
    __shared__ uint32_t s_id[kBBatch];
    const uint32_t tile = blockIdx.x;
    const uint32_t beg = min(w.tile_off[tile], w.cap), end = min(w.tile_off[tile + 1], w.cap);
    if (beg >= end) return;
    int v, tx, ty;
    view_of_tile(vs, tile, v, tx, ty);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int lx, ly;
    pixel_of(tid, lx, ly);
    const int W = vs.cam[v].W, H = vs.cam[v].H;
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool inside = px < W && py < H;
    const float xc = (float)lx + 0.5f, yc = (float)ly + 0.5f;
    const float bx0 = (float)((warp & 1) * 8) + 0.5f, bx1 = bx0 + 7.0f;
    const float by0 = (float)((warp >> 1) * 4) + 0.5f, by1 = by0 + 3.0f;
    float Cf[3] = {0.f, 0.f, 0.f}, gC[3] = {0.f, 0.f, 0.f}, P[3] = {0.f, 0.f, 0.f};
    if (inside) {
        const size_t pix = 3 * ((size_t)py * W + px);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            Cf[ch] = rg.rgb[v][pix + ch];
            gC[ch] = rg.grad[v][pix + ch];
        }
    }
    float T = 1.0f;
    bool done = !inside;
    const size_t vbase = (size_t)vs.vrec[v];
    for (uint32_t b0 = beg; b0 < end; b0 += kBBatch) {
        const int nb = (int)min((uint32_t)kBBatch, end - b0);
        if (tid < nb) {
            const uint32_t g = (uint32_t)w.pairs[b0 + tid];
            const float4 g0 = tile_local(w.geom0[vbase + g], w.rect[vbase + g], tx, ty);
            const float4 g1 = w.geom1[vbase + g];
            s_g0[tid] = g0;
            s_g1[tid] = g1;
            s_box[tid] = footprint_box(g0, g1);
            s_c[tid] = w.color[vbase + g];
            s_id[tid] = g;
        }
        __syncthreads();
        for (int j = 0; j < nb; ++j) {
            const float4 bb = s_box[j];                       // warp-uniform, as in the forward
            if (bb.x > bx1 || bb.y < bx0 || bb.z > by1 || bb.w < by0) continue;
            const float4 g0 = s_g0[j];
            const float4 g1 = s_g1[j];
            const float4 c = s_c[j];
            float val[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) val[k] = 0.f;
            bool add = false;
            if (!done) {
                const float alpha = render_alpha(g0, g1, xc, yc);
                if (alpha >= kAlphaMin) {
                    const float Tn = render_transmit(T, alpha);
                    if (Tn < kTMin) {
                        done = true;
                    } else {
                        add = true;
                        const float wgt = alpha * T;
                        const float cc[3] = {c.x, c.y, c.z};
                        float ga = 0.f;
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) {
                            P[ch] = fmaf(wgt, cc[ch], P[ch]);
                            ga = fmaf(gC[ch], cc[ch] * T - (Cf[ch] - P[ch]) / (1.0f - alpha), ga);
                            val[6 + ch] = wgt * gC[ch];
                        }
                        const float ex = xc - g0.x, ey = yc - g0.y;
                        const float z1 = ex * g0.z;
                        const float z2 = fmaf(-g0.w, ex, ey) * g1.x;
                        const float G = exp2f(-fmaf(z2, z2, z1 * z1));
                        if (__fmul_rn(g1.y, G) < 0.99f) {             // alpha = o G, not clamped
                            val[5] = G * ga;
                            const float gG = g1.y * ga;
                            // G = 2^-(z1^2 + z2^2): dG/dmu = ln2 G dp/d(ex, ey)
                            const float dpx = 2.f * (z1 * g0.z - z2 * g0.w * g1.x);
                            const float dpy = 2.f * z2 * g1.x;
                            val[0] = gG * kLn2 * G * dpx;
                            val[1] = gG * kLn2 * G * dpy;
                            // G = exp(-d^T Q d / 2): dG/dQ
                            val[2] = gG * (-0.5f * G * ex * ex);
                            val[3] = gG * (-G * ex * ey);
                            val[4] = gG * (-0.5f * G * ey * ey);
                        }
                        T = Tn;
                    }
                }
            }
            if (__any_sync(0xffffffffu, add)) {
                const float r = warp_transpose_sum16(val, lane);
                if ((lane & 1) == 0 && (lane >> 1) < 9)
                    atomicAdd(&rg.acc[(vbase + s_id[j]) * kGradStride + (lane >> 1)], r);
            }
        }
        if (__syncthreads_count(!done) == 0) break;
    }
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

cudaError_t launch_render_backward(const ViewSet& vs, const Work& w, uint32_t NT, const RenderGrad& rg,
                                   const float* sh, int sh_degree, size_t records, cudaStream_t st)
{
    if (vs.nmax == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(rg.acc, 0, records * kGradStride * sizeof(float), st);
    if (e != cudaSuccess) return e;
    if (NT > 0) k_render_backward<<<NT, kTilePx, 0, st>>>(vs, w, rg);
    dim3 grid((vs.nmax + 127) / 128, vs.F);
    k_render_backward_project<<<grid, 128, 0, st>>>(vs, w, rg, sh, sh_degree);
    return cudaGetLastError();
}

}  // namespace tsp

// solve.cu -- a6 per-view affine solve and a7-a9 multi-view update.
//
// a6 (Eq. 4, Eq. 2, Sec. 4.3.5, Sec. 5.1), one thread per (view, Gaussian):
//   the moment record holds sums over the Gaussian's pixels with coordinates
//   x~ = x - mu_2D.  Writing Eq. 4 in that basis, V1 = sum w [x~;1][x~;1]^T and
//   V2 = sum w [x~;1] x'^T with x' - mu_2D = x~ + d, so V1^-1 V2 = [I;0] + V1^-1 D
//   with D = sum w [x~;1] d^T.  The 3x3 system is solved through its Schur
//   complement S = sum w x~ x~^T - (sum w x~)(sum w x~)^T / sum w (the weighted
//   pixel scatter), which keeps FP32 well conditioned.
// a7 (Sec. 4.4.1), one thread per Gaussian: linear triangulation in pixel units,
//   rows (u' P3 - P1) and (v' P3 - P2) of P = K [R|t], written about the old mean
//   (X = mu + delta) so the right-hand side is -z_mu times the per-view shift of
//   the centre: no cancellation.  FP32 normal equations, FP64 Cholesky.
// a8 (Sec. 4.4.2): vech(T Sigma T^T) = vech(Sigma_2D') per solved view with
//   T = J' W at the new mean, 6 unknowns, normal equations and Cholesky in FP64.
// a9 (Sec. 4.4.3): Jacobi eigen decomposition in FP64; discard if an eigenvalue
//   is <= 0; new axis k takes the eigenpair whose rank matches the rank of the old
//   scale s_k; each axis is flipped to agree with the old one; a reflection is
//   undone on the least-aligned axis; the quaternion sign follows the old one.
#include "launch.h"

namespace tsp {

namespace {

// Per-view records written by a6 and read by a7/a8:
//   vres0 = (mu'_x, mu'_y, c_x, c_y) with c = mu' - mu_2D the shift of the centre,
//   vres1 = (B00, B01, B02, sum w), vres3 = (B10, B11, B12, 0) with Sigma_2D' = B B^T,
//   vres2 = (flags, pixels).

__global__ void __launch_bounds__(256) k_view_solve(const ViewSet vs, const float4* __restrict__ mo,
                                                    const float4* __restrict__ q,
                                                    const float4* __restrict__ s, const FitParams fp,
                                                    const Work w, float* __restrict__ view_affine,
                                                    uint32_t* __restrict__ view_flags)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    if (g >= vs.n) return;
    const size_t i = (size_t)v * vs.n + g;
    uint32_t flags = 0;
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = make_float4(0.f, 0.f, 0.f, 0.f);
    float A00 = 0.f, A01 = 0.f, A10 = 0.f, A11 = 0.f, b0 = 0.f, b1 = 0.f;
    float npix = 0.f;
    if (w.touched[i] == 0u) {
        flags = TSP_VIEW_CULLED | TSP_VIEW_FEW_PX | TSP_VIEW_LOW_ALPHA;
    } else {
        float M[16];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 t = w.moments[4 * i + k];
            M[4 * k] = t.x; M[4 * k + 1] = t.y; M[4 * k + 2] = t.z; M[4 * k + 3] = t.w;
        }
        const float sw = M[0];
        npix = M[13];
        r1.w = sw;
        if (npix < (float)fp.min_px_view) flags |= TSP_VIEW_FEW_PX;
        if (!(sw >= fp.sumw_min_view)) flags |= TSP_VIEW_LOW_ALPHA;
        if (flags == 0u) {
            const float isw = 1.0f / sw;
            const float mx = M[1] * isw, my = M[2] * isw;
            const float cxx = M[3] * isw - mx * mx;
            const float cxy = M[4] * isw - mx * my;
            const float cyy = M[5] * isw - my * my;
            const float detC = cxx * cyy - cxy * cxy;
            const float tr = cxx + cyy;
            const float lmin = 0.5f * (tr - sqrtf(fmaxf(tr * tr - 4.0f * detC, 0.0f)));
            const float det3 = sw * sw * sw * detC;   // det V1 = (sum w)^3 det(scatter / sum w)
            if (!(det3 >= fp.det_min) || !(lmin >= fp.lam_min_px2)) {
                flags = TSP_VIEW_SINGULAR;
            } else {
                const float Sxx = sw * cxx, Sxy = sw * cxy, Syy = sw * cyy;
                const float idS = 1.0f / (Sxx * Syy - Sxy * Sxy);
                const float Rx0 = M[8] - M[1] * M[6] * isw, Rx1 = M[9] - M[1] * M[7] * isw;
                const float Ry0 = M[10] - M[2] * M[6] * isw, Ry1 = M[11] - M[2] * M[7] * isw;
                const float Y00 = (Syy * Rx0 - Sxy * Ry0) * idS, Y01 = (Syy * Rx1 - Sxy * Ry1) * idS;
                const float Y10 = (Sxx * Ry0 - Sxy * Rx0) * idS, Y11 = (Sxx * Ry1 - Sxy * Rx1) * idS;
                // intercept at the moment origin o = mu + delta; the displacement sums
                // were taken about the reference r, which only shifts the intercept
                const float2 rf = w.dref[i];
                const float co0 = (M[6] - M[1] * Y00 - M[2] * Y10) * isw + rf.x;
                const float co1 = (M[7] - M[1] * Y01 - M[2] * Y11) * isw + rf.y;
                A00 = 1.0f + Y00; A01 = Y10; A10 = Y01; A11 = 1.0f + Y11;
                KeyProj p;
                key_project(vs.cam[v], mo[g], q[g], s[g], vs.tiles_x[v], vs.tiles_y[v], p);
                float2 mxd, myd;
                mean2d_df(vs.cam[v], mo[g], mxd, myd);
                // shift of the centre: mu' - mu = c_o + (I - A) delta
                const float2 dl = moment_origin_shift(mxd, myd, vs.cam[v].W, vs.cam[v].H);
                const float c0 = co0 + dl.x - (A00 * dl.x + A01 * dl.y);
                const float c1 = co1 + dl.y - (A10 * dl.x + A11 * dl.y);
                const float ux = mxd.x + (mxd.y + c0), uy = myd.x + (myd.y + c1);
                // Eq. 2 with the undilated Sigma_2D = V V^T: Sigma' = (A V)(A V)^T.
                // The factor B = A V is kept (not the entries of Sigma'), so a thin
                // footprint's small eigenvalue survives the FP32 hand-over to a8.
                const float B00 = A00 * p.V0[0] + A01 * p.V1[0], B01 = A00 * p.V0[1] + A01 * p.V1[1];
                const float B02 = A00 * p.V0[2] + A01 * p.V1[2];
                const float B10 = A10 * p.V0[0] + A11 * p.V1[0], B11 = A10 * p.V0[1] + A11 * p.V1[1];
                const float B12 = A10 * p.V0[2] + A11 * p.V1[2];
                r0 = make_float4(ux, uy, c0, c1);
                r1 = make_float4(B00, B01, B02, sw);
                w.vres3[i] = make_float4(B10, B11, B12, 0.f);
                b0 = (mxd.x - (A00 * mxd.x + A01 * myd.x)) + (c0 + mxd.y - (A00 * mxd.y + A01 * myd.y));
                b1 = (myd.x - (A10 * mxd.x + A11 * myd.x)) + (c1 + myd.y - (A10 * mxd.y + A11 * myd.y));
                flags = TSP_VIEW_OK;
            }
        }
    }
    w.vres0[i] = r0;
    w.vres1[i] = r1;
    w.vres2[i] = make_uint2(flags, (uint32_t)npix);
    if (view_flags) view_flags[i] = flags;
    if (view_affine) {
        float* a = view_affine + 6 * i;
        a[0] = A00; a[1] = A01; a[2] = A10; a[3] = A11; a[4] = b0; a[5] = b1;
    }
}

// ---------------------------------------------------------------- FP64 helpers

// In-place Cholesky solve of the SPD system A x = b (A row-major N x N, lower
// triangle used).  Returns false if a pivot falls below rel * max diagonal.
template <int N>
__device__ bool chol_solve(double (&A)[N][N], double (&b)[N], double rel)
{
    double dmax = 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) dmax = fmax(dmax, A[k][k]);
    if (!(dmax > 0.0)) return false;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        double d = A[k][k];
#pragma unroll
        for (int j = 0; j < k; ++j) d -= A[k][j] * A[k][j];
        if (!(d > rel * dmax)) return false;
        const double l = sqrt(d);
        A[k][k] = l;
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            double x = A[i][k];
#pragma unroll
            for (int j = 0; j < k; ++j) x -= A[i][j] * A[k][j];
            A[i][k] = x / l;
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {          // L y = b
        double x = b[i];
#pragma unroll
        for (int j = 0; j < i; ++j) x -= A[i][j] * b[j];
        b[i] = x / A[i][i];
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {     // L^T x = y
        double x = b[i];
#pragma unroll
        for (int j = i + 1; j < N; ++j) x -= A[j][i] * b[j];
        b[i] = x / A[i][i];
    }
    return true;
}

// Cholesky with diagonal pivoting (largest remaining Schur diagonal first), which
// reveals rank deficiency: a rank-5 system (two views leave the variance along
// their common normal free) ends with a pivot at rounding level.  Returns false
// if a pivot falls below rel * max diagonal; otherwise b holds the solution.
template <int N>
__device__ bool chol_solve_pivoted(double (&A)[N][N], double (&b)[N], double rel)
{
    int perm[N];
    double dmax = 0.0;
    for (int k = 0; k < N; ++k) {
        perm[k] = k;
        dmax = fmax(dmax, A[k][k]);
    }
    if (!(dmax > 0.0)) return false;
    for (int k = 0; k < N; ++k) {
        int p = k;
        for (int j = k + 1; j < N; ++j)
            if (A[j][j] > A[p][p]) p = j;
        if (p != k) {
            for (int j = 0; j < N; ++j) { const double t = A[k][j]; A[k][j] = A[p][j]; A[p][j] = t; }
            for (int j = 0; j < N; ++j) { const double t = A[j][k]; A[j][k] = A[j][p]; A[j][p] = t; }
            const double tb = b[k]; b[k] = b[p]; b[p] = tb;
            const int tp = perm[k]; perm[k] = perm[p]; perm[p] = tp;
        }
        const double d = A[k][k];
        if (!(d > rel * dmax)) return false;
        const double l = sqrt(d);
        A[k][k] = l;
        for (int i = k + 1; i < N; ++i) A[i][k] /= l;
        for (int i = k + 1; i < N; ++i)
            for (int j = k + 1; j <= i; ++j) {
                A[i][j] -= A[i][k] * A[j][k];
                A[j][i] = A[i][j];
            }
    }
    double y[N];
    for (int i = 0; i < N; ++i) {
        double x = b[i];
        for (int j = 0; j < i; ++j) x -= A[i][j] * y[j];
        y[i] = x / A[i][i];
    }
    for (int i = N - 1; i >= 0; --i) {
        double x = y[i];
        for (int j = i + 1; j < N; ++j) x -= A[j][i] * y[j];
        y[i] = x / A[i][i];
    }
    for (int i = 0; i < N; ++i) b[perm[i]] = y[i];
    return true;
}

// Classic Jacobi: rotate away the largest off-diagonal element until the matrix
// is diagonal to rounding.  Eigenvectors are the columns of E.
__device__ void eig_sym3(double (&S)[3][3], double (&lam)[3], double (&E)[3][3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) E[i][j] = i == j ? 1.0 : 0.0;
    for (int it = 0; it < 64; ++it) {
        int p = 0, r = 1;
        double big = fabs(S[0][1]);
        if (fabs(S[0][2]) > big) { big = fabs(S[0][2]); p = 0; r = 2; }
        if (fabs(S[1][2]) > big) { big = fabs(S[1][2]); p = 1; r = 2; }
        const double scale = fabs(S[0][0]) + fabs(S[1][1]) + fabs(S[2][2]);
        if (big <= 1e-17 * scale || big == 0.0) break;
        const double app = S[p][p], arr = S[r][r], apr = S[p][r];
        const double th = 0.5 * (arr - app) / apr;
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
        // S <- G^T S G with G the rotation in the (p, r) plane
        for (int k = 0; k < 3; ++k) {
            const double skp = S[k][p], skr = S[k][r];
            S[k][p] = c * skp - sn * skr;
            S[k][r] = sn * skp + c * skr;
        }
        for (int k = 0; k < 3; ++k) {
            const double spk = S[p][k], srk = S[r][k];
            S[p][k] = c * spk - sn * srk;
            S[r][k] = sn * spk + c * srk;
        }
        for (int k = 0; k < 3; ++k) {
            const double ekp = E[k][p], ekr = E[k][r];
            E[k][p] = c * ekp - sn * ekr;
            E[k][r] = sn * ekp + c * ekr;
        }
    }
    lam[0] = S[0][0]; lam[1] = S[1][1]; lam[2] = S[2][2];
}

__device__ __forceinline__ void rank_ascending(const double (&x)[3], int (&o)[3])
{
    // stable: ties keep index order
    o[0] = 0; o[1] = 1; o[2] = 2;
    if (x[o[1]] < x[o[0]]) { const int t = o[0]; o[0] = o[1]; o[1] = t; }
    if (x[o[2]] < x[o[1]]) { const int t = o[1]; o[1] = o[2]; o[2] = t; }
    if (x[o[1]] < x[o[0]]) { const int t = o[0]; o[0] = o[1]; o[1] = t; }
}

__device__ void quat_of(const double (&R)[3][3], double (&q)[4])
{
    const double d0 = R[0][0], d1 = R[1][1], d2 = R[2][2], tr = d0 + d1 + d2;
    if (tr >= d0 && tr >= d1 && tr >= d2) {
        const double h = 2.0 * sqrt(1.0 + tr);
        q[0] = 0.25 * h; q[1] = (R[2][1] - R[1][2]) / h; q[2] = (R[0][2] - R[2][0]) / h; q[3] = (R[1][0] - R[0][1]) / h;
    } else if (d0 >= d1 && d0 >= d2) {
        const double h = 2.0 * sqrt(1.0 + d0 - d1 - d2);
        q[0] = (R[2][1] - R[1][2]) / h; q[1] = 0.25 * h; q[2] = (R[0][1] + R[1][0]) / h; q[3] = (R[0][2] + R[2][0]) / h;
    } else if (d1 >= d2) {
        const double h = 2.0 * sqrt(1.0 - d0 + d1 - d2);
        q[0] = (R[0][2] - R[2][0]) / h; q[1] = (R[0][1] + R[1][0]) / h; q[2] = 0.25 * h; q[3] = (R[1][2] + R[2][1]) / h;
    } else {
        const double h = 2.0 * sqrt(1.0 - d0 - d1 + d2);
        q[0] = (R[1][0] - R[0][1]) / h; q[1] = (R[0][2] + R[2][0]) / h; q[2] = (R[1][2] + R[2][1]) / h; q[3] = 0.25 * h;
    }
}

__global__ void __launch_bounds__(128) k_multiview(const ViewSet vs, const float4* __restrict__ mo,
                                                   const float4* __restrict__ qin,
                                                   const float4* __restrict__ sin_, const FitParams fp,
                                                   const Work w, float4* __restrict__ om,
                                                   float4* __restrict__ oq, float4* __restrict__ os,
                                                   uint32_t* __restrict__ ost)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= vs.n) return;
    const int n = vs.n;
    const float4 m = mo[g], qi = qin[g], si = sin_[g];
    int nv = 0;
    float sw = 0.f, npx = 0.f;
    for (int v = 0; v < vs.V; ++v) {
        const uint2 f = w.vres2[(size_t)v * n + g];
        if (f.x & TSP_VIEW_OK) {
            ++nv;
            sw += w.vres1[(size_t)v * n + g].w;
            npx += (float)f.y;
        }
    }
    uint32_t st = (uint32_t)min(nv, 255) << 16;
    if (nv < fp.min_views) st |= TSP_FEW_VIEWS;
    if (!(sw >= fp.sumw_min_total)) st |= TSP_LOW_ALPHA;
    if (npx < (float)fp.min_px_total) st |= TSP_FEW_PX;
    float4 outm = m, outq = qi, outs = si;
    if (st & (TSP_FEW_VIEWS | TSP_LOW_ALPHA | TSP_FEW_PX)) {
        om[g] = outm; oq[g] = outq; os[g] = outs; ost[g] = st;
        return;
    }

    // ---- a7 triangulation about the old mean
    float N00 = 0.f, N01 = 0.f, N02 = 0.f, N11 = 0.f, N12 = 0.f, N22 = 0.f;
    float r0 = 0.f, r1 = 0.f, r2 = 0.f;
    for (int v = 0; v < vs.V; ++v) {
        const size_t i = (size_t)v * n + g;
        if (!(w.vres2[i].x & TSP_VIEW_OK)) continue;
        const DevCam& c = vs.cam[v];
        const float4 a = w.vres0[i];
        const float zmu = c.R[6] * m.x + c.R[7] * m.y + c.R[8] * m.z + c.t[2];
        const float du = a.x - c.cx, dv = a.y - c.cy;
        const float ax = du * c.R[6] - c.fx * c.R[0], ay = du * c.R[7] - c.fx * c.R[1], az = du * c.R[8] - c.fx * c.R[2];
        const float bx = dv * c.R[6] - c.fy * c.R[3], by = dv * c.R[7] - c.fy * c.R[4], bz = dv * c.R[8] - c.fy * c.R[5];
        const float ra = -zmu * a.z, rb = -zmu * a.w;
        N00 += ax * ax + bx * bx; N01 += ax * ay + bx * by; N02 += ax * az + bx * bz;
        N11 += ay * ay + by * by; N12 += ay * az + by * bz; N22 += az * az + bz * bz;
        r0 += ax * ra + bx * rb; r1 += ay * ra + by * rb; r2 += az * ra + bz * rb;
    }
    double Nt[3][3] = {{N00, N01, N02}, {N01, N11, N12}, {N02, N12, N22}};
    double dl[3] = {r0, r1, r2};
    if (!chol_solve<3>(Nt, dl, 1e-24)) {
        om[g] = outm; oq[g] = outq; os[g] = outs; ost[g] = st | TSP_TRI_SINGULAR;
        return;
    }
    const double X[3] = {(double)m.x + dl[0], (double)m.y + dl[1], (double)m.z + dl[2]};
    st |= TSP_POS_OK;
    outm = make_float4((float)X[0], (float)X[1], (float)X[2], m.w);

    // ---- a8 covariance: 3 equations per solved view, unknowns (xx, xy, xz, yy, yz, zz)
    double A6[6][6], b6[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        b6[a] = 0.0;
#pragma unroll
        for (int b = 0; b < 6; ++b) A6[a][b] = 0.0;
    }
    for (int v = 0; v < vs.V; ++v) {
        const size_t i = (size_t)v * n + g;
        if (!(w.vres2[i].x & TSP_VIEW_OK)) continue;
        const DevCam& c = vs.cam[v];
        double p[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            p[k] = (double)c.R[3 * k] * X[0] + (double)c.R[3 * k + 1] * X[1] + (double)c.R[3 * k + 2] * X[2] + (double)c.t[k];
        const double iz = 1.0 / p[2];
        const double j00 = c.fx * iz, j02 = -c.fx * p[0] * iz * iz;
        const double j11 = c.fy * iz, j12 = -c.fy * p[1] * iz * iz;
        double T[2][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T[0][k] = j00 * c.R[k] + j02 * c.R[6 + k];
            T[1][k] = j11 * c.R[3 + k] + j12 * c.R[6 + k];
        }
        const float4 b0v = w.vres1[i], b1v = w.vres3[i];
        const double B0[3] = {b0v.x, b0v.y, b0v.z}, B1[3] = {b1v.x, b1v.y, b1v.z};
        const double rhs[3] = {B0[0] * B0[0] + B0[1] * B0[1] + B0[2] * B0[2],
                               B0[0] * B1[0] + B0[1] * B1[1] + B0[2] * B1[2],
                               B1[0] * B1[0] + B1[1] * B1[1] + B1[2] * B1[2]};
        const int ii[3] = {0, 0, 1}, jj[3] = {0, 1, 1};
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int a = ii[e], b = jj[e];
            double cf[6];
            cf[0] = T[a][0] * T[b][0];
            cf[1] = T[a][0] * T[b][1] + T[a][1] * T[b][0];
            cf[2] = T[a][0] * T[b][2] + T[a][2] * T[b][0];
            cf[3] = T[a][1] * T[b][1];
            cf[4] = T[a][1] * T[b][2] + T[a][2] * T[b][1];
            cf[5] = T[a][2] * T[b][2];
#pragma unroll
            for (int u = 0; u < 6; ++u) {
                b6[u] += cf[u] * rhs[e];
#pragma unroll
                for (int k = 0; k < 6; ++k) A6[u][k] += cf[u] * cf[k];
            }
        }
    }
    const double rc2 = (double)fp.cov_rcond_min * (double)fp.cov_rcond_min;
    if (!chol_solve_pivoted<6>(A6, b6, rc2)) {
        om[g] = outm; oq[g] = outq; os[g] = outs; ost[g] = st | TSP_COV_SINGULAR;
        return;
    }
    double S[3][3] = {{b6[0], b6[1], b6[2]}, {b6[1], b6[3], b6[4]}, {b6[2], b6[4], b6[5]}};

    // ---- a9 eigen decomposition and the reorder / sign rules
    double lam[3], E[3][3];
    eig_sym3(S, lam, E);
    if (!(lam[0] > 0.0) || !(lam[1] > 0.0) || !(lam[2] > 0.0)) {
        om[g] = outm; oq[g] = outq; os[g] = outs; ost[g] = st | TSP_NEG_EIG;
        return;
    }
    // old rotation from the normalised input quaternion (w, x, y, z)
    const double qn = sqrt((double)qi.x * qi.x + (double)qi.y * qi.y + (double)qi.z * qi.z + (double)qi.w * qi.w);
    const double qw = qi.x / qn, qx = qi.y / qn, qy = qi.z / qn, qz = qi.w / qn;
    const double Ro[3][3] = {
        {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
        {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
        {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
    const double so[3] = {si.x, si.y, si.z};
    int ro[3], rn[3];
    rank_ascending(so, ro);
    rank_ascending(lam, rn);
    double Rn[3][3], ln[3], al[3];
    for (int r = 0; r < 3; ++r) {
        const int k = ro[r], e = rn[r];
        ln[k] = lam[e];
        for (int i = 0; i < 3; ++i) Rn[i][k] = E[i][e];
    }
    for (int k = 0; k < 3; ++k) {
        double d = Rn[0][k] * Ro[0][k] + Rn[1][k] * Ro[1][k] + Rn[2][k] * Ro[2][k];
        if (d < 0.0) {
            for (int i = 0; i < 3; ++i) Rn[i][k] = -Rn[i][k];
            d = -d;
        }
        al[k] = d;
    }
    const double det = Rn[0][0] * (Rn[1][1] * Rn[2][2] - Rn[1][2] * Rn[2][1])
                     - Rn[0][1] * (Rn[1][0] * Rn[2][2] - Rn[1][2] * Rn[2][0])
                     + Rn[0][2] * (Rn[1][0] * Rn[2][1] - Rn[1][1] * Rn[2][0]);
    if (det < 0.0) {
        int kmin = 0;
        if (al[1] < al[kmin]) kmin = 1;
        if (al[2] < al[kmin]) kmin = 2;
        for (int i = 0; i < 3; ++i) Rn[i][kmin] = -Rn[i][kmin];
    }
    double qq[4];
    quat_of(Rn, qq);
    if (qq[0] * qw + qq[1] * qx + qq[2] * qy + qq[3] * qz < 0.0)
        for (int k = 0; k < 4; ++k) qq[k] = -qq[k];
    outq = make_float4((float)qq[0], (float)qq[1], (float)qq[2], (float)qq[3]);
    outs = make_float4((float)sqrt(ln[0]), (float)sqrt(ln[1]), (float)sqrt(ln[2]), 0.f);
    om[g] = outm; oq[g] = outq; os[g] = outs; ost[g] = st | TSP_COV_OK;
}

}  // namespace

cudaError_t launch_view_solve(const ViewSet& vs, const float4* mo, const float4* q, const float4* s,
                              const FitParams& fp, const Work& w, float* view_affine,
                              uint32_t* view_flags, cudaStream_t st)
{
    if (vs.n == 0 || vs.V == 0) return cudaSuccess;
    dim3 grid((vs.n + 255) / 256, vs.V);
    k_view_solve<<<grid, 256, 0, st>>>(vs, mo, q, s, fp, w, view_affine, view_flags);
    return cudaGetLastError();
}

cudaError_t launch_multiview(const ViewSet& vs, const float4* mo, const float4* q, const float4* s,
                             const FitParams& fp, const Work& w, float4* out_means, float4* out_quats,
                             float4* out_scales, uint32_t* out_status, cudaStream_t st)
{
    if (vs.n == 0) return cudaSuccess;
    k_multiview<<<(vs.n + 127) / 128, 128, 0, st>>>(vs, mo, q, s, fp, w, out_means, out_quats,
                                                     out_scales, out_status);
    return cudaGetLastError();
}

}  // namespace tsp

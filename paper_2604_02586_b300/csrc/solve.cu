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
//   the centre: no cancellation.  FP32 normal equations, double-float Cholesky.
// a8 (Sec. 4.4.2): vech(T Sigma T^T) = vech(Sigma_2D') per solved view with
//   T = J' W at the new mean, 6 unknowns.  Two views are always rank 5 (each T
//   annihilates its viewing ray d, so sym(d1 d2^T) is a null vector) and are
//   reported singular without a solve.  With 3+ views: FP32 rows, normal
//   equations accumulated from exact products in double-float, then a
//   double-float LDL^T with diagonal pivoting whose last pivot ratio decides rank
//   deficiency.
// a9 (Sec. 4.4.3): cyclic Jacobi in FP32 for the eigenvectors, eigenvalues as
//   double-float Rayleigh quotients; discard if an eigenvalue is <= 0; new axis k takes
//   the eigenpair whose rank matches the rank of the old scale s_k; each axis is
//   flipped to agree with the old one; a reflection is undone on the
//   least-aligned axis; the quaternion sign follows the old one.
#include "launch.h"

namespace tsp {

namespace {

// ---------------------------------------------------------------- double-float
// A value hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2 (Dekker's
// double-length arithmetic built on the error-free TwoSum and FMA-based TwoProd):
// about 48 significant bits.  It replaces FP64 in the small dense solves: this
// GPU's FP64 rate is a small fraction of its FP32 rate.
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_of(float a) { return df{a, 0.f}; }

__device__ __forceinline__ df df_norm(float a, float b)
{
    df r;
    two_sum(a, b, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df operator+(df a, df b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    df r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df operator-(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b)
{
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    df r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df operator*(df a, float b)
{
    float p, e;
    two_prod(a.hi, b, p, e);
    e = __fmaf_rn(a.lo, b, e);
    df r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// a / b: an FP32 quotient corrected once by the double-float remainder.
__device__ __forceinline__ df operator/(df a, df b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const df r = a - b * q1;
    const float q2 = __fdiv_rn(r.hi, b.hi);
    df q;
    fast_two_sum(q1, q2, q.hi, q.lo);
    return q;
}

// sqrt(a) for a > 0: the FP32 root corrected by the exact remainder a - x^2.
__device__ __forceinline__ df df_sqrt(df a)
{
    const float x = __fsqrt_rn(a.hi);
    float p, e;
    two_prod(x, x, p, e);
    const float rem = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), e), a.lo);
    df r;
    fast_two_sum(x, __fdiv_rn(rem, __fmul_rn(2.f, x)), r.hi, r.lo);
    return r;
}

__device__ __forceinline__ bool operator<(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df a, df b) { return b < a; }
__device__ __forceinline__ bool operator==(df a, df b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ float df_float(df a) { return __fadd_rn(a.hi, a.lo); }

// Per-view records written by a6 and read by a7/a8:
//   vres0 = (mu'_x, mu'_y, c_x, c_y) with c = mu' - mu_2D the shift of the centre,
//   vres1 = (B00, B01, B02, sum w), vres3 = (B10, B11, B12, 0) with Sigma_2D' = B B^T,
//   vres2 = (flags, pixels).

__global__ void __launch_bounds__(256) k_view_solve(const ViewSet vs, const FitParams fp, const Work w,
                                                    const FrameOut fo)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    const int n = vs.vn[v];
    if (g >= n || gate_closed(w)) return;
    const size_t i = (size_t)vs.vrec[v] + g;
    const int f = vs.vframe[v];
    const float4* __restrict__ mo = vs.fmo[f];
    const float4* __restrict__ q = vs.fq[f];
    const float4* __restrict__ s = vs.fs[f];
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
                const float4 rc3 = w.rec[4 * i + kRecCorner];
                const float2 rf = make_float2(rc3.z, rc3.w);
                const float co0 = (M[6] - M[1] * Y00 - M[2] * Y10) * isw + rf.x;
                const float co1 = (M[7] - M[1] * Y01 - M[2] * Y11) * isw + rf.y;
                A00 = 1.0f + Y00; A01 = Y10; A10 = Y01; A11 = 1.0f + Y11;
                KeyProj p;
                key_project(vs.cam[v], mo[g], q[g], s[g], vs.tiles_x[v], vs.tiles_y[v], vs.tw, vs.th, p);
                float2 mxd, myd;
                mean2d_df(vs.cam[v], mo[g], mxd, myd);
                // shift of the centre: mu' - mu = c_o + (I - A) delta
                const float rx = __fadd_rn(__fsub_rn(mxd.x, (float)(p.x0 * vs.tw)), mxd.y);
                const float ry = __fadd_rn(__fsub_rn(myd.x, (float)(p.y0 * vs.th)), myd.y);
                const float2 dl = moment_origin_shift(mxd, myd, rx, ry, p.x0 * vs.tw, p.y0 * vs.th,
                                                      vs.cam[v].W, vs.cam[v].H);
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
    // per-frame outputs: [views of the frame][n]
    const size_t fi = (size_t)(v - vs.fview[f]) * n + g;
    if (fo.view_flags[f]) fo.view_flags[f][fi] = flags;
    if (fo.view_affine[f]) {
        float* a = fo.view_affine[f] + 6 * fi;
        a[0] = A00; a[1] = A01; a[2] = A10; a[3] = A11; a[4] = b0; a[5] = b1;
    }
}

// ---------------------------------------------------------------- solvers

// In-place Cholesky solve of the SPD system A x = b (A row-major N x N, lower
// triangle used).  Returns false if a pivot falls below rel * max diagonal.
template <int N>
__device__ bool chol_solve(df (&A)[N][N], df (&b)[N], float rel)
{
    float dmax = 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k) dmax = fmaxf(dmax, A[k][k].hi);
    if (!(dmax > 0.f)) return false;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        df d = A[k][k];
#pragma unroll
        for (int j = 0; j < k; ++j) d = d - A[k][j] * A[k][j];
        if (!(d.hi > rel * dmax)) return false;
        const df l = df_sqrt(d);
        A[k][k] = l;
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            df x = A[i][k];
#pragma unroll
            for (int j = 0; j < k; ++j) x = x - A[i][j] * A[k][j];
            A[i][k] = x / l;
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {          // L y = b
        df x = b[i];
#pragma unroll
        for (int j = 0; j < i; ++j) x = x - A[i][j] * b[j];
        b[i] = x / A[i][i];
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {     // L^T x = y
        df x = b[i];
#pragma unroll
        for (int j = i + 1; j < N; ++j) x = x - A[j][i] * b[j];
        b[i] = x / A[i][i];
    }
    return true;
}

// Packed lower storage of a symmetric N x N matrix: element (i, j) at tri(i, j).
__host__ __device__ constexpr int tri(int i, int j)
{
    return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i;
}

// hi + lo += a * b with the product taken exactly (TwoProd) and added by TwoSum:
// the sum keeps ~44 bits, so normal equations formed from FP32 rows lose nothing
// to the squaring of their condition number.
__device__ __forceinline__ void df_madd(float& hi, float& lo, float a, float b)
{
    float p, e, s, f;
    two_prod(a, b, p, e);
    two_sum(hi, p, s, f);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(f, e));
}

// Swap rows and columns k < j of a packed symmetric matrix, including the
// already factorised columns (rows of L) left of k.
template <int N>
__device__ __forceinline__ void sym_swap(df (&A)[N * (N + 1) / 2], int k, int j)
{
#pragma unroll
    for (int m = 0; m < N; ++m) {
        if (m == k || m == j) continue;
        const df t = A[tri(k, m)];
        A[tri(k, m)] = A[tri(j, m)];
        A[tri(j, m)] = t;
    }
    const df t = A[tri(k, k)];
    A[tri(k, k)] = A[tri(j, j)];
    A[tri(j, j)] = t;
}

// Solve A x = b for symmetric positive semi-definite A (packed, N x N) by LDL^T
// with diagonal pivoting: each step takes the largest remaining Schur diagonal,
// so a rank-deficient system ends with a pivot at rounding level.  Returns false
// when a pivot is <= rel * (largest diagonal of A); otherwise b holds x.  Every
// index is a compile-time constant after unrolling, so A stays in registers.
template <int N>
__device__ __forceinline__ bool ldl_solve_pivoted(df (&A)[N * (N + 1) / 2], df (&b)[N], float rel)
{
    static_assert(N <= 8, "permutation packed as 4-bit fields");
    uint32_t perm = 0;                       // original index of row i in bits 4i..4i+3
    df dinv[N];
    float dmax = 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        perm |= (uint32_t)k << (4 * k);
        dmax = fmaxf(dmax, A[tri(k, k)].hi);
    }
    if (!(dmax > 0.f)) return false;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        int p = k;
        df best = A[tri(k, k)];
#pragma unroll
        for (int j = k + 1; j < N; ++j)
            if (A[tri(j, j)] > best) { best = A[tri(j, j)]; p = j; }
#pragma unroll
        for (int j = k + 1; j < N; ++j)
            if (p == j) {
                sym_swap<N>(A, k, j);
                const df tb = b[k]; b[k] = b[j]; b[j] = tb;
                const uint32_t x = ((perm >> (4 * k)) ^ (perm >> (4 * j))) & 15u;
                perm ^= (x << (4 * k)) | (x << (4 * j));
            }
        const df d = A[tri(k, k)];
        if (!(d.hi > rel * dmax)) return false;
        const df di = df_of(1.f) / d;
        dinv[k] = di;
#pragma unroll
        for (int i = k + 1; i < N; ++i) {          // Schur complement of the pivot
            const df li = A[tri(i, k)] * di;
#pragma unroll
            for (int j = k + 1; j <= i; ++j) A[tri(i, j)] = A[tri(i, j)] - li * A[tri(j, k)];
        }
#pragma unroll
        for (int i = k + 1; i < N; ++i) A[tri(i, k)] = A[tri(i, k)] * di;   // column k of L
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {                  // L z = P b, then D^-1
#pragma unroll
        for (int m = 0; m < i; ++m) b[i] = b[i] - A[tri(i, m)] * b[m];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) b[i] = b[i] * dinv[i];
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {             // L^T y = z
#pragma unroll
        for (int m = i + 1; m < N; ++m) b[i] = b[i] - A[tri(m, i)] * b[m];
    }
    df x[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {                  // x = P^T y
        x[j] = df_of(0.f);
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (((perm >> (4 * i)) & 15u) == (uint32_t)j) x[j] = b[i];
    }
#pragma unroll
    for (int j = 0; j < N; ++j) b[j] = x[j];
    return true;
}

// One Jacobi rotation of the symmetric 3x3 S in the (p, r) plane (q the third
// index) that zeroes S[p][r]; the diagonal is updated by +-t S[p][r] and the
// zeroed entry is set exactly, so off-diagonal rounding never feeds back into
// the diagonal.  E accumulates the rotations in its columns.  Skips the pair
// once |S[p][r]| <= 2^-24 sqrt|S[p][p] S[r][r]| (relative-accuracy criterion).
__device__ __forceinline__ bool jacobi_rotate(float (&S)[3][3], float (&E)[3][3], int p, int r, int q)
{
    const float apr = S[p][r], app = S[p][p], arr = S[r][r];
    if (!(fabsf(apr) > 5.9604645e-8f * sqrtf(fabsf(app * arr)))) return false;
    const float th = __fdiv_rn(__fsub_rn(arr, app), __fmul_rn(2.f, apr));
    const float ath = fabsf(th);
    const float t = ath > 1e18f ? __fdiv_rn(0.5f, th)
                                : copysignf(__fdiv_rn(1.f, __fadd_rn(ath, __fsqrt_rn(__fmaf_rn(th, th, 1.f)))), th);
    const float c = __frsqrt_rn(__fmaf_rn(t, t, 1.f)), s = __fmul_rn(t, c);
    const float tau = __fmul_rn(t, apr);
    S[p][p] = __fsub_rn(app, tau);
    S[r][r] = __fadd_rn(arr, tau);
    S[p][r] = S[r][p] = 0.f;
    const float sqp = S[q][p], sqr = S[q][r];
    S[q][p] = S[p][q] = c * sqp - s * sqr;
    S[q][r] = S[r][q] = s * sqp + c * sqr;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float ekp = E[k][p], ekr = E[k][r];
        E[k][p] = c * ekp - s * ekr;
        E[k][r] = s * ekp + c * ekr;
    }
    return true;
}

// Cyclic Jacobi on the FP32 copy of S (at most 8 sweeps; quadratic convergence
// ends it in 2-4), eigenvalues refined as double-float Rayleigh quotients
// e^T S e / e^T e.
// The Rayleigh quotient error is second order in the FP32 eigenvector error, so
// the small eigenvalues of an elongated Gaussian keep their relative accuracy.
__device__ __forceinline__ void eig_sym3(const df (&S)[3][3], df (&lam)[3], float (&E)[3][3])
{
    float A[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            A[i][j] = df_float(S[i][j]);
            E[i][j] = i == j ? 1.f : 0.f;
        }
    for (int sweep = 0; sweep < 8; ++sweep) {
        bool any = jacobi_rotate(A, E, 0, 1, 2);
        any |= jacobi_rotate(A, E, 0, 2, 1);
        any |= jacobi_rotate(A, E, 1, 2, 0);
        if (!any) break;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float e0 = E[0][k], e1 = E[1][k], e2 = E[2][k];
        const df se0 = S[0][0] * e0 + S[0][1] * e1 + S[0][2] * e2;
        const df se1 = S[1][0] * e0 + S[1][1] * e1 + S[1][2] * e2;
        const df se2 = S[2][0] * e0 + S[2][1] * e1 + S[2][2] * e2;
        const df ee = df_of(e0) * df_of(e0) + df_of(e1) * df_of(e1) + df_of(e2) * df_of(e2);
        lam[k] = (se0 * e0 + se1 * e1 + se2 * e2) / ee;
    }
}

// Rank of each of three values in ascending order, ties by index (a stable sort).
template <typename T>
__device__ __forceinline__ void ranks3(const T (&x)[3], int (&rk)[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        rk[k] = 0;
#pragma unroll
        for (int j = 0; j < 3; ++j)
            if (j != k && (x[j] < x[k] || (x[j] == x[k] && j < k))) ++rk[k];
    }
}

// Unit quaternion (w, x, y, z) of a rotation matrix, branch on the largest of
// the trace and the diagonal (Shepperd) so the divisor is never small.
__device__ __forceinline__ void quat_of(const float (&R)[3][3], float (&q)[4])
{
    const float d0 = R[0][0], d1 = R[1][1], d2 = R[2][2], tr = d0 + d1 + d2;
    if (tr >= d0 && tr >= d1 && tr >= d2) {
        const float h = 2.f * sqrtf(1.f + tr), ih = 1.f / h;
        q[0] = 0.25f * h; q[1] = (R[2][1] - R[1][2]) * ih; q[2] = (R[0][2] - R[2][0]) * ih; q[3] = (R[1][0] - R[0][1]) * ih;
    } else if (d0 >= d1 && d0 >= d2) {
        const float h = 2.f * sqrtf(1.f + d0 - d1 - d2), ih = 1.f / h;
        q[0] = (R[2][1] - R[1][2]) * ih; q[1] = 0.25f * h; q[2] = (R[0][1] + R[1][0]) * ih; q[3] = (R[0][2] + R[2][0]) * ih;
    } else if (d1 >= d2) {
        const float h = 2.f * sqrtf(1.f - d0 + d1 - d2), ih = 1.f / h;
        q[0] = (R[0][2] - R[2][0]) * ih; q[1] = (R[0][1] + R[1][0]) * ih; q[2] = 0.25f * h; q[3] = (R[1][2] + R[2][1]) * ih;
    } else {
        const float h = 2.f * sqrtf(1.f - d0 - d1 + d2), ih = 1.f / h;
        q[0] = (R[1][0] - R[0][1]) * ih; q[1] = (R[0][2] + R[2][0]) * ih; q[2] = (R[1][2] + R[2][1]) * ih; q[3] = 0.25f * h;
    }
}

// grid (ceil(nmax/128), F): one thread per Gaussian of frame blockIdx.y, over the
// frame's views [fview[f], fview[f+1]).
__global__ void __launch_bounds__(128) k_multiview(const ViewSet vs, const FitParams fp, const Work w,
                                                   const FrameOut fo)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int f = blockIdx.y;
    if (g >= vs.fn[f] || gate_closed(w)) return;
    const int v0 = vs.fview[f], v1 = vs.fview[f + 1];
    float4* __restrict__ om = fo.means[f];
    float4* __restrict__ oq = fo.quats[f];
    float4* __restrict__ os = fo.scales[f];
    uint32_t* __restrict__ ost = fo.status[f];
    const float4 m = vs.fmo[f][g], qi = vs.fq[f][g], si = vs.fs[f][g];

    // One pass over the views gathers the view counts (status) and a7's normal
    // equations about the old mean.  The records of kChunkA views are loaded
    // before any of them is used, whatever their flags (every record of the
    // frame exists), so the pass pays one memory latency per chunk, not two per
    // view; sums are still taken in view order.
    constexpr int kChunkA = 6;
    int nv = 0;
    float sw = 0.f, npx = 0.f;
    float N00 = 0.f, N01 = 0.f, N02 = 0.f, N11 = 0.f, N12 = 0.f, N22 = 0.f;
    float r0 = 0.f, r1 = 0.f, r2 = 0.f;
    for (int vb = v0; vb < v1; vb += kChunkA) {
        uint2 fl[kChunkA];
        float swv[kChunkA];
        float4 a[kChunkA];
#pragma unroll
        for (int u = 0; u < kChunkA; ++u) {
            fl[u] = make_uint2(0u, 0u);
            swv[u] = 0.f;
            a[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (vb + u < v1) {
                const size_t i = (size_t)vs.vrec[vb + u] + g;
                fl[u] = w.vres2[i];
                swv[u] = w.vres1[i].w;
                a[u] = w.vres0[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kChunkA; ++u) {
            if (!(fl[u].x & TSP_VIEW_OK)) continue;      // also every slot past v1
            const DevCam& c = vs.cam[vb + u];
            ++nv;
            sw += swv[u];
            npx += (float)fl[u].y;
            const float zmu = c.R[6] * m.x + c.R[7] * m.y + c.R[8] * m.z + c.t[2];
            const float du = a[u].x - c.cx, dv = a[u].y - c.cy;
            const float ax = du * c.R[6] - c.fx * c.R[0], ay = du * c.R[7] - c.fx * c.R[1], az = du * c.R[8] - c.fx * c.R[2];
            const float bx = dv * c.R[6] - c.fy * c.R[3], by = dv * c.R[7] - c.fy * c.R[4], bz = dv * c.R[8] - c.fy * c.R[5];
            const float ra = -zmu * a[u].z, rb = -zmu * a[u].w;
            N00 += ax * ax + bx * bx; N01 += ax * ay + bx * by; N02 += ax * az + bx * bz;
            N11 += ay * ay + by * by; N12 += ay * az + by * bz; N22 += az * az + bz * bz;
            r0 += ax * ra + bx * rb; r1 += ay * ra + by * rb; r2 += az * ra + bz * rb;
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
    df Nt[3][3] = {{df_of(N00), df_of(N01), df_of(N02)},
                   {df_of(N01), df_of(N11), df_of(N12)},
                   {df_of(N02), df_of(N12), df_of(N22)}};
    df dl[3] = {df_of(r0), df_of(r1), df_of(r2)};
    if (!chol_solve<3>(Nt, dl, 1e-24f)) {
        om[g] = outm; oq[g] = outq; os[g] = outs; ost[g] = st | TSP_TRI_SINGULAR;
        return;
    }
    const float X0 = df_float(df_of(m.x) + dl[0]), X1 = df_float(df_of(m.y) + dl[1]),
                X2 = df_float(df_of(m.z) + dl[2]);
    st |= TSP_POS_OK;
    outm = make_float4(X0, X1, X2, m.w);

    // ---- a8 covariance: 3 equations per solved view, unknowns (xx, xy, xz, yy, yz, zz).
    // Each view's T = J' W annihilates its viewing ray d, so sym(d1 d2^T) solves the
    // homogeneous system of any two views: two views are always rank 5.
    if (nv < 3) {
        om[g] = outm; oq[g] = outq; os[g] = outs; ost[g] = st | TSP_COV_SINGULAR;
        return;
    }
    float Ah[21], Al[21], bh[6], bl[6];
#pragma unroll
    for (int u = 0; u < 21; ++u) { Ah[u] = 0.f; Al[u] = 0.f; }
#pragma unroll
    for (int u = 0; u < 6; ++u) { bh[u] = 0.f; bl[u] = 0.f; }
    // the next view's records are loaded while this view's equations are added
    uint32_t fl_n = w.vres2[(size_t)vs.vrec[v0] + g].x;
    float4 b0_n = w.vres1[(size_t)vs.vrec[v0] + g], b1_n = w.vres3[(size_t)vs.vrec[v0] + g];
    for (int v = v0; v < v1; ++v) {
        const uint32_t flv = fl_n;
        const float4 b0v = b0_n, b1v = b1_n;
        if (v + 1 < v1) {
            const size_t i1 = (size_t)vs.vrec[v + 1] + g;
            fl_n = w.vres2[i1].x;
            b0_n = w.vres1[i1];
            b1_n = w.vres3[i1];
        }
        if (!(flv & TSP_VIEW_OK)) continue;
        const DevCam& c = vs.cam[v];
        const float p0 = fmaf(c.R[0], X0, fmaf(c.R[1], X1, fmaf(c.R[2], X2, c.t[0])));
        const float p1 = fmaf(c.R[3], X0, fmaf(c.R[4], X1, fmaf(c.R[5], X2, c.t[1])));
        const float p2 = fmaf(c.R[6], X0, fmaf(c.R[7], X1, fmaf(c.R[8], X2, c.t[2])));
        const float iz = 1.f / p2;
        const float j00 = c.fx * iz, j02 = -c.fx * p0 * iz * iz;
        const float j11 = c.fy * iz, j12 = -c.fy * p1 * iz * iz;
        float T[2][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T[0][k] = fmaf(j00, c.R[k], j02 * c.R[6 + k]);
            T[1][k] = fmaf(j11, c.R[3 + k], j12 * c.R[6 + k]);
        }
        const float rhs[3] = {fmaf(b0v.x, b0v.x, fmaf(b0v.y, b0v.y, b0v.z * b0v.z)),
                              fmaf(b0v.x, b1v.x, fmaf(b0v.y, b1v.y, b0v.z * b1v.z)),
                              fmaf(b1v.x, b1v.x, fmaf(b1v.y, b1v.y, b1v.z * b1v.z))};
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int a = e == 2 ? 1 : 0, b = e == 0 ? 0 : 1;
            float cf[6];
            cf[0] = T[a][0] * T[b][0];
            cf[1] = fmaf(T[a][0], T[b][1], T[a][1] * T[b][0]);
            cf[2] = fmaf(T[a][0], T[b][2], T[a][2] * T[b][0]);
            cf[3] = T[a][1] * T[b][1];
            cf[4] = fmaf(T[a][1], T[b][2], T[a][2] * T[b][1]);
            cf[5] = T[a][2] * T[b][2];
#pragma unroll
            for (int u = 0; u < 6; ++u) {
                df_madd(bh[u], bl[u], cf[u], rhs[e]);
#pragma unroll
                for (int k = 0; k <= u; ++k) df_madd(Ah[tri(u, k)], Al[tri(u, k)], cf[u], cf[k]);
            }
        }
    }
    df A6[21], b6[6];
#pragma unroll
    for (int u = 0; u < 21; ++u) A6[u] = df_norm(Ah[u], Al[u]);
#pragma unroll
    for (int u = 0; u < 6; ++u) b6[u] = df_norm(bh[u], bl[u]);
    const float rc2 = fp.cov_rcond_min * fp.cov_rcond_min;
    if (!ldl_solve_pivoted<6>(A6, b6, rc2)) {
        om[g] = outm; oq[g] = outq; os[g] = outs; ost[g] = st | TSP_COV_SINGULAR;
        return;
    }
    const df S[3][3] = {{b6[0], b6[1], b6[2]}, {b6[1], b6[3], b6[4]}, {b6[2], b6[4], b6[5]}};

    // ---- a9 eigen decomposition and the reorder / sign rules
    df lam[3];
    float E[3][3];
    eig_sym3(S, lam, E);
    if (!(lam[0].hi > 0.f) || !(lam[1].hi > 0.f) || !(lam[2].hi > 0.f)) {
        om[g] = outm; oq[g] = outq; os[g] = outs; ost[g] = st | TSP_NEG_EIG;
        return;
    }
    // old rotation from the normalised input quaternion (w, x, y, z)
    const float qn = 1.f / sqrtf(qi.x * qi.x + qi.y * qi.y + qi.z * qi.z + qi.w * qi.w);
    const float qw = qi.x * qn, qx = qi.y * qn, qy = qi.z * qn, qz = qi.w * qn;
    const float Ro[3][3] = {
        {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
        {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
        {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)}};
    const float so[3] = {si.x, si.y, si.z};
    int ro[3], rn[3];
    ranks3(so, ro);
    ranks3(lam, rn);
    float Rn[3][3], al[3];
    df ln[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)          // old axis k takes the eigenpair of equal rank
#pragma unroll
        for (int e = 0; e < 3; ++e)
            if (ro[k] == rn[e]) {
                ln[k] = lam[e];
#pragma unroll
                for (int i = 0; i < 3; ++i) Rn[i][k] = E[i][e];
            }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float d = Rn[0][k] * Ro[0][k] + Rn[1][k] * Ro[1][k] + Rn[2][k] * Ro[2][k];
        if (d < 0.f) {
#pragma unroll
            for (int i = 0; i < 3; ++i) Rn[i][k] = -Rn[i][k];
            d = -d;
        }
        al[k] = d;
    }
    const float det = Rn[0][0] * (Rn[1][1] * Rn[2][2] - Rn[1][2] * Rn[2][1])
                    - Rn[0][1] * (Rn[1][0] * Rn[2][2] - Rn[1][2] * Rn[2][0])
                    + Rn[0][2] * (Rn[1][0] * Rn[2][1] - Rn[1][1] * Rn[2][0]);
    if (det < 0.f) {
        int kmin = al[1] < al[0] ? 1 : 0;
        if (al[2] < fminf(al[0], al[1])) kmin = 2;
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (k == kmin) {
#pragma unroll
                for (int i = 0; i < 3; ++i) Rn[i][k] = -Rn[i][k];
            }
    }
    float qq[4];
    quat_of(Rn, qq);
    if (qq[0] * qw + qq[1] * qx + qq[2] * qy + qq[3] * qz < 0.f)
#pragma unroll
        for (int k = 0; k < 4; ++k) qq[k] = -qq[k];
    outq = make_float4(qq[0], qq[1], qq[2], qq[3]);
    outs = make_float4(sqrtf(df_float(ln[0])), sqrtf(df_float(ln[1])), sqrtf(df_float(ln[2])), 0.f);
    om[g] = outm; oq[g] = outq; os[g] = outs; ost[g] = st | TSP_COV_OK;
}

}  // namespace

cudaError_t launch_view_solve(const ViewSet& vs, const FitParams& fp, const Work& w, const FrameOut& fo,
                              cudaStream_t st)
{
    if (vs.nmax == 0 || vs.V == 0) return cudaSuccess;
    dim3 grid((vs.nmax + 255) / 256, vs.V);
    k_view_solve<<<grid, 256, 0, st>>>(vs, fp, w, fo);
    return cudaGetLastError();
}

cudaError_t launch_multiview(const ViewSet& vs, const FitParams& fp, const Work& w, const FrameOut& fo,
                             cudaStream_t st)
{
    if (vs.nmax == 0 || vs.F == 0) return cudaSuccess;
    dim3 grid((vs.nmax + 127) / 128, vs.F);
    k_multiview<<<grid, 128, 0, st>>>(vs, fp, w, fo);
    return cudaGetLastError();
}

}  // namespace tsp

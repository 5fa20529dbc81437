/*
 * oracle.c -- plain, slow CPU oracle of the TrackerSplat motion-compensation path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header or constant
 * table with the CUDA path; it is written from the paper (arXiv 2604.02586):
 *
 *   Eq. 1 (Sec. 3.1)   projection of a 3D Gaussian, Sigma_2D = J W Sigma_3D W^T J^T
 *   Sec. 3.1           front-to-back alpha blending in depth order
 *   Eq. 2 (Sec. 4.2)   Sigma_2D' = A Sigma_2D A^T,  mu_2D' = A mu_2D + b
 *   Eq. 3/4 (Sec. 4.3) weighted least squares [A|b] = V1^-1 V2, w_i = alpha_i T_i
 *   Sec. 4.3.5         per-Gaussian accumulation during rendering, per-view discard
 *   Sec. 4.4.1         triangulation of mu_3D' "using SVD"
 *   Sec. 4.4.2         linear system Sigma_2D' = J W Sigma_3D' W^T J^T (3 eq./view, 6 unknowns)
 *   Sec. 4.4.3         eigen decomposition, negative-eigenvalue discard, reorder
 *   Sec. 4.5.2         static-pixel counters accumulated during rendering
 *   Sec. 5.1           thresholds: det V1 < 1e-12, accumulated alpha < 1e-3, < 2 px;
 *                      multi-view: < 2 views, accumulated alpha < 1e-3, < 3 px
 *
 * Precision: FP64 everywhere, except the "key path" (culling, depth key, tile
 * rectangle) which decides integers and is therefore evaluated in FP32 with a
 * fixed sequence of correctly rounded operations (fmaf, *, +, -, /, sqrtf,
 * floorf, ceilf, fmaxf, fminf, fabsf); compile with -ffp-contract=off.  The static
 * pixel test |x' - x| < 1 is also an integer decision on FP32 tracks, taken in FP32.
 *
 * Readings where the paper is silent (listed in the design notes):
 *   pixel (i,j) has centre (i+0.5, j+0.5); blending constants follow 3DGS
 *   (near plane 0.2, +0.3 px^2 dilation, alpha = min(0.99, o G), skip alpha < 1/255,
 *   stop before a Gaussian when T (1 - alpha) < 1e-4, radius ceil(3 sqrt(lambda_max)));
 *   visibility-0 pixels blend but add no moments; w = alpha T with T the
 *   transmittance before the Gaussian; motion uses the undilated Sigma_2D;
 *   Eq. 4 is accumulated with pixel coordinates measured from mu_2D (a change of
 *   origin under which [A|b] is unchanged); an added per-view guard rejects pixel
 *   sets whose weighted scatter has lambda_min < 1e-4 px^2; triangulation is the
 *   inhomogeneous linear DLT in pixel units; the covariance system uses J at the
 *   new mean; unsolvable Gaussians keep their input parameters.
 *
 * Parallelism: OpenMP over views (each view owns its accumulators), so every
 * sum is taken in a fixed order and results are deterministic.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Public types (mirrored by oracle/__init__.py)                              */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R[9];          /* world -> camera rotation, row-major */
    float t[3];          /* world -> camera translation */
} orc_camera;

typedef struct {
    int32_t tile_w, tile_h;
    double det_min;        /* Sec. 5.1: det V1 below this -> unsolvable in the view   */
    double sumw_min_view;  /* Sec. 5.1: accumulated alpha (sum of w) below this       */
    int32_t min_px_view;   /* Sec. 5.1: fewer pixels than this                        */
    double lam_min_px2;    /* added guard on the weighted pixel scatter (px^2)        */
    int32_t min_views;     /* Sec. 5.1: fewer valid views than this                   */
    double sumw_min_total; /* Sec. 5.1: accumulated alpha over views below this       */
    int32_t min_px_total;  /* Sec. 5.1: fewer pixels over views than this             */
    double cov_rcond_min;  /* covariance system: sigma_min / sigma_max below this     */
} orc_options;

/* Per-view flags */
enum { OV_OK = 1, OV_FEW_PX = 2, OV_LOW_ALPHA = 4, OV_SINGULAR = 8, OV_CULLED = 16 };
/* Per-Gaussian status bits; bits 16..23 hold the number of valid views */
enum { OS_POS_OK = 1, OS_COV_OK = 2, OS_NEG_EIG = 4, OS_FEW_VIEWS = 8, OS_LOW_ALPHA = 16,
       OS_FEW_PX = 32, OS_COV_SINGULAR = 64, OS_TRI_SINGULAR = 128 };

/* Blend constants as FP32 numbers (the thresholds are FP32 constants). */
#define ALPHA_MIN ((double)(1.0f / 255.0f))
#define ALPHA_MAX ((double)0.99f)
#define T_MIN ((double)1e-4f)
#define DILATION 0.3
/* Relative half-widths of the windows in which an FP32 evaluation may decide a
 * blend threshold differently from this FP64 one (used to flag, not to decide). */
#define ALPHA_WIN (2e-4 * ALPHA_MIN)
#define T_WIN (1e-4 * T_MIN)

/* ------------------------------------------------------------------------- */
/* Key path (FP32, fixed operation order)                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t visible;       /* 0 = culled or no tile touched */
    uint32_t depth_bits;   /* bits of the FP32 camera depth */
    int32_t x0, y0, x1, y1;/* tile rectangle [x0,x1) x [y0,y1) */
    uint32_t tiles;        /* (x1-x0)*(y1-y0) or 0 */
} keyrec;

static void keypath(const float* m, const float* q, const float* s, const orc_camera* c,
                    int tw, int th, keyrec* k)
{
    memset(k, 0, sizeof(*k));
    const float* R = c->R;
    const float px = fmaf(R[0], m[0], fmaf(R[1], m[1], fmaf(R[2], m[2], c->t[0])));
    const float py = fmaf(R[3], m[0], fmaf(R[4], m[1], fmaf(R[5], m[2], c->t[1])));
    const float pz = fmaf(R[6], m[0], fmaf(R[7], m[1], fmaf(R[8], m[2], c->t[2])));
    if (!(pz > 0.2f)) return;
    const float iz = 1.0f / pz;
    const float un = px * iz, vn = py * iz;
    const float limx = 1.3f * ((0.5f * (float)c->width) / c->fx);
    const float limy = 1.3f * ((0.5f * (float)c->height) / c->fy);
    if (!(fabsf(un) <= limx) || !(fabsf(vn) <= limy)) return;
    const float mx = fmaf(c->fx, un, c->cx);
    const float my = fmaf(c->fy, vn, c->cy);

    const float n2 = fmaf(q[0], q[0], fmaf(q[1], q[1], fmaf(q[2], q[2], q[3] * q[3])));
    if (!(n2 > 0.0f)) return;
    const float inv = 1.0f / sqrtf(n2);
    const float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
    const float xx = x * x, yy = y * y, zz = z * z;
    const float xy = x * y, xz = x * z, yz = y * z;
    const float wx = w * x, wy = w * y, wz = w * z;
    float Q[3][3];
    Q[0][0] = 1.0f - 2.0f * (yy + zz); Q[0][1] = 2.0f * (xy - wz);        Q[0][2] = 2.0f * (xz + wy);
    Q[1][0] = 2.0f * (xy + wz);        Q[1][1] = 1.0f - 2.0f * (xx + zz); Q[1][2] = 2.0f * (yz - wx);
    Q[2][0] = 2.0f * (xz - wy);        Q[2][1] = 2.0f * (yz + wx);        Q[2][2] = 1.0f - 2.0f * (xx + yy);
    float M[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = Q[i][j] * s[j];

    const float j00 = c->fx * iz, j02 = -((c->fx * un) * iz);
    const float j11 = c->fy * iz, j12 = -((c->fy * vn) * iz);
    float T[2][3];
    for (int j = 0; j < 3; ++j) {
        T[0][j] = fmaf(j00, R[0 * 3 + j], j02 * R[2 * 3 + j]);
        T[1][j] = fmaf(j11, R[1 * 3 + j], j12 * R[2 * 3 + j]);
    }
    float Vm[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            Vm[i][j] = fmaf(T[i][0], M[0][j], fmaf(T[i][1], M[1][j], T[i][2] * M[2][j]));
    const float a = fmaf(Vm[0][0], Vm[0][0], fmaf(Vm[0][1], Vm[0][1], Vm[0][2] * Vm[0][2]));
    const float b = fmaf(Vm[0][0], Vm[1][0], fmaf(Vm[0][1], Vm[1][1], Vm[0][2] * Vm[1][2]));
    const float cc = fmaf(Vm[1][0], Vm[1][0], fmaf(Vm[1][1], Vm[1][1], Vm[1][2] * Vm[1][2]));
    const float ad = a + 0.3f, cd = cc + 0.3f;
    const float det = fmaf(ad, cd, -(b * b));
    if (!(det > 0.0f)) return;
    const float mid = 0.5f * (ad + cd);
    const float disc = fmaxf(0.1f, fmaf(mid, mid, -det));
    const float lam = mid + sqrtf(disc);
    const float r = ceilf(3.0f * sqrtf(lam));

    const int tiles_x = (c->width + tw - 1) / tw, tiles_y = (c->height + th - 1) / th;
    const float ftw = (float)tw, fth = (float)th;
    const float gx = (float)tiles_x, gy = (float)tiles_y;
    const float fx0 = fminf(fmaxf(floorf((mx - r) / ftw), 0.0f), gx);
    const float fx1 = fminf(fmaxf(floorf((mx + r) / ftw) + 1.0f, 0.0f), gx);
    const float fy0 = fminf(fmaxf(floorf((my - r) / fth), 0.0f), gy);
    const float fy1 = fminf(fmaxf(floorf((my + r) / fth) + 1.0f, 0.0f), gy);
    const int x0 = (int)fx0, x1 = (int)fx1, y0 = (int)fy0, y1 = (int)fy1;
    if (x1 <= x0 || y1 <= y0) return;
    k->visible = 1;
    memcpy(&k->depth_bits, &pz, 4);
    k->x0 = x0; k->x1 = x1; k->y0 = y0; k->y1 = y1;
    k->tiles = (uint32_t)((x1 - x0) * (y1 - y0));
}

/* ------------------------------------------------------------------------- */
/* FP64 geometry                                                             */
/* ------------------------------------------------------------------------- */

static void quat_to_rot(const float* qf, double Q[3][3], double qn[4])
{
    double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
    const double n = sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z;
    Q[0][0] = 1 - 2 * (y * y + z * z); Q[0][1] = 2 * (x * y - w * z);     Q[0][2] = 2 * (x * z + w * y);
    Q[1][0] = 2 * (x * y + w * z);     Q[1][1] = 1 - 2 * (x * x + z * z); Q[1][2] = 2 * (y * z - w * x);
    Q[2][0] = 2 * (x * z - w * y);     Q[2][1] = 2 * (y * z + w * x);     Q[2][2] = 1 - 2 * (x * x + y * y);
}

/* Sigma_3D = Q diag(s^2) Q^T (Sec. 3.1) */
static void cov3d(const float* q, const float* s, double S[3][3])
{
    double Q[3][3], qn[4];
    quat_to_rot(q, Q, qn);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += Q[i][k] * ((double)s[k] * s[k]) * Q[j][k];
            S[i][j] = acc;
        }
}

/* J W for the camera at world point X (Eq. 1): J is the Jacobian of the
 * perspective map at the camera-space point p = R X + t. */
static void jw_at(const orc_camera* c, const double X[3], double T[2][3], double p[3])
{
    for (int i = 0; i < 3; ++i)
        p[i] = c->R[3 * i] * X[0] + c->R[3 * i + 1] * X[1] + c->R[3 * i + 2] * X[2] + c->t[i];
    const double J[2][3] = {{c->fx / p[2], 0.0, -c->fx * p[0] / (p[2] * p[2])},
                            {0.0, c->fy / p[2], -c->fy * p[1] / (p[2] * p[2])}};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            T[i][j] = J[i][0] * c->R[j] + J[i][1] * c->R[3 + j] + J[i][2] * c->R[6 + j];
}

typedef struct {
    double mx, my;       /* mu_2D */
    double cov[3];       /* undilated Sigma_2D: xx, xy, yy */
    double conic[3];     /* inverse of the dilated Sigma_2D */
    double opacity;
    double color[3];
} proj64;

static void project64(const float* mo, const float* q, const float* s, const orc_camera* c,
                      proj64* P)
{
    const double X[3] = {mo[0], mo[1], mo[2]};
    double T[2][3], p[3], S[3][3];
    jw_at(c, X, T, p);
    cov3d(q, s, S);
    double TS[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            TS[i][j] = T[i][0] * S[0][j] + T[i][1] * S[1][j] + T[i][2] * S[2][j];
    double C[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            C[i][j] = TS[i][0] * T[j][0] + TS[i][1] * T[j][1] + TS[i][2] * T[j][2];
    P->mx = c->fx * p[0] / p[2] + c->cx;
    P->my = c->fy * p[1] / p[2] + c->cy;
    P->cov[0] = C[0][0]; P->cov[1] = 0.5 * (C[0][1] + C[1][0]); P->cov[2] = C[1][1];
    const double a = P->cov[0] + DILATION, b = P->cov[1], d = P->cov[2] + DILATION;
    const double det = a * d - b * b;
    P->conic[0] = d / det; P->conic[1] = -b / det; P->conic[2] = a / det;
    P->opacity = mo[3];
    P->color[0] = P->color[1] = P->color[2] = 0.0;
}

/* Real spherical harmonics up to degree 3 (Condon-Shortley phase), evaluated at
 * the unit direction (x, y, z) from the camera centre to the Gaussian. */
static void sh_basis(double x, double y, double z, double Y[16])
{
    const double pi = 3.14159265358979323846;
    const double k0 = 0.5 / sqrt(pi);
    const double k1 = sqrt(3.0 / (4.0 * pi));
    const double k2a = 0.5 * sqrt(15.0 / pi), k2b = 0.25 * sqrt(5.0 / pi), k2c = 0.25 * sqrt(15.0 / pi);
    const double k3a = 0.25 * sqrt(35.0 / (2.0 * pi)), k3b = 0.5 * sqrt(105.0 / pi);
    const double k3c = 0.25 * sqrt(21.0 / (2.0 * pi)), k3d = 0.25 * sqrt(7.0 / pi);
    const double k3e = 0.25 * sqrt(105.0 / pi);
    const double xx = x * x, yy = y * y, zz = z * z;
    Y[0] = k0;
    Y[1] = -k1 * y; Y[2] = k1 * z; Y[3] = -k1 * x;
    Y[4] = k2a * x * y; Y[5] = -k2a * y * z; Y[6] = k2b * (2 * zz - xx - yy);
    Y[7] = -k2a * x * z; Y[8] = k2c * (xx - yy);
    Y[9] = -k3a * y * (3 * xx - yy); Y[10] = k3b * x * y * z;
    Y[11] = -k3c * y * (4 * zz - xx - yy); Y[12] = k3d * z * (2 * zz - 3 * xx - 3 * yy);
    Y[13] = -k3c * x * (4 * zz - xx - yy); Y[14] = k3e * z * (xx - yy);
    Y[15] = -k3a * x * (xx - 3 * yy);
}

static void sh_color(const float* mo, const float* sh, int deg, const orc_camera* c, double rgb[3])
{
    /* camera centre C = -R^T t */
    double C[3];
    for (int i = 0; i < 3; ++i)
        C[i] = -(c->R[i] * (double)c->t[0] + c->R[3 + i] * (double)c->t[1] + c->R[6 + i] * (double)c->t[2]);
    double d[3] = {mo[0] - C[0], mo[1] - C[1], mo[2] - C[2]};
    const double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    d[0] /= n; d[1] /= n; d[2] /= n;
    double Y[16];
    sh_basis(d[0], d[1], d[2], Y);
    const int nb = (deg + 1) * (deg + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.5;
        for (int k = 0; k < nb; ++k) acc += Y[k] * sh[k * 3 + ch];
        rgb[ch] = acc > 0 ? acc : 0;
    }
}

/* ------------------------------------------------------------------------- */
/* Small dense linear algebra (FP64)                                          */
/* ------------------------------------------------------------------------- */

/* Solve A X = B for 3x3 A and 3 x nrhs B by LU with partial pivoting.
 * Returns 0 if a pivot is exactly zero. */
static int lu_solve3(const double Ain[3][3], double* B, int nrhs)
{
    double A[3][3];
    memcpy(A, Ain, sizeof(A));
    for (int k = 0; k < 3; ++k) {
        int p = k;
        for (int i = k + 1; i < 3; ++i)
            if (fabs(A[i][k]) > fabs(A[p][k])) p = i;
        if (A[p][k] == 0.0) return 0;
        if (p != k) {
            for (int j = 0; j < 3; ++j) { double t = A[k][j]; A[k][j] = A[p][j]; A[p][j] = t; }
            for (int j = 0; j < nrhs; ++j) { double t = B[k * nrhs + j]; B[k * nrhs + j] = B[p * nrhs + j]; B[p * nrhs + j] = t; }
        }
        for (int i = k + 1; i < 3; ++i) {
            const double f = A[i][k] / A[k][k];
            for (int j = k; j < 3; ++j) A[i][j] -= f * A[k][j];
            for (int j = 0; j < nrhs; ++j) B[i * nrhs + j] -= f * B[k * nrhs + j];
        }
    }
    for (int k = 2; k >= 0; --k)
        for (int j = 0; j < nrhs; ++j) {
            double acc = B[k * nrhs + j];
            for (int i = k + 1; i < 3; ++i) acc -= A[k][i] * B[i * nrhs + j];
            B[k * nrhs + j] = acc / A[k][k];
        }
    return 1;
}

static double det3(const double A[3][3])
{
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
         - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
         + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

/* One-sided Jacobi SVD (Hestenes) of the m x n column-major matrix A (n <= 8).
 * On return A holds U * diag(sigma), V is n x n (column-major), sigma[n]. */
static void jacobi_svd(double* A, int m, int n, double* V, double* sigma)
{
    for (int i = 0; i < n * n; ++i) V[i] = 0.0;
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double alpha = 0, beta = 0, gamma = 0;
                for (int i = 0; i < m; ++i) {
                    const double ap = A[p * m + i], aq = A[q * m + i];
                    alpha += ap * ap; beta += aq * aq; gamma += ap * aq;
                }
                if (gamma == 0.0) continue;
                const double r = fabs(gamma) / sqrt(alpha * beta);
                if (r > off) off = r;
                if (r < 1e-15) continue;
                const double zeta = (beta - alpha) / (2.0 * gamma);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int i = 0; i < m; ++i) {
                    const double ap = A[p * m + i], aq = A[q * m + i];
                    A[p * m + i] = cs * ap - sn * aq;
                    A[q * m + i] = sn * ap + cs * aq;
                }
                for (int i = 0; i < n; ++i) {
                    const double vp = V[p * n + i], vq = V[q * n + i];
                    V[p * n + i] = cs * vp - sn * vq;
                    V[q * n + i] = sn * vp + cs * vq;
                }
            }
        if (off < 1e-15) break;
    }
    for (int j = 0; j < n; ++j) {
        double s = 0;
        for (int i = 0; i < m; ++i) s += A[j * m + i] * A[j * m + i];
        sigma[j] = sqrt(s);
    }
}

/* Least squares min ||A x - b|| by SVD (A m x n column-major, consumed).
 * Returns sigma_min / sigma_max. */
static double svd_lstsq(double* A, int m, int n, const double* b, double* x)
{
    double V[64], sig[8], c[8];
    jacobi_svd(A, m, n, V, sig);
    double smax = 0, smin = INFINITY;
    for (int j = 0; j < n; ++j) { if (sig[j] > smax) smax = sig[j]; if (sig[j] < smin) smin = sig[j]; }
    for (int j = 0; j < n; ++j) {
        /* A[:,j] = sigma_j u_j, so (u_j . b) / sigma_j = (A[:,j] . b) / sigma_j^2 */
        double acc = 0;
        for (int i = 0; i < m; ++i) acc += A[j * m + i] * b[i];
        c[j] = sig[j] > 0 ? acc / (sig[j] * sig[j]) : 0.0;
    }
    for (int i = 0; i < n; ++i) {
        double acc = 0;
        for (int j = 0; j < n; ++j) acc += V[j * n + i] * c[j];
        x[i] = acc;
    }
    return smax > 0 ? smin / smax : 0.0;
}

/* Cyclic Jacobi eigen decomposition of a symmetric 3x3 matrix.
 * Eigenvalues in lam[k], eigenvectors in the columns of E. */
static void jacobi_eig3(const double Sin[3][3], double lam[3], double E[3][3])
{
    double A[3][3];
    memcpy(A, Sin, sizeof(A));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) E[i][j] = (i == j);
    for (int sweep = 0; sweep < 100; ++sweep) {
        const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        const double diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off <= 1e-32 * diag || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {        /* A <- A G */
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {        /* A <- G^T A */
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {        /* E <- E G */
                    const double ekp = E[k][p], ekq = E[k][q];
                    E[k][p] = c * ekp - s * ekq;
                    E[k][q] = s * ekp + c * ekq;
                }
            }
    }
    for (int k = 0; k < 3; ++k) lam[k] = A[k][k];
}

/* ------------------------------------------------------------------------- */
/* Binning: per (view, tile) lists of (depth bits, Gaussian) in ascending order */
/* ------------------------------------------------------------------------- */

typedef struct {
    int V, n, tw, th;
    int32_t* tiles_x; int32_t* tiles_y; int64_t* toff;   /* per view */
    int64_t NT;
    keyrec* keys;        /* [V][n] */
} binctx;

static int cmp_u64(const void* a, const void* b)
{
    const uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : x > y;
}

static void binctx_init(binctx* B, int n, int V, const float* mo, const float* q, const float* s,
                        const orc_camera* cams, int tw, int th)
{
    B->V = V; B->n = n; B->tw = tw; B->th = th;
    B->tiles_x = malloc(sizeof(int32_t) * (V > 0 ? V : 1));
    B->tiles_y = malloc(sizeof(int32_t) * (V > 0 ? V : 1));
    B->toff = malloc(sizeof(int64_t) * (V + 1));
    B->toff[0] = 0;
    for (int v = 0; v < V; ++v) {
        B->tiles_x[v] = (cams[v].width + tw - 1) / tw;
        B->tiles_y[v] = (cams[v].height + th - 1) / th;
        B->toff[v + 1] = B->toff[v] + (int64_t)B->tiles_x[v] * B->tiles_y[v];
    }
    B->NT = B->toff[V];
    B->keys = malloc(sizeof(keyrec) * ((size_t)V * n + 1));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)V * n; ++i) {
        const int v = (int)(i / n), g = (int)(i % n);
        keypath(mo + 4 * (size_t)g, q + 4 * (size_t)g, s + 4 * (size_t)g, &cams[v], tw, th,
                &B->keys[i]);
    }
}

static void binctx_free(binctx* B)
{
    free(B->tiles_x); free(B->tiles_y); free(B->toff); free(B->keys);
}

/* Fill per-tile lists: offsets[NT+1], entries[K] sorted by (depth bits, g). */
static void build_lists(const binctx* B, int64_t* offsets, uint64_t* entries)
{
    const int64_t NT = B->NT;
    memset(offsets, 0, sizeof(int64_t) * (NT + 1));
    for (int v = 0; v < B->V; ++v)
        for (int g = 0; g < B->n; ++g) {
            const keyrec* k = &B->keys[(size_t)v * B->n + g];
            if (!k->visible) continue;
            for (int ty = k->y0; ty < k->y1; ++ty)
                for (int tx = k->x0; tx < k->x1; ++tx)
                    offsets[B->toff[v] + (int64_t)ty * B->tiles_x[v] + tx + 1]++;
        }
    for (int64_t t = 0; t < NT; ++t) offsets[t + 1] += offsets[t];
    int64_t* fill = calloc((size_t)NT + 1, sizeof(int64_t));
    for (int v = 0; v < B->V; ++v)
        for (int g = 0; g < B->n; ++g) {
            const keyrec* k = &B->keys[(size_t)v * B->n + g];
            if (!k->visible) continue;
            const uint64_t e = ((uint64_t)k->depth_bits << 32) | (uint32_t)g;
            for (int ty = k->y0; ty < k->y1; ++ty)
                for (int tx = k->x0; tx < k->x1; ++tx) {
                    const int64_t t = B->toff[v] + (int64_t)ty * B->tiles_x[v] + tx;
                    entries[offsets[t] + fill[t]++] = e;
                }
        }
    free(fill);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < NT; ++t)
        qsort(entries + offsets[t], (size_t)(offsets[t + 1] - offsets[t]), sizeof(uint64_t), cmp_u64);
}

static int64_t count_pairs(const binctx* B)
{
    int64_t K = 0;
    for (int64_t i = 0; i < (int64_t)B->V * B->n; ++i) K += B->keys[i].tiles;
    return K;
}

/* ------------------------------------------------------------------------- */
/* Exported: key path and binning                                            */
/* ------------------------------------------------------------------------- */

/* Per (view, Gaussian) key-path results; arrays are [V][n] (rect: [V][n][4]). */
int orc_keys(int n, int V, const float* means_opacity, const float* quats, const float* scales,
             const orc_camera* cams, int tile_w, int tile_h,
             int32_t* visible, uint32_t* depth_bits, int32_t* rect, uint32_t* tiles_touched)
{
    binctx B;
    binctx_init(&B, n, V, means_opacity, quats, scales, cams, tile_w, tile_h);
    for (int64_t i = 0; i < (int64_t)V * n; ++i) {
        const keyrec* k = &B.keys[i];
        if (visible) visible[i] = k->visible;
        if (depth_bits) depth_bits[i] = k->depth_bits;
        if (tiles_touched) tiles_touched[i] = k->tiles;
        if (rect) { rect[4 * i] = k->x0; rect[4 * i + 1] = k->y0; rect[4 * i + 2] = k->x1; rect[4 * i + 3] = k->y1; }
    }
    binctx_free(&B);
    return 0;
}

int64_t orc_count_pairs(int n, int V, const float* means_opacity, const float* quats,
                        const float* scales, const orc_camera* cams, int tile_w, int tile_h)
{
    binctx B;
    binctx_init(&B, n, V, means_opacity, quats, scales, cams, tile_w, tile_h);
    const int64_t K = count_pairs(&B);
    binctx_free(&B);
    return K;
}

/* offsets: [NT+1] with NT = sum over views of tiles_x * tiles_y; entries: [K]. */
int orc_bin(int n, int V, const float* means_opacity, const float* quats, const float* scales,
            const orc_camera* cams, int tile_w, int tile_h, int64_t* offsets, uint64_t* entries)
{
    binctx B;
    binctx_init(&B, n, V, means_opacity, quats, scales, cams, tile_w, tile_h);
    build_lists(&B, offsets, entries);
    binctx_free(&B);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Raster-accumulate (Sec. 4.3.5) and render (Sec. 3.1)                        */
/* ------------------------------------------------------------------------- */

/* Moment record per (view, Gaussian); coordinates are pixel centres minus mu_2D.
 *  0..5  V1 = sum w [x;1][x;1]^T : xx, xy, x1, yy, y1, 11 (= sum w)      (Eq. 4)
 *  6..11 V2 = sum w [x;1] x'^T   : x x', x y', y x', y y', 1 x', 1 y'   (Eq. 4)
 *  12    sum of w over static pixels (|x' - x| < 1 px)                  (Sec. 4.5.2)
 *  13    number of pixels that added moments
 *  14    number of those pixels that are static
 *  15    sum of w at pixels where this or an earlier blend decision (alpha vs
 *        1/255, T (1 - alpha) vs 1e-4) lay inside the FP32 window -- bookkeeping
 *        for comparisons with an FP32 implementation, not part of the method
 *  16    number of such pixels
 *  17    sum of w |d|^2 (d = the track's displacement) -- bookkeeping: the scale
 *        of the displacement terms, for modelling FP32 rounding of the sums */
#define NMOM 18

typedef struct {
    const float* disp;    /* [H][W][2] */
    const uint8_t* vis;   /* [H][W]    */
} orc_tracks;

/* Blend the pixels of one view.  mom (nullable) receives moments for the
 * Gaussians with want[g] != 0 (want NULL = all); rgb/T/flag (nullable) receive
 * the render.  tile_need (nullable) restricts work to tiles with a non-zero entry. */
static void blend_view(int v, const binctx* B, const int64_t* offsets, const uint64_t* entries,
                       const proj64* P /* [n] for this view */, const orc_camera* cam,
                       const orc_tracks* tr, const uint8_t* want, const uint8_t* tile_need,
                       double* mom /* [n][NMOM] */, float* rgb, float* Tout, uint8_t* flag)
{
    const int tw = B->tw, th = B->th, W = cam->width, H = cam->height;
    for (int ty = 0; ty < B->tiles_y[v]; ++ty)
        for (int tx = 0; tx < B->tiles_x[v]; ++tx) {
            const int64_t t = B->toff[v] + (int64_t)ty * B->tiles_x[v] + tx;
            if (tile_need && !tile_need[t - B->toff[v]]) continue;
            const int64_t e0 = offsets[t], e1 = offsets[t + 1];
            for (int py = ty * th; py < (ty + 1) * th && py < H; ++py)
                for (int px = tx * tw; px < (tx + 1) * tw && px < W; ++px) {
                    const double xc = px + 0.5, yc = py + 0.5;
                    const size_t pix = (size_t)py * W + px;
                    float ddx = 0.0f, ddy = 0.0f;
                    int vis = 0;
                    if (tr && tr->disp) {
                        ddx = tr->disp[2 * pix]; ddy = tr->disp[2 * pix + 1];
                        vis = tr->vis[pix] != 0;
                    }
                    /* static test in FP32, as the tracks are FP32 (Sec. 4.5.2) */
                    const int stat = fmaf(ddx, ddx, ddy * ddy) < 1.0f;
                    double T = 1.0, col[3] = {0, 0, 0};
                    int pert = 0;
                    for (int64_t e = e0; e < e1; ++e) {
                        const int g = (int)(uint32_t)entries[e];
                        const proj64* G = &P[g];
                        const double dx = xc - G->mx, dy = yc - G->my;
                        const double qf = G->conic[0] * dx * dx + 2.0 * G->conic[1] * dx * dy
                                        + G->conic[2] * dy * dy;
                        double alpha = G->opacity * exp(-0.5 * qf);
                        if (alpha > ALPHA_MAX) alpha = ALPHA_MAX;
                        if (fabs(alpha - ALPHA_MIN) <= ALPHA_WIN) {
                            pert = 1;
                            if (mom && vis && (!want || want[g]) && alpha < ALPHA_MIN) {
                                mom[(size_t)g * NMOM + 16] += 1.0;   /* the FP32 side may add this pixel */
                            }
                        }
                        if (alpha < ALPHA_MIN) continue;
                        const double Tn = T * (1.0 - alpha);
                        if (fabs(Tn - T_MIN) <= T_WIN) {
                            pert = 1;
                            if (mom && vis && (!want || want[g]) && Tn < T_MIN)
                                mom[(size_t)g * NMOM + 16] += 1.0;
                        }
                        if (Tn < T_MIN) break;
                        const double w = alpha * T;
                        if (rgb)
                            for (int ch = 0; ch < 3; ++ch) col[ch] += w * G->color[ch];
                        if (mom && vis && (!want || want[g])) {
                            double* M = mom + (size_t)g * NMOM;
                            if (pert) { M[15] += w; M[16] += 1.0; }
                            const double xp = dx + ddx, yp = dy + ddy;   /* x' - mu_2D */
                            M[0] += w * dx * dx; M[1] += w * dx * dy; M[2] += w * dx;
                            M[3] += w * dy * dy; M[4] += w * dy;      M[5] += w;
                            M[6] += w * dx * xp; M[7] += w * dx * yp;
                            M[8] += w * dy * xp; M[9] += w * dy * yp;
                            M[10] += w * xp;     M[11] += w * yp;
                            if (stat) { M[12] += w; M[14] += 1.0; }
                            M[13] += 1.0;
                            M[17] += w * ((double)ddx * ddx + (double)ddy * ddy);
                        }
                        T = Tn;
                    }
                    if (rgb)
                        for (int ch = 0; ch < 3; ++ch) rgb[3 * pix + ch] = (float)col[ch];
                    if (Tout) Tout[pix] = (float)T;
                    if (flag) flag[pix] = (uint8_t)pert;
                }
        }
}

/* ------------------------------------------------------------------------- */
/* Per-view solve (Eq. 4, Eq. 2, Sec. 4.3.5, Sec. 5.1)                         */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint32_t flags;
    double A[2][2], b[2];      /* [A|b] in absolute pixel coordinates */
    double mu_new[2];          /* mu_2D' = A mu_2D + b */
    double cov_new[3];         /* Sigma_2D' = A Sigma_2D A^T (xx, xy, yy) */
} viewsol;

static void view_solve(const double* M, const proj64* G, const orc_options* o, viewsol* S)
{
    memset(S, 0, sizeof(*S));
    const double sw = M[5];
    if (M[13] < o->min_px_view) S->flags |= OV_FEW_PX;
    if (!(sw >= o->sumw_min_view)) S->flags |= OV_LOW_ALPHA;
    if (S->flags) return;
    const double V1[3][3] = {{M[0], M[1], M[2]}, {M[1], M[3], M[4]}, {M[2], M[4], M[5]}};
    /* weighted pixel scatter C = (sum w x x^T)/sum w - m m^T, m = (sum w x)/sum w */
    const double mx = M[2] / sw, my = M[4] / sw;
    const double cxx = M[0] / sw - mx * mx, cxy = M[1] / sw - mx * my, cyy = M[3] / sw - my * my;
    const double tr = cxx + cyy, dt = cxx * cyy - cxy * cxy;
    const double lmin = 0.5 * (tr - sqrt(fmax(tr * tr - 4.0 * dt, 0.0)));
    if (!(det3(V1) >= o->det_min) || !(lmin >= o->lam_min_px2)) { S->flags |= OV_SINGULAR; return; }
    double Z[6] = {M[6], M[7], M[8], M[9], M[10], M[11]};   /* V2, 3x2 row-major */
    if (!lu_solve3(V1, Z, 2)) { S->flags |= OV_SINGULAR; return; }
    /* x' - mu = Z^T [x - mu; 1]  ->  A = Z[0:2]^T, intercept c = Z[2] */
    S->A[0][0] = Z[0]; S->A[0][1] = Z[2];
    S->A[1][0] = Z[1]; S->A[1][1] = Z[3];
    const double c0 = Z[4], c1 = Z[5];
    S->mu_new[0] = G->mx + c0;
    S->mu_new[1] = G->my + c1;
    S->b[0] = S->mu_new[0] - (S->A[0][0] * G->mx + S->A[0][1] * G->my);
    S->b[1] = S->mu_new[1] - (S->A[1][0] * G->mx + S->A[1][1] * G->my);
    const double C[2][2] = {{G->cov[0], G->cov[1]}, {G->cov[1], G->cov[2]}};
    double AC[2][2], N[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) AC[i][j] = S->A[i][0] * C[0][j] + S->A[i][1] * C[1][j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) N[i][j] = AC[i][0] * S->A[j][0] + AC[i][1] * S->A[j][1];
    S->cov_new[0] = N[0][0]; S->cov_new[1] = 0.5 * (N[0][1] + N[1][0]); S->cov_new[2] = N[1][1];
    S->flags = OV_OK;
}

/* ------------------------------------------------------------------------- */
/* Multi-view update (Sec. 4.4)                                               */
/* ------------------------------------------------------------------------- */

static void rank3(const double v[3], int order[3])
{
    /* indices sorted by ascending value, ties by index (stable) */
    order[0] = 0; order[1] = 1; order[2] = 2;
    for (int i = 1; i < 3; ++i)
        for (int j = i; j > 0 && v[order[j]] < v[order[j - 1]]; --j) {
            const int t = order[j]; order[j] = order[j - 1]; order[j - 1] = t;
        }
}

static void rot_to_quat(const double R[3][3], double q[4])
{
    /* Shepperd's method: branch on the largest of trace and the diagonal */
    const double tr = R[0][0] + R[1][1] + R[2][2];
    if (tr >= R[0][0] && tr >= R[1][1] && tr >= R[2][2]) {
        const double r = sqrt(1.0 + tr);
        q[0] = 0.5 * r;
        q[1] = (R[2][1] - R[1][2]) / (2 * r);
        q[2] = (R[0][2] - R[2][0]) / (2 * r);
        q[3] = (R[1][0] - R[0][1]) / (2 * r);
    } else if (R[0][0] >= R[1][1] && R[0][0] >= R[2][2]) {
        const double r = sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]);
        q[1] = 0.5 * r;
        q[0] = (R[2][1] - R[1][2]) / (2 * r);
        q[2] = (R[0][1] + R[1][0]) / (2 * r);
        q[3] = (R[0][2] + R[2][0]) / (2 * r);
    } else if (R[1][1] >= R[2][2]) {
        const double r = sqrt(1.0 - R[0][0] + R[1][1] - R[2][2]);
        q[2] = 0.5 * r;
        q[0] = (R[0][2] - R[2][0]) / (2 * r);
        q[1] = (R[0][1] + R[1][0]) / (2 * r);
        q[3] = (R[1][2] + R[2][1]) / (2 * r);
    } else {
        const double r = sqrt(1.0 - R[0][0] - R[1][1] + R[2][2]);
        q[3] = 0.5 * r;
        q[0] = (R[1][0] - R[0][1]) / (2 * r);
        q[1] = (R[0][2] + R[2][0]) / (2 * r);
        q[2] = (R[1][2] + R[2][1]) / (2 * r);
    }
}

typedef struct {
    double mean[3], quat[4], scale[3];
    uint32_t status;
    double cov3d[6];      /* fitted Sigma_3D' (xx, xy, xz, yy, yz, zz), 0 if not fitted */
} gaussout;

/* sols: [V] per-view solutions of this Gaussian; moms: [V] pointers to its moments */
static void multiview_fit(int V, const orc_camera* cams, const viewsol* sols, const double* const* moms,
                          const float* mo, const float* qf, const float* sf, const orc_options* o,
                          gaussout* out)
{
    memset(out, 0, sizeof(*out));
    for (int i = 0; i < 3; ++i) out->mean[i] = mo[i];
    for (int i = 0; i < 4; ++i) out->quat[i] = qf[i];
    for (int i = 0; i < 3; ++i) out->scale[i] = sf[i];
    int nv = 0;
    double sw = 0, npx = 0;
    for (int v = 0; v < V; ++v)
        if (sols[v].flags & OV_OK) { nv++; sw += moms[v][5]; npx += moms[v][13]; }
    uint32_t st = (uint32_t)(nv > 255 ? 255 : nv) << 16;
    if (nv < o->min_views) st |= OS_FEW_VIEWS;
    if (!(sw >= o->sumw_min_total)) st |= OS_LOW_ALPHA;
    if (npx < o->min_px_total) st |= OS_FEW_PX;
    if (st & (OS_FEW_VIEWS | OS_LOW_ALPHA | OS_FEW_PX)) { out->status = st; return; }

    /* Triangulation (Sec. 4.4.1): rows (u' P_3 - P_1), (v' P_3 - P_2), P = K [R|t] */
    const int m = 2 * nv;
    double* A = malloc(sizeof(double) * 3 * m);
    double* rhs = malloc(sizeof(double) * m);
    int r = 0;
    for (int v = 0; v < V; ++v) {
        if (!(sols[v].flags & OV_OK)) continue;
        const orc_camera* c = &cams[v];
        double P[3][4];
        for (int j = 0; j < 3; ++j) {
            P[0][j] = (double)c->fx * c->R[j] + (double)c->cx * c->R[6 + j];
            P[1][j] = (double)c->fy * c->R[3 + j] + (double)c->cy * c->R[6 + j];
            P[2][j] = c->R[6 + j];
        }
        P[0][3] = (double)c->fx * c->t[0] + (double)c->cx * c->t[2];
        P[1][3] = (double)c->fy * c->t[1] + (double)c->cy * c->t[2];
        P[2][3] = c->t[2];
        const double uv[2] = {sols[v].mu_new[0], sols[v].mu_new[1]};
        for (int k = 0; k < 2; ++k, ++r) {
            for (int j = 0; j < 3; ++j) A[j * m + r] = uv[k] * P[2][j] - P[k][j];
            rhs[r] = -(uv[k] * P[2][3] - P[k][3]);
        }
    }
    double X[3];
    const double rc = svd_lstsq(A, m, 3, rhs, X);
    free(A); free(rhs);
    if (!(rc > 1e-12)) { out->status = st | OS_TRI_SINGULAR; return; }
    st |= OS_POS_OK;
    for (int i = 0; i < 3; ++i) out->mean[i] = X[i];

    /* Covariance (Sec. 4.4.2): vech(T Sigma T^T) = vech(Sigma_2D'), T = J' W at mu_3D' */
    const int mc = 3 * nv;
    double* Ac = malloc(sizeof(double) * 6 * mc);
    double* bc = malloc(sizeof(double) * mc);
    static const int ki[6] = {0, 0, 0, 1, 1, 2}, li[6] = {0, 1, 2, 1, 2, 2};
    static const int pi_[3] = {0, 0, 1}, pj_[3] = {0, 1, 1};
    r = 0;
    for (int v = 0; v < V; ++v) {
        if (!(sols[v].flags & OV_OK)) continue;
        double T[2][3], p[3];
        jw_at(&cams[v], X, T, p);
        for (int e = 0; e < 3; ++e, ++r) {
            const int i = pi_[e], j = pj_[e];
            for (int u = 0; u < 6; ++u) {
                const int k = ki[u], l = li[u];
                Ac[u * mc + r] = (k == l) ? T[i][k] * T[j][k] : T[i][k] * T[j][l] + T[i][l] * T[j][k];
            }
            bc[r] = sols[v].cov_new[e];
        }
    }
    double sig[6];
    const double rcc = svd_lstsq(Ac, mc, 6, bc, sig);
    free(Ac); free(bc);
    if (!(rcc >= o->cov_rcond_min)) { out->status = st | OS_COV_SINGULAR; return; }
    for (int i = 0; i < 6; ++i) out->cov3d[i] = sig[i];

    /* Eigen decomposition and the reorder / sign rules (Sec. 4.4.3) */
    const double S[3][3] = {{sig[0], sig[1], sig[2]}, {sig[1], sig[3], sig[4]}, {sig[2], sig[4], sig[5]}};
    double lam[3], E[3][3];
    jacobi_eig3(S, lam, E);
    if (!(lam[0] > 0) || !(lam[1] > 0) || !(lam[2] > 0)) { out->status = st | OS_NEG_EIG; return; }
    double Q[3][3], qn[4];
    quat_to_rot(qf, Q, qn);
    const double sold[3] = {sf[0], sf[1], sf[2]};
    int ro[3], rn[3];
    rank3(sold, ro);
    rank3(lam, rn);
    double Rn[3][3], ln[3];
    for (int rr = 0; rr < 3; ++rr) {
        const int k = ro[rr], e = rn[rr];
        ln[k] = lam[e];
        for (int i = 0; i < 3; ++i) Rn[i][k] = E[i][e];
    }
    double dots[3];
    for (int k = 0; k < 3; ++k) {
        double d = 0;
        for (int i = 0; i < 3; ++i) d += Rn[i][k] * Q[i][k];
        if (d < 0) { for (int i = 0; i < 3; ++i) Rn[i][k] = -Rn[i][k]; d = -d; }
        dots[k] = d;
    }
    if (det3(Rn) < 0) {
        int kmin = 0;
        for (int k = 1; k < 3; ++k) if (dots[k] < dots[kmin]) kmin = k;
        for (int i = 0; i < 3; ++i) Rn[i][kmin] = -Rn[i][kmin];
    }
    double qq[4];
    rot_to_quat(Rn, qq);
    if (qq[0] * qn[0] + qq[1] * qn[1] + qq[2] * qn[2] + qq[3] * qn[3] < 0)
        for (int i = 0; i < 4; ++i) qq[i] = -qq[i];
    for (int i = 0; i < 4; ++i) out->quat[i] = qq[i];
    for (int k = 0; k < 3; ++k) out->scale[k] = sqrt(ln[k]);
    out->status = st | OS_COV_OK;
}

/* ------------------------------------------------------------------------- */
/* Exported: the whole path                                                   */
/* ------------------------------------------------------------------------- */

typedef struct {
    /* per (view, Gaussian), [V][n][...]; each nullable */
    double* moments;        /* [V][n][16], see NMOM */
    double* mean2d;         /* [V][n][2]  mu_2D */
    double* cov2d;          /* [V][n][3]  undilated Sigma_2D */
    uint32_t* view_flags;   /* [V][n]     OV_* */
    double* view_affine;    /* [V][n][6]  A00 A01 A10 A11 b0 b1 */
    double* view_mean2d;    /* [V][n][2]  mu_2D' */
    double* view_cov2d;     /* [V][n][3]  Sigma_2D' */
    /* per Gaussian, [n][...]; each nullable */
    double* out_mean;       /* [n][3] */
    double* out_quat;       /* [n][4] */
    double* out_scale;      /* [n][3] */
    double* out_cov3d;      /* [n][6] */
    uint32_t* out_status;   /* [n] */
} orc_outputs;

/* Run the motion fit.  tracks: [V] (disp [H][W][2] f32, vis [H][W] u8).
 * sample (nullable): only the listed Gaussians are accumulated and fitted, and
 * only tiles their rectangles touch are blended; other outputs stay untouched.
 * Returns the thread count used. */
int orc_fit_motion(int n, int V, const float* means_opacity, const float* quats,
                   const float* scales, const orc_camera* cams, const orc_tracks* tracks,
                   const orc_options* opt, const int32_t* sample, int n_sample,
                   orc_outputs* out)
{
    binctx B;
    binctx_init(&B, n, V, means_opacity, quats, scales, cams, opt->tile_w, opt->tile_h);
    const int64_t K = count_pairs(&B);
    int64_t* offsets = malloc(sizeof(int64_t) * (B.NT + 1));
    uint64_t* entries = malloc(sizeof(uint64_t) * (K > 0 ? K : 1));
    build_lists(&B, offsets, entries);

    uint8_t* want = NULL;
    uint8_t* need = NULL;
    if (sample) {
        want = calloc((size_t)n + 1, 1);
        need = calloc((size_t)B.NT + 1, 1);
        for (int i = 0; i < n_sample; ++i) want[sample[i]] = 1;
        for (int v = 0; v < V; ++v)
            for (int i = 0; i < n_sample; ++i) {
                const keyrec* k = &B.keys[(size_t)v * n + sample[i]];
                if (!k->visible) continue;
                for (int ty = k->y0; ty < k->y1; ++ty)
                    for (int tx = k->x0; tx < k->x1; ++tx)
                        need[B.toff[v] + (int64_t)ty * B.tiles_x[v] + tx] = 1;
            }
    }

    proj64* P = calloc((size_t)V * n + 1, sizeof(proj64));
    double* mom = calloc((size_t)V * n * NMOM + 1, sizeof(double));
    viewsol* sols = calloc((size_t)V * n + 1, sizeof(viewsol));
    int nthreads = 1;
#pragma omp parallel
    {
#ifdef _OPENMP
#pragma omp single
        nthreads = omp_get_num_threads();
#endif
#pragma omp for schedule(dynamic, 1)
        for (int v = 0; v < V; ++v) {
            proj64* Pv = P + (size_t)v * n;
            for (int g = 0; g < n; ++g)
                if (B.keys[(size_t)v * n + g].visible)
                    project64(means_opacity + 4 * (size_t)g, quats + 4 * (size_t)g,
                              scales + 4 * (size_t)g, &cams[v], &Pv[g]);
            blend_view(v, &B, offsets, entries, Pv, &cams[v], &tracks[v], want,
                       need ? need + B.toff[v] : NULL, mom + (size_t)v * n * NMOM, NULL, NULL, NULL);
            for (int g = 0; g < n; ++g) {
                if (want && !want[g]) continue;
                viewsol* S = &sols[(size_t)v * n + g];
                if (!B.keys[(size_t)v * n + g].visible) {
                    memset(S, 0, sizeof(*S));
                    S->flags = OV_CULLED | OV_FEW_PX | OV_LOW_ALPHA;
                    continue;
                }
                view_solve(mom + ((size_t)v * n + g) * NMOM, &Pv[g], opt, S);
            }
        }
    }
    /* outputs per (v, g) */
    for (int v = 0; v < V; ++v)
        for (int g = 0; g < n; ++g) {
            if (want && !want[g]) continue;
            const size_t i = (size_t)v * n + g;
            const proj64* G = &P[i];
            const int vis = B.keys[i].visible;
            if (out->moments) memcpy(out->moments + i * NMOM, mom + i * NMOM, sizeof(double) * NMOM);
            if (out->mean2d) { out->mean2d[2 * i] = vis ? G->mx : 0; out->mean2d[2 * i + 1] = vis ? G->my : 0; }
            if (out->cov2d) for (int k = 0; k < 3; ++k) out->cov2d[3 * i + k] = vis ? G->cov[k] : 0;
            if (out->view_flags) out->view_flags[i] = sols[i].flags;
            if (out->view_affine) {
                double* a = out->view_affine + 6 * i;
                a[0] = sols[i].A[0][0]; a[1] = sols[i].A[0][1]; a[2] = sols[i].A[1][0];
                a[3] = sols[i].A[1][1]; a[4] = sols[i].b[0]; a[5] = sols[i].b[1];
            }
            if (out->view_mean2d) { out->view_mean2d[2 * i] = sols[i].mu_new[0]; out->view_mean2d[2 * i + 1] = sols[i].mu_new[1]; }
            if (out->view_cov2d) for (int k = 0; k < 3; ++k) out->view_cov2d[3 * i + k] = sols[i].cov_new[k];
        }
    /* multi-view update per Gaussian */
#pragma omp parallel
    {
        viewsol* sv = malloc(sizeof(viewsol) * (V > 0 ? V : 1));
        const double** mv = malloc(sizeof(double*) * (V > 0 ? V : 1));
#pragma omp for schedule(dynamic, 256)
        for (int g = 0; g < n; ++g) {
            if (want && !want[g]) continue;
            for (int v = 0; v < V; ++v) {
                sv[v] = sols[(size_t)v * n + g];
                mv[v] = mom + ((size_t)v * n + g) * NMOM;
            }
            gaussout go;
            multiview_fit(V, cams, sv, mv, means_opacity + 4 * (size_t)g, quats + 4 * (size_t)g,
                          scales + 4 * (size_t)g, opt, &go);
            if (out->out_mean) for (int k = 0; k < 3; ++k) out->out_mean[3 * (size_t)g + k] = go.mean[k];
            if (out->out_quat) for (int k = 0; k < 4; ++k) out->out_quat[4 * (size_t)g + k] = go.quat[k];
            if (out->out_scale) for (int k = 0; k < 3; ++k) out->out_scale[3 * (size_t)g + k] = go.scale[k];
            if (out->out_cov3d) for (int k = 0; k < 6; ++k) out->out_cov3d[6 * (size_t)g + k] = go.cov3d[k];
            if (out->out_status) out->out_status[g] = go.status;
        }
        free(sv); free(mv);
    }
    free(P); free(mom); free(sols); free(want); free(need);
    free(offsets); free(entries);
    binctx_free(&B);
    return nthreads;
}

/* Render colour and final transmittance of every view (Sec. 3.1).
 * rgb: [V][H][W][3], T: [V][H][W], flag (nullable): [V][H][W] = 1 where a blend
 * threshold decision fell inside the FP32 window. */
int orc_render(int n, int V, const float* means_opacity, const float* quats, const float* scales,
               const float* sh, int sh_degree, const orc_camera* cams, int tile_w, int tile_h,
               float* const* rgb, float* const* Tout, uint8_t* const* flag)
{
    binctx B;
    binctx_init(&B, n, V, means_opacity, quats, scales, cams, tile_w, tile_h);
    const int64_t K = count_pairs(&B);
    int64_t* offsets = malloc(sizeof(int64_t) * (B.NT + 1));
    uint64_t* entries = malloc(sizeof(uint64_t) * (K > 0 ? K : 1));
    build_lists(&B, offsets, entries);
    const int nb = (sh_degree + 1) * (sh_degree + 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int v = 0; v < V; ++v) {
        proj64* Pv = calloc((size_t)n + 1, sizeof(proj64));
        for (int g = 0; g < n; ++g)
            if (B.keys[(size_t)v * n + g].visible) {
                project64(means_opacity + 4 * (size_t)g, quats + 4 * (size_t)g,
                          scales + 4 * (size_t)g, &cams[v], &Pv[g]);
                sh_color(means_opacity + 4 * (size_t)g, sh + (size_t)g * nb * 3, sh_degree, &cams[v],
                         Pv[g].color);
            }
        blend_view(v, &B, offsets, entries, Pv, &cams[v], NULL, NULL, NULL, NULL, rgb[v], Tout[v],
                   flag ? flag[v] : NULL);
        free(Pv);
    }
    free(offsets); free(entries);
    binctx_free(&B);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Render gradient (the adjoint of the blend, for gradient refinement)         */
/* ------------------------------------------------------------------------- */
/* For L = sum over views, pixels and channels of W[v][p][ch] * C[v][p][ch], C the
 * colour orc_render gives, the gradient with respect to every Gaussian's mean,
 * linear scales, raw (unnormalised) quaternion, opacity and colour coefficients.
 * The chain rule runs through the blend of Sec. 3.1 (C = sum c_i alpha_i T_i with
 * its decisions -- tile rectangle, alpha >= 1/255, the transmittance cut-off,
 * the clamps of alpha at 0.99 and of the colour at 0 -- held fixed), the inverse
 * of the dilated Sigma_2D, Sigma_2D = (J W) Sigma_3D (J W)^T and the perspective
 * map (Eq. 1), Sigma_3D = R(q) diag(s^2) R(q)^T, and the colour basis along the
 * direction from the camera centre.  Written from those definitions; no step of
 * it is shared with the GPU code. */

typedef struct {
    proj64 P;
    double p[3];          /* camera-space mean */
    double T[2][3];       /* J W */
    double S[3][3];       /* Sigma_3D */
    double R[3][3];       /* R(q) */
    double qn[4], qnorm;
    double dir[3], dist;  /* unit direction camera centre -> mean, distance */
    double Y[16];
    double raw[3];        /* colour before the clamp at 0 */
} vgauss;

static void vgauss_make(const float* mo, const float* q, const float* s, const float* sh, int deg,
                        const orc_camera* c, vgauss* G)
{
    project64(mo, q, s, c, &G->P);
    const double X[3] = {mo[0], mo[1], mo[2]};
    jw_at(c, X, G->T, G->p);
    cov3d(q, s, G->S);
    quat_to_rot(q, G->R, G->qn);
    G->qnorm = sqrt((double)q[0] * q[0] + (double)q[1] * q[1] + (double)q[2] * q[2] + (double)q[3] * q[3]);
    double Cc[3];
    for (int i = 0; i < 3; ++i)
        Cc[i] = -(c->R[i] * (double)c->t[0] + c->R[3 + i] * (double)c->t[1] + c->R[6 + i] * (double)c->t[2]);
    double d[3] = {X[0] - Cc[0], X[1] - Cc[1], X[2] - Cc[2]};
    G->dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int i = 0; i < 3; ++i) G->dir[i] = d[i] / G->dist;
    sh_basis(G->dir[0], G->dir[1], G->dir[2], G->Y);
    const int nb = (deg + 1) * (deg + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.5;
        for (int k = 0; k < nb; ++k) acc += G->Y[k] * sh[k * 3 + ch];
        G->raw[ch] = acc;
        G->P.color[ch] = acc > 0 ? acc : 0;
    }
}

/* Gradient of each basis function with respect to (x, y, z), the functions read
 * as polynomials (their restriction to the unit sphere is the basis). */
static void sh_basis_grad(double x, double y, double z, double dY[16][3])
{
    const double pi = 3.14159265358979323846;
    const double k1 = sqrt(3.0 / (4.0 * pi));
    const double k2a = 0.5 * sqrt(15.0 / pi), k2b = 0.25 * sqrt(5.0 / pi), k2c = 0.25 * sqrt(15.0 / pi);
    const double k3a = 0.25 * sqrt(35.0 / (2.0 * pi)), k3b = 0.5 * sqrt(105.0 / pi);
    const double k3c = 0.25 * sqrt(21.0 / (2.0 * pi)), k3d = 0.25 * sqrt(7.0 / pi);
    const double k3e = 0.25 * sqrt(105.0 / pi);
    const double xx = x * x, yy = y * y, zz = z * z;
    const double g[16][3] = {
        {0, 0, 0},
        {0, -k1, 0}, {0, 0, k1}, {-k1, 0, 0},
        {k2a * y, k2a * x, 0}, {0, -k2a * z, -k2a * y}, {-2 * k2b * x, -2 * k2b * y, 4 * k2b * z},
        {-k2a * z, 0, -k2a * x}, {2 * k2c * x, -2 * k2c * y, 0},
        {-6 * k3a * x * y, -3 * k3a * (xx - yy), 0},
        {k3b * y * z, k3b * x * z, k3b * x * y},
        {2 * k3c * x * y, -k3c * (4 * zz - xx - 3 * yy), -8 * k3c * y * z},
        {-6 * k3d * x * z, -6 * k3d * y * z, k3d * (6 * zz - 3 * xx - 3 * yy)},
        {-k3c * (4 * zz - 3 * xx - yy), 2 * k3c * x * y, -8 * k3c * x * z},
        {2 * k3e * x * z, -2 * k3e * y * z, k3e * (xx - yy)},
        {-3 * k3a * (xx - yy), 6 * k3a * x * y, 0}};
    memcpy(dY, g, sizeof(g));
}

typedef struct { int g; double a, T, G; int clamped; double dx, dy; } contrib;

/* One view: the loss (optional) and, with gp != NULL, the gradient with respect
 * to each Gaussian's 2D quantities: gp[g] = (mu_x, mu_y, conic 00, conic 01 (the
 * off-diagonal parameter), conic 11, opacity, colour r, g, b). */
static void grad_view(int v, const binctx* B, const int64_t* offsets, const uint64_t* entries,
                      const vgauss* VG, const orc_camera* cam, const float* W, double* loss, double* gp)
{
    const int tw = B->tw, th = B->th, Wd = cam->width, H = cam->height;
    int64_t cap = 256;
    contrib* cs = malloc(sizeof(contrib) * cap);
    double L = 0.0;
    for (int ty = 0; ty < B->tiles_y[v]; ++ty)
        for (int tx = 0; tx < B->tiles_x[v]; ++tx) {
            const int64_t t = B->toff[v] + (int64_t)ty * B->tiles_x[v] + tx;
            const int64_t e0 = offsets[t], e1 = offsets[t + 1];
            if (e1 - e0 > cap) { cap = e1 - e0; cs = realloc(cs, sizeof(contrib) * cap); }
            for (int py = ty * th; py < (ty + 1) * th && py < H; ++py)
                for (int px = tx * tw; px < (tx + 1) * tw && px < Wd; ++px) {
                    const double xc = px + 0.5, yc = py + 0.5;
                    double T = 1.0, C[3] = {0, 0, 0};
                    int m = 0;
                    for (int64_t e = e0; e < e1; ++e) {
                        const int g = (int)(uint32_t)entries[e];
                        const proj64* G = &VG[g].P;
                        const double dx = xc - G->mx, dy = yc - G->my;
                        const double qf = G->conic[0] * dx * dx + 2.0 * G->conic[1] * dx * dy
                                        + G->conic[2] * dy * dy;
                        const double Gv = exp(-0.5 * qf);
                        double a = G->opacity * Gv;
                        const int clamped = a > ALPHA_MAX;
                        if (clamped) a = ALPHA_MAX;
                        if (a < ALPHA_MIN) continue;
                        const double Tn = T * (1.0 - a);
                        if (Tn < T_MIN) break;
                        for (int ch = 0; ch < 3; ++ch) C[ch] += a * T * G->color[ch];
                        cs[m++] = (contrib){g, a, T, Gv, clamped, dx, dy};
                        T = Tn;
                    }
                    const float* w = W + 3 * ((size_t)py * Wd + px);
                    L += w[0] * C[0] + w[1] * C[1] + w[2] * C[2];
                    if (!gp) continue;
                    double P[3] = {0, 0, 0};
                    for (int i = 0; i < m; ++i) {
                        const contrib* k = &cs[i];
                        const proj64* G = &VG[k->g].P;
                        double ga = 0.0;
                        for (int ch = 0; ch < 3; ++ch) {
                            P[ch] += k->a * k->T * G->color[ch];
                            /* dC/dalpha_i = c_i T_i - (C - P_i) / (1 - alpha_i) */
                            ga += w[ch] * (G->color[ch] * k->T - (C[ch] - P[ch]) / (1.0 - k->a));
                        }
                        double* o = gp + 9 * (size_t)k->g;
                        for (int ch = 0; ch < 3; ++ch) o[6 + ch] += k->a * k->T * w[ch];
                        if (k->clamped) continue;
                        o[5] += k->G * ga;                                   /* alpha = o G */
                        const double gG = G->opacity * ga;
                        /* G = exp(-d^T Q d / 2), d = x - mu: dG/dmu = G Q d */
                        o[0] += gG * k->G * (G->conic[0] * k->dx + G->conic[1] * k->dy);
                        o[1] += gG * k->G * (G->conic[1] * k->dx + G->conic[2] * k->dy);
                        o[2] += gG * (-0.5 * k->G * k->dx * k->dx);
                        o[3] += gG * (-k->G * k->dx * k->dy);
                        o[4] += gG * (-0.5 * k->G * k->dy * k->dy);
                    }
                }
        }
    free(cs);
    if (loss) *loss = L;
}

/* The 2D gradient gp (grad_view's layout) of Gaussian G in camera c, carried back
 * to the 3D parameters and added to gm[3], gs[3], gq[4], *go, gsh[nb][3]. */
static void chain_view(const vgauss* G, const double* gp, const orc_camera* c, const float* sh, int deg,
                       const float* s_lin, double* gm, double* gs, double* gq, double* go, double* gsh)
{
    /* conic = inverse of the dilated Sigma_2D [[a, b], [b, d]] */
    const double a = G->P.cov[0] + DILATION, b = G->P.cov[1], d = G->P.cov[2] + DILATION;
    const double det = a * d - b * b, i2 = 1.0 / (det * det);
    const double q00 = gp[2], q01 = gp[3], q11 = gp[4];
    const double ga = q00 * (-d * d * i2) + q01 * (b * d * i2) + q11 * (1.0 / det - a * d * i2);
    const double gd = q00 * (1.0 / det - a * d * i2) + q01 * (a * b * i2) + q11 * (-a * a * i2);
    const double gb = q00 * (2.0 * b * d * i2) + q01 * (-1.0 / det - 2.0 * b * b * i2) + q11 * (2.0 * a * b * i2);
    const double G2[2][2] = {{ga, 0.5 * gb}, {0.5 * gb, gd}};   /* dL/dSigma_2D, symmetric */
    /* Sigma_2D = T S T^T */
    double gS[3][3], gT[2][3], TS[2][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int u = 0; u < 2; ++u)
                for (int w = 0; w < 2; ++w) acc += G->T[u][i] * G2[u][w] * G->T[w][j];
            gS[i][j] = acc;
        }
    for (int u = 0; u < 2; ++u)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += G->T[u][k] * G->S[k][j];
            TS[u][j] = acc;
        }
    for (int u = 0; u < 2; ++u)
        for (int j = 0; j < 3; ++j) gT[u][j] = 2.0 * (G2[u][0] * TS[0][j] + G2[u][1] * TS[1][j]);
    /* T = J W with W the camera rotation (row-major R) */
    double gJ[2][3];
    for (int u = 0; u < 2; ++u)
        for (int k = 0; k < 3; ++k)
            gJ[u][k] = gT[u][0] * c->R[3 * k] + gT[u][1] * c->R[3 * k + 1] + gT[u][2] * c->R[3 * k + 2];
    const double px = G->p[0], py = G->p[1], pz = G->p[2], fx = c->fx, fy = c->fy;
    const double iz = 1.0 / pz, iz2 = iz * iz, iz3 = iz2 * iz;
    double gpc[3];
    gpc[0] = gJ[0][2] * (-fx * iz2) + gp[0] * fx * iz;
    gpc[1] = gJ[1][2] * (-fy * iz2) + gp[1] * fy * iz;
    gpc[2] = gJ[0][0] * (-fx * iz2) + gJ[0][2] * (2.0 * fx * px * iz3) + gJ[1][1] * (-fy * iz2)
           + gJ[1][2] * (2.0 * fy * py * iz3) - gp[0] * fx * px * iz2 - gp[1] * fy * py * iz2;
    for (int j = 0; j < 3; ++j) gm[j] += c->R[j] * gpc[0] + c->R[3 + j] * gpc[1] + c->R[6 + j] * gpc[2];
    /* colour: c = max(0, 0.5 + sum_k Y_k(dir) sh_k) */
    const int nb = (deg + 1) * (deg + 1);
    double gY[16] = {0};
    for (int ch = 0; ch < 3; ++ch) {
        if (!(G->raw[ch] > 0)) continue;
        for (int k = 0; k < nb; ++k) {
            gsh[3 * k + ch] += G->Y[k] * gp[6 + ch];
            gY[k] += sh[3 * k + ch] * gp[6 + ch];
        }
    }
    double dY[16][3], gdir[3] = {0, 0, 0};
    sh_basis_grad(G->dir[0], G->dir[1], G->dir[2], dY);
    for (int k = 0; k < nb; ++k)
        for (int i = 0; i < 3; ++i) gdir[i] += gY[k] * dY[k][i];
    const double dd = G->dir[0] * gdir[0] + G->dir[1] * gdir[1] + G->dir[2] * gdir[2];
    for (int i = 0; i < 3; ++i) gm[i] += (gdir[i] - G->dir[i] * dd) / G->dist;
    *go += gp[5];
    /* Sigma_3D = R D R^T, D = diag(s^2) */
    const double s2[3] = {(double)s_lin[0] * s_lin[0], (double)s_lin[1] * s_lin[1], (double)s_lin[2] * s_lin[2]};
    for (int k = 0; k < 3; ++k) {
        double acc = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) acc += G->R[i][k] * gS[i][j] * G->R[j][k];
        gs[k] += 2.0 * s_lin[k] * acc;
    }
    double gR[3][3];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int j = 0; j < 3; ++j) acc += gS[i][j] * G->R[j][k];
            gR[i][k] = 2.0 * acc * s2[k];
        }
    const double w = G->qn[0], x = G->qn[1], y = G->qn[2], z = G->qn[3];
    const double dRw[3][3] = {{0, -2 * z, 2 * y}, {2 * z, 0, -2 * x}, {-2 * y, 2 * x, 0}};
    const double dRx[3][3] = {{0, 2 * y, 2 * z}, {2 * y, -4 * x, -2 * w}, {2 * z, 2 * w, -4 * x}};
    const double dRy[3][3] = {{-4 * y, 2 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, 2 * z, -4 * y}};
    const double dRz[3][3] = {{-4 * z, -2 * w, 2 * x}, {2 * w, -4 * z, 2 * y}, {2 * x, 2 * y, 0}};
    double gh[4] = {0, 0, 0, 0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            gh[0] += gR[i][j] * dRw[i][j]; gh[1] += gR[i][j] * dRx[i][j];
            gh[2] += gR[i][j] * dRy[i][j]; gh[3] += gR[i][j] * dRz[i][j];
        }
    const double hq = gh[0] * w + gh[1] * x + gh[2] * y + gh[3] * z;
    gq[0] += (gh[0] - w * hq) / G->qnorm;
    gq[1] += (gh[1] - x * hq) / G->qnorm;
    gq[2] += (gh[2] - y * hq) / G->qnorm;
    gq[3] += (gh[3] - z * hq) / G->qnorm;
}

int orc_render_grad(int n, int V, const float* means_opacity, const float* quats, const float* scales,
                    const float* sh, int sh_degree, const orc_camera* cams, int tile_w, int tile_h,
                    const float* const* W, double* loss, double* g_means, double* g_scales, double* g_quats,
                    double* g_opacity, double* g_sh)
{
    binctx B;
    binctx_init(&B, n, V, means_opacity, quats, scales, cams, tile_w, tile_h);
    const int64_t K = count_pairs(&B);
    int64_t* offsets = malloc(sizeof(int64_t) * (B.NT + 1));
    uint64_t* entries = malloc(sizeof(uint64_t) * (K > 0 ? K : 1));
    build_lists(&B, offsets, entries);
    const int nb = (sh_degree + 1) * (sh_degree + 1);
    const int want = g_means != NULL;
    const size_t per = (size_t)n * (3 + 3 + 4 + 1 + 3 * nb);
    double* acc = want ? calloc((size_t)V * per + 1, sizeof(double)) : NULL;
    double* lv = calloc((size_t)V + 1, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int v = 0; v < V; ++v) {
        vgauss* VG = calloc((size_t)n + 1, sizeof(vgauss));
        for (int g = 0; g < n; ++g)
            if (B.keys[(size_t)v * n + g].visible)
                vgauss_make(means_opacity + 4 * (size_t)g, quats + 4 * (size_t)g, scales + 4 * (size_t)g,
                            sh + (size_t)g * nb * 3, sh_degree, &cams[v], &VG[g]);
        double* gp = want ? calloc((size_t)n * 9 + 1, sizeof(double)) : NULL;
        grad_view(v, &B, offsets, entries, VG, &cams[v], W[v], &lv[v], gp);
        if (want) {
            double* a = acc + (size_t)v * per;
            for (int g = 0; g < n; ++g) {
                if (!B.keys[(size_t)v * n + g].visible) continue;
                double* base = a + (size_t)g * (11 + 3 * nb);
                chain_view(&VG[g], gp + 9 * (size_t)g, &cams[v], sh + (size_t)g * nb * 3, sh_degree,
                           scales + 4 * (size_t)g, base, base + 3, base + 6, base + 10, base + 11);
            }
            free(gp);
        }
        free(VG);
    }
    double L = 0;
    for (int v = 0; v < V; ++v) L += lv[v];
    if (loss) *loss = L;
    if (want) {
        for (int g = 0; g < n; ++g) {
            double* om = g_means + 3 * (size_t)g; double* os = g_scales + 3 * (size_t)g;
            double* oq = g_quats + 4 * (size_t)g; double* osh = g_sh + (size_t)g * nb * 3;
            for (int i = 0; i < 3; ++i) { om[i] = 0; os[i] = 0; }
            for (int i = 0; i < 4; ++i) oq[i] = 0;
            g_opacity[g] = 0;
            for (int i = 0; i < 3 * nb; ++i) osh[i] = 0;
            for (int v = 0; v < V; ++v) {
                const double* b = acc + (size_t)v * per + (size_t)g * (11 + 3 * nb);
                for (int i = 0; i < 3; ++i) { om[i] += b[i]; os[i] += b[3 + i]; }
                for (int i = 0; i < 4; ++i) oq[i] += b[6 + i];
                g_opacity[g] += b[10];
                for (int i = 0; i < 3 * nb; ++i) osh[i] += b[11 + i];
            }
        }
        free(acc);
    }
    free(lv);
    free(offsets); free(entries);
    binctx_free(&B);
    return 0;
}

/* Brute-force render of one view: every Gaussian that passes the key path is
 * blended at every pixel, in (depth bits, index) order, with no tiles.  With
 * use_rect != 0 a Gaussian only reaches pixels inside its tile rectangle, which
 * makes the result equal to the tiled render. */
int orc_render_bruteforce(int n, const float* means_opacity, const float* quats, const float* scales,
                          const float* sh, int sh_degree, const orc_camera* cam, int tile_w, int tile_h,
                          int use_rect, float* rgb, float* Tout)
{
    binctx B;
    binctx_init(&B, n, 1, means_opacity, quats, scales, cam, tile_w, tile_h);
    uint64_t* order = malloc(sizeof(uint64_t) * ((size_t)n + 1));
    int m = 0;
    for (int g = 0; g < n; ++g)
        if (B.keys[g].visible) order[m++] = ((uint64_t)B.keys[g].depth_bits << 32) | (uint32_t)g;
    qsort(order, (size_t)m, sizeof(uint64_t), cmp_u64);
    const int nb = (sh_degree + 1) * (sh_degree + 1);
    proj64* P = calloc((size_t)n + 1, sizeof(proj64));
    for (int i = 0; i < m; ++i) {
        const int g = (int)(uint32_t)order[i];
        project64(means_opacity + 4 * (size_t)g, quats + 4 * (size_t)g, scales + 4 * (size_t)g, cam, &P[g]);
        sh_color(means_opacity + 4 * (size_t)g, sh + (size_t)g * nb * 3, sh_degree, cam, P[g].color);
    }
    const int W = cam->width, H = cam->height;
#pragma omp parallel for schedule(dynamic, 4)
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            const int tx = px / tile_w, ty = py / tile_h;
            double T = 1.0, col[3] = {0, 0, 0};
            for (int i = 0; i < m; ++i) {
                const int g = (int)(uint32_t)order[i];
                if (use_rect) {
                    const keyrec* k = &B.keys[g];
                    if (tx < k->x0 || tx >= k->x1 || ty < k->y0 || ty >= k->y1) continue;
                }
                const proj64* G = &P[g];
                const double dx = px + 0.5 - G->mx, dy = py + 0.5 - G->my;
                const double qf = G->conic[0] * dx * dx + 2.0 * G->conic[1] * dx * dy + G->conic[2] * dy * dy;
                double alpha = G->opacity * exp(-0.5 * qf);
                if (alpha > ALPHA_MAX) alpha = ALPHA_MAX;
                if (alpha < ALPHA_MIN) continue;
                const double Tn = T * (1.0 - alpha);
                if (Tn < T_MIN) break;
                for (int ch = 0; ch < 3; ++ch) col[ch] += alpha * T * G->color[ch];
                T = Tn;
            }
            const size_t pix = (size_t)py * W + px;
            for (int ch = 0; ch < 3; ++ch) rgb[3 * pix + ch] = (float)col[ch];
            Tout[pix] = (float)T;
        }
    free(order); free(P);
    binctx_free(&B);
    return 0;
}

/* Eq. 3 directly: stack X = [x^T 1] (n x 3) and Y = x'^T (n x 2), weight rows by
 * sqrt(w) and solve the least-squares problem by Householder QR.
 * out: A00 A01 A10 A11 b0 b1.  Returns 0 if R is singular. */
int orc_naive_ls(int n, const double* x /* [n][2] */, const double* xp /* [n][2] */,
                 const double* w /* [n] or NULL */, double* out)
{
    double* A = malloc(sizeof(double) * 3 * n);   /* column-major n x 3 */
    double* Y = malloc(sizeof(double) * 2 * n);   /* column-major n x 2 */
    for (int i = 0; i < n; ++i) {
        const double s = w ? sqrt(w[i]) : 1.0;
        A[0 * n + i] = s * x[2 * i]; A[1 * n + i] = s * x[2 * i + 1]; A[2 * n + i] = s;
        Y[0 * n + i] = s * xp[2 * i]; Y[1 * n + i] = s * xp[2 * i + 1];
    }
    double Rm[3][3] = {{0}};
    for (int k = 0; k < 3; ++k) {
        double nrm = 0;
        for (int i = k; i < n; ++i) nrm += A[k * n + i] * A[k * n + i];
        nrm = sqrt(nrm);
        if (nrm == 0.0) { free(A); free(Y); return 0; }
        const double alpha = A[k * n + k] > 0 ? -nrm : nrm;
        /* v = a_k - alpha e_k, H = I - 2 v v^T / v^T v */
        A[k * n + k] -= alpha;
        double vtv = 0;
        for (int i = k; i < n; ++i) vtv += A[k * n + i] * A[k * n + i];
        for (int j = k + 1; j < 3; ++j) {
            double d = 0;
            for (int i = k; i < n; ++i) d += A[k * n + i] * A[j * n + i];
            const double f = 2.0 * d / vtv;
            for (int i = k; i < n; ++i) A[j * n + i] -= f * A[k * n + i];
        }
        for (int j = 0; j < 2; ++j) {
            double d = 0;
            for (int i = k; i < n; ++i) d += A[k * n + i] * Y[j * n + i];
            const double f = 2.0 * d / vtv;
            for (int i = k; i < n; ++i) Y[j * n + i] -= f * A[k * n + i];
        }
        Rm[k][k] = alpha;
        for (int j = k + 1; j < 3; ++j) Rm[k][j] = A[j * n + k];
    }
    double Z[3][2];
    for (int j = 0; j < 2; ++j)
        for (int k = 2; k >= 0; --k) {
            double acc = Y[j * n + k];
            for (int i = k + 1; i < 3; ++i) acc -= Rm[k][i] * Z[i][j];
            Z[k][j] = acc / Rm[k][k];
        }
    out[0] = Z[0][0]; out[1] = Z[1][0]; out[2] = Z[0][1]; out[3] = Z[1][1];
    out[4] = Z[2][0]; out[5] = Z[2][1];
    free(A); free(Y);
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Building blocks exposed for the pins                                      */
/* ------------------------------------------------------------------------- */

int orc_project(const float* mo, const float* q, const float* s, const orc_camera* cam,
                double* mean2d, double* cov2d, double* conic)
{
    proj64 P;
    project64(mo, q, s, cam, &P);
    mean2d[0] = P.mx; mean2d[1] = P.my;
    for (int k = 0; k < 3; ++k) { cov2d[k] = P.cov[k]; conic[k] = P.conic[k]; }
    return 0;
}

int orc_eig3(const double* S /* [9] */, double* lam, double* E /* [9] row-major */)
{
    double A[3][3], Em[3][3];
    memcpy(A, S, sizeof(A));
    jacobi_eig3(A, lam, Em);
    memcpy(E, Em, sizeof(Em));
    return 0;
}

/* min ||A x - b||, A row-major m x n (n <= 8). Returns sigma_min / sigma_max. */
double orc_lstsq(int m, int n, const double* A, const double* b, double* x)
{
    double* Ac = malloc(sizeof(double) * m * n);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) Ac[j * m + i] = A[i * n + j];
    const double rc = svd_lstsq(Ac, m, n, b, x);
    free(Ac);
    return rc;
}

/* Per-view solve on a given moment record (layout of NMOM). */
int orc_view_solve(const double* mom, const double* mean2d, const double* cov2d,
                   const orc_options* opt, uint32_t* flags, double* affine, double* mean2d_new,
                   double* cov2d_new)
{
    proj64 G;
    memset(&G, 0, sizeof(G));
    G.mx = mean2d[0]; G.my = mean2d[1];
    for (int k = 0; k < 3; ++k) G.cov[k] = cov2d[k];
    viewsol S;
    view_solve(mom, &G, opt, &S);
    *flags = S.flags;
    affine[0] = S.A[0][0]; affine[1] = S.A[0][1]; affine[2] = S.A[1][0]; affine[3] = S.A[1][1];
    affine[4] = S.b[0]; affine[5] = S.b[1];
    mean2d_new[0] = S.mu_new[0]; mean2d_new[1] = S.mu_new[1];
    for (int k = 0; k < 3; ++k) cov2d_new[k] = S.cov_new[k];
    return 0;
}

/* Multi-view update of one Gaussian from given per-view results.
 * flags[V], sumw[V], npix[V], mean2d_new[V][2], cov2d_new[V][3];
 * out: mean[3], quat[4], scale[3], cov3d[6], status. */
int orc_multiview(int V, const orc_camera* cams, const uint32_t* flags, const double* sumw,
                  const double* npix, const double* mean2d_new, const double* cov2d_new,
                  const float* mo, const float* q, const float* s, const orc_options* opt,
                  double* mean, double* quat, double* scale, double* cov3d, uint32_t* status)
{
    viewsol* sv = calloc((size_t)(V > 0 ? V : 1), sizeof(viewsol));
    double* mrec = calloc((size_t)(V > 0 ? V : 1) * NMOM, sizeof(double));
    const double** mv = malloc(sizeof(double*) * (V > 0 ? V : 1));
    for (int v = 0; v < V; ++v) {
        sv[v].flags = flags[v];
        sv[v].mu_new[0] = mean2d_new[2 * v]; sv[v].mu_new[1] = mean2d_new[2 * v + 1];
        for (int k = 0; k < 3; ++k) sv[v].cov_new[k] = cov2d_new[3 * v + k];
        mrec[v * NMOM + 5] = sumw[v];
        mrec[v * NMOM + 13] = npix[v];
        mv[v] = mrec + v * NMOM;
    }
    gaussout go;
    multiview_fit(V, cams, sv, mv, mo, q, s, opt, &go);
    for (int k = 0; k < 3; ++k) { mean[k] = go.mean[k]; scale[k] = go.scale[k]; }
    for (int k = 0; k < 4; ++k) quat[k] = go.quat[k];
    for (int k = 0; k < 6; ++k) cov3d[k] = go.cov3d[k];
    *status = go.status;
    free(sv); free(mrec); free(mv);
    return 0;
}

/* Colour basis: Y[16] at the unit direction (x, y, z). */
int orc_sh_basis(double x, double y, double z, double* Y)
{
    sh_basis(x, y, z, Y);
    return 0;
}

/* Threads the parallel regions use from now on (timing only: a single-thread
 * time of the oracle); n <= 0 restores the default. */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    static int dflt = 0;
    if (!dflt) dflt = omp_get_max_threads();
    omp_set_num_threads(n > 0 ? n : dflt);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Motion regularization (Sec. 4.5)                                            */
/* ------------------------------------------------------------------------- */
/* Readings (the text leaves them open):
 *  - a Gaussian's motion components are its position change dmu = mu' - mu
 *    (available when its position was solved) and, when its covariance was
 *    solved, its scale change ds = s' - s (linear scales) and rotation change
 *    dR = R' R^T as Euler angles (x, y, z) with dR = Rz(ez) Ry(ey) Rx(ex);
 *  - static (Sec. 4.5.2): hit by more than min_px pixels with more than frac of
 *    them static in at least min_views views; its motion is discarded;
 *  - median filtering (Sec. 4.5.1): a Gaussian with a component gets, per
 *    coordinate, the median over itself and its K nearest other Gaussians with
 *    that component (static ones excluded);
 *  - propagation (Sec. 4.5.2), after the filtering: a non-static Gaussian
 *    without a component gets the mean of the filtered component over its K
 *    nearest Gaussians with it;
 *  - nearness: squared distance between first-frame means, in FP32 as
 *    ((dx*dx + dy*dy) + dz*dz) with dx = x_q - x_p (the same decisions as the
 *    FP32 implementation), ties by index.
 * The new parameters are mu + dmu, s + ds, R(e) R (quaternion sign kept close
 * to the old one). */

#define REG_STATIC 1u
#define REG_POS_MEDIAN 2u
#define REG_POS_PROPAGATED 4u
#define REG_COV_MEDIAN 8u
#define REG_COV_PROPAGATED 16u

static float dist2_f32(const float* a, const float* b)
{
    const float dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    const float xx = dx * dx, yy = dy * dy, zz = dz * dz;
    const float s = xx + yy;
    return s + zz;
}

/* The k nearest members of `mask` other than q (by (d2, index)); returns their count. */
static int knn_brute(int n, const float* mo, const uint8_t* mask, int q, int k, int* out)
{
    float bd[64];
    int bi[64], m = 0;
    for (int p = 0; p < n; ++p) {
        if (p == q || !mask[p]) continue;
        const float d = dist2_f32(mo + 4 * (size_t)q, mo + 4 * (size_t)p);
        if (m == k && !(d < bd[k - 1] || (d == bd[k - 1] && p < bi[k - 1]))) continue;
        int j = m < k ? m++ : k - 1;
        while (j > 0 && (d < bd[j - 1] || (d == bd[j - 1] && p < bi[j - 1]))) {
            bd[j] = bd[j - 1]; bi[j] = bi[j - 1]; --j;
        }
        bd[j] = d; bi[j] = p;
    }
    for (int j = 0; j < m; ++j) out[j] = bi[j];
    return m;
}

static int cmp_double(const void* a, const void* b)
{
    const double x = *(const double*)a, y = *(const double*)b;
    return x < y ? -1 : x > y;
}

static double median_of(double* v, int m)
{
    qsort(v, (size_t)m, sizeof(double), cmp_double);
    return (m & 1) ? v[m / 2] : 0.5 * (v[m / 2 - 1] + v[m / 2]);
}

static void rot_of_quat(const float* q, double R[3][3])
{
    double qn[4];
    quat_to_rot(q, R, qn);
}

static void euler_of(const double R[3][3], double e[3])
{
    /* R = Rz(c) Ry(b) Rx(a): R20 = -sin b, R21 = cos b sin a, R22 = cos b cos a,
     * R10 = sin c cos b, R00 = cos c cos b */
    double sb = -R[2][0];
    if (sb > 1) sb = 1;
    if (sb < -1) sb = -1;
    e[1] = asin(sb);
    e[0] = atan2(R[2][1], R[2][2]);
    e[2] = atan2(R[1][0], R[0][0]);
}

static void rot_of_euler(const double e[3], double R[3][3])
{
    const double ca = cos(e[0]), sa = sin(e[0]), cb = cos(e[1]), sb = sin(e[1]), cc = cos(e[2]), sc = sin(e[2]);
    R[0][0] = cc * cb; R[0][1] = cc * sb * sa - sc * ca; R[0][2] = cc * sb * ca + sc * sa;
    R[1][0] = sc * cb; R[1][1] = sc * sb * sa + cc * ca; R[1][2] = sc * sb * ca - cc * sa;
    R[2][0] = -sb;     R[2][1] = cb * sa;                R[2][2] = cb * ca;
}

static void quat_of_rot(const double R[3][3], double q[4])
{
    /* the largest of 1 + tr and 1 + 2 R_kk - tr picks the stable branch */
    const double tr = R[0][0] + R[1][1] + R[2][2];
    if (tr >= R[0][0] && tr >= R[1][1] && tr >= R[2][2]) {
        const double h = 2.0 * sqrt(1.0 + tr);
        q[0] = 0.25 * h; q[1] = (R[2][1] - R[1][2]) / h; q[2] = (R[0][2] - R[2][0]) / h; q[3] = (R[1][0] - R[0][1]) / h;
    } else if (R[0][0] >= R[1][1] && R[0][0] >= R[2][2]) {
        const double h = 2.0 * sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]);
        q[0] = (R[2][1] - R[1][2]) / h; q[1] = 0.25 * h; q[2] = (R[0][1] + R[1][0]) / h; q[3] = (R[0][2] + R[2][0]) / h;
    } else if (R[1][1] >= R[2][2]) {
        const double h = 2.0 * sqrt(1.0 - R[0][0] + R[1][1] - R[2][2]);
        q[0] = (R[0][2] - R[2][0]) / h; q[1] = (R[0][1] + R[1][0]) / h; q[2] = 0.25 * h; q[3] = (R[1][2] + R[2][1]) / h;
    } else {
        const double h = 2.0 * sqrt(1.0 - R[0][0] - R[1][1] + R[2][2]);
        q[0] = (R[1][0] - R[0][1]) / h; q[1] = (R[0][2] + R[2][0]) / h; q[2] = (R[1][2] + R[2][1]) / h; q[3] = 0.25 * h;
    }
}

/* Static test of Sec. 4.5.2 from per-view counts npix[V][n], nstat[V][n], in
 * FP32 (nstat > frac * npix) as the FP32 implementation takes it. */
int orc_static_flags(int n, int V, const float* npix, const float* nstat, float min_px, float frac, int min_views,
                     uint8_t* is_static)
{
    for (int g = 0; g < n; ++g) {
        int views = 0;
        for (int v = 0; v < V; ++v) {
            const float np = npix[(size_t)v * n + g], ns = nstat[(size_t)v * n + g];
            if (np > min_px && ns > frac * np) ++views;
        }
        is_static[g] = views >= min_views;
    }
    return 0;
}

int orc_knn(int n, const float* means_opacity, const uint8_t* mask, int k, int* nbr /* [n][k], -1 pad */)
{
    if (k > 64) return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int q = 0; q < n; ++q) {
        int out[64];
        const int m = knn_brute(n, means_opacity, mask, q, k, out);
        for (int j = 0; j < k; ++j) nbr[(size_t)q * k + j] = j < m ? out[j] : -1;
    }
    return 0;
}

int orc_regularize(int n, const float* mo0, const float* q0, const float* s0, const float* mo1, const float* q1,
                   const float* s1, const uint32_t* status, const uint8_t* is_static, int k,
                   float* mo_out, float* q_out, float* s_out, uint32_t* flags)
{
    if (k > 64) return -1;
    uint8_t* has_pos = calloc((size_t)n + 1, 1);
    uint8_t* has_cov = calloc((size_t)n + 1, 1);
    double* dpos = calloc((size_t)n * 3 + 1, sizeof(double));
    double* dcov = calloc((size_t)n * 6 + 1, sizeof(double));    /* ds (3), rotation Euler angles (3) */
    for (int g = 0; g < n; ++g) {
        has_pos[g] = !is_static[g] && (status[g] & OS_POS_OK);
        has_cov[g] = !is_static[g] && (status[g] & OS_COV_OK);
        for (int i = 0; i < 3; ++i) dpos[3 * g + i] = (double)mo1[4 * g + i] - (double)mo0[4 * g + i];
        double Ra[3][3], Rb[3][3], D[3][3];
        rot_of_quat(q0 + 4 * (size_t)g, Ra);
        rot_of_quat(q1 + 4 * (size_t)g, Rb);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) D[i][j] = Rb[i][0] * Ra[j][0] + Rb[i][1] * Ra[j][1] + Rb[i][2] * Ra[j][2];
        for (int i = 0; i < 3; ++i) dcov[6 * g + i] = (double)s1[4 * g + i] - (double)s0[4 * g + i];
        euler_of(D, dcov + 6 * (size_t)g + 3);
    }
    int* np = malloc(sizeof(int) * ((size_t)n * k + 1));
    int* nc = malloc(sizeof(int) * ((size_t)n * k + 1));
    orc_knn(n, mo0, has_pos, k, np);
    orc_knn(n, mo0, has_cov, k, nc);
    /* pass 1: median filter of every Gaussian that has the component */
    double* fpos = calloc((size_t)n * 3 + 1, sizeof(double));
    double* fcov = calloc((size_t)n * 6 + 1, sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
    for (int g = 0; g < n; ++g) {
        double vals[65];
        for (int part = 0; part < 2; ++part) {
            const int* nb = (part == 0 ? np : nc) + (size_t)g * k;
            const uint8_t* has = part == 0 ? has_pos : has_cov;
            const double* d = part == 0 ? dpos : dcov;
            double* fo = part == 0 ? fpos : fcov;
            const int dim = part == 0 ? 3 : 6;
            if (!has[g]) continue;
            int m = 0;
            while (m < k && nb[m] >= 0) ++m;
            for (int c = 0; c < dim; ++c) {
                vals[0] = d[(size_t)dim * g + c];
                for (int j = 0; j < m; ++j) vals[1 + j] = d[(size_t)dim * nb[j] + c];
                fo[(size_t)dim * g + c] = median_of(vals, m + 1);
            }
        }
    }
    /* pass 2: propagation of the filtered motion; new parameters */
#pragma omp parallel for schedule(dynamic, 64)
    for (int g = 0; g < n; ++g) {
        uint32_t fl = is_static[g] ? REG_STATIC : 0u;
        double newpos[3] = {0, 0, 0}, newcov[6] = {0, 0, 0, 0, 0, 0};
        for (int part = 0; part < 2; ++part) {
            const int* nb = (part == 0 ? np : nc) + (size_t)g * k;
            const uint8_t* has = part == 0 ? has_pos : has_cov;
            const double* fd = part == 0 ? fpos : fcov;
            const int dim = part == 0 ? 3 : 6;
            double* out = part == 0 ? newpos : newcov;
            if (is_static[g]) continue;                          /* motion discarded */
            int m = 0;
            while (m < k && nb[m] >= 0) ++m;
            if (has[g]) {
                for (int c = 0; c < dim; ++c) out[c] = fd[(size_t)dim * g + c];
                fl |= part == 0 ? REG_POS_MEDIAN : REG_COV_MEDIAN;
            } else if (m > 0) {
                for (int c = 0; c < dim; ++c) {
                    double acc = 0;
                    for (int j = 0; j < m; ++j) acc += fd[(size_t)dim * nb[j] + c];
                    out[c] = acc / m;
                }
                fl |= part == 0 ? REG_POS_PROPAGATED : REG_COV_PROPAGATED;
            }
        }
        for (int i = 0; i < 3; ++i) mo_out[4 * g + i] = (float)((double)mo0[4 * g + i] + newpos[i]);
        mo_out[4 * g + 3] = mo0[4 * g + 3];
        for (int i = 0; i < 3; ++i) s_out[4 * g + i] = (float)((double)s0[4 * g + i] + newcov[i]);
        s_out[4 * g + 3] = s0[4 * g + 3];
        double Ra[3][3], E[3][3], Rn[3][3], qn[4];
        rot_of_quat(q0 + 4 * (size_t)g, Ra);
        rot_of_euler(newcov + 3, E);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Rn[i][j] = E[i][0] * Ra[0][j] + E[i][1] * Ra[1][j] + E[i][2] * Ra[2][j];
        quat_of_rot(Rn, qn);
        const double dot = qn[0] * q0[4 * g] + qn[1] * q0[4 * g + 1] + qn[2] * q0[4 * g + 2] + qn[3] * q0[4 * g + 3];
        for (int i = 0; i < 4; ++i) q_out[4 * g + i] = (float)(dot < 0 ? -qn[i] : qn[i]);
        flags[g] = fl;
    }
    free(fpos); free(fcov);
    free(has_pos); free(has_cov); free(dpos); free(dcov); free(np); free(nc);
    return 0;
}

"""Hand-built scenes with known answers, for the pins and the parity tests.

Everything here is computed independently of the oracle and of the CUDA path:
the projected covariance uses the exact derivative of the pinhole map (complex-
step differentiation) and scipy's quaternion convention, so a slip in either
implementation's Eq. 1 shows up as a mismatch.
"""
from __future__ import annotations

import copy

import numpy as np
from scipy.spatial.transform import Rotation

import synth


def rotmat(q_wxyz) -> np.ndarray:
    q = np.asarray(q_wxyz, np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()


def cov3d(q_wxyz, s) -> np.ndarray:
    Rq = rotmat(q_wxyz)
    return Rq @ np.diag(np.asarray(s, np.float64) ** 2) @ Rq.T


def pinhole(scene, v, X):
    R = scene.R[v].astype(np.float64)
    t = scene.t[v].astype(np.float64)
    p = R @ X + t
    return np.array([float(scene.fx[v]) * p[0] / p[2] + float(scene.cx[v]),
                     float(scene.fy[v]) * p[1] / p[2] + float(scene.cy[v])])


def pinhole_jacobian(scene, v, X) -> np.ndarray:
    """d pinhole / d X by complex-step differentiation (exact to rounding)."""
    h = 1e-30
    J = np.zeros((2, 3))
    for k in range(3):
        Xc = np.asarray(X, np.float64).astype(complex)
        Xc[k] += 1j * h
        J[:, k] = pinhole(scene, v, Xc).imag / h
    return J


def projected(scene, v, X, S3):
    """(mu_2D, Sigma_2D) of a 3D Gaussian (mean X, covariance S3) in view v."""
    J = pinhole_jacobian(scene, v, X)
    return pinhole(scene, v, np.asarray(X, np.float64)).real, J @ S3 @ J.T


def affine_between(mu, S, mu2, S2):
    """An affine [A|b] with A S A^T = S2 and A mu + b = mu2 (Eq. 2)."""
    L = np.linalg.cholesky(S)
    L2 = np.linalg.cholesky(S2)
    A = L2 @ np.linalg.inv(L)
    return A, mu2 - A @ mu


def with_gaussians(base, means, quats, scales, opacity, rgb=None):
    """A scene with the cameras of ``base`` and the given Gaussians (SH degree 0)."""
    s = copy.copy(base)
    n = len(means)
    mo = np.zeros((n, 4), np.float32)
    mo[:, :3] = means
    mo[:, 3] = opacity
    sc = np.zeros((n, 4), np.float32)
    sc[:, :3] = scales
    q = np.asarray(quats, np.float32).reshape(n, 4)
    s.means_opacity, s.quats, s.scales = mo, q, sc
    rgb = np.full((n, 3), 0.75) if rgb is None else np.asarray(rgb, np.float64)
    s.sh_degree = 0
    s.sh = ((rgb - 0.5) / (0.5 / np.sqrt(np.pi))).reshape(n, 1, 3).astype(np.float32)
    s.labels = np.zeros(n, np.int32)
    s.disp = [np.zeros((int(s.height[v]), int(s.width[v]), 2), np.float32) for v in range(s.num_views)]
    s.vis = [np.ones((int(s.height[v]), int(s.width[v])), np.uint8) for v in range(s.num_views)]
    return s


def base_cameras(preset="tiny", views=None):
    return synth.make_scene(preset, seed=1, n=1, views=views, tracks=False)


def pixel_centres(scene, v):
    H, W = int(scene.height[v]), int(scene.width[v])
    xs, ys = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    return np.stack([xs, ys], -1)


def paint_affine(scene, v, A, b, mask=None):
    """Set tracks of view v to the affine field d(x) = A x + b - x (where mask)."""
    x = pixel_centres(scene, v)
    d = x @ np.asarray(A).T + b - x
    if mask is None:
        scene.disp[v] = d.astype(np.float32)
    else:
        scene.disp[v][mask] = d[mask].astype(np.float32)


def footprint_radius(S2, opacity):
    """Radius beyond which alpha < 1/255 for a 2D Gaussian (dilated by 0.3 px^2)."""
    lam = np.linalg.eigvalsh(S2 + 0.3 * np.eye(2)).max()
    return np.sqrt(max(2.0 * np.log(255.0 * opacity), 0.0) * lam)


def rigid_apply(scene, Rg, tg):
    """The same scene moved by the rigid transform X -> Rg X + tg (cameras follow).

    Tracks are kept: every camera sees exactly the same images.  Inputs are
    rounded to FP32 after the transform.
    """
    s = copy.copy(scene)
    X = scene.means_opacity[:, :3].astype(np.float64)
    mo = scene.means_opacity.copy()
    mo[:, :3] = (X @ Rg.T + tg).astype(np.float32)
    qg = Rotation.from_matrix(Rg)
    q = scene.quats.astype(np.float64)
    rq = qg * Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], 1))
    xyzw = rq.as_quat()
    s.means_opacity = mo
    s.quats = np.stack([xyzw[:, 3], xyzw[:, 0], xyzw[:, 1], xyzw[:, 2]], 1).astype(np.float32)
    R = scene.R.astype(np.float64)
    t = scene.t.astype(np.float64)
    s.R = np.einsum("vij,kj->vik", R, Rg).astype(np.float32)          # R Rg^T
    s.t = (t - np.einsum("vij,j->vi", s.R.astype(np.float64), tg)).astype(np.float32)
    return s


def masked_weights(sc, rng, margin=0.05):
    """Random loss weights, zero at pixels where some Gaussian's alpha lies within
    `margin` of the 1/255 cut or the 0.99 clamp: there a small parameter change
    could flip a blend decision, which the gradient (like any derivative of the
    blend) holds fixed."""
    import oracle
    cams = oracle.cameras(sc)
    W = []
    for v in range(sc.num_views):
        H, Wd = int(sc.height[v]), int(sc.width[v])
        w = rng.normal(size=(H, Wd, 3)).astype(np.float32)
        ys, xs = np.mgrid[0:H, 0:Wd] + 0.5
        mask = np.zeros((H, Wd), bool)
        for g in range(sc.n):
            m2, _, cn = oracle.project(sc.means_opacity[g], sc.quats[g], sc.scales[g], cams[v])
            dx, dy = xs - m2[0], ys - m2[1]
            a = sc.means_opacity[g, 3] * np.exp(-0.5 * (cn[0] * dx * dx + 2 * cn[1] * dx * dy + cn[2] * dy * dy))
            mask |= (np.abs(a * 255 - 1) < margin) | (np.abs(a / 0.99 - 1) < margin)
        w[mask] = 0
        W.append(w)
    return W

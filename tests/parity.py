"""Run the CUDA path through the C ABI and compare it with the oracle.

Tolerances (per solvable Gaussian, from the motion-fit target): position
1e-4 of the scene extent, rotation 1e-3 rad, scale 1e-4 relative; rendered
colour and transmittance 1e-4 absolute; per-view new mean 1e-3 px.

Conditioning.  An FP32 implementation differs from the FP64 oracle in two ways:
per-pixel weights carry ~1e-6 relative error, and the per-(view, Gaussian) moment
sums are stored in FP32.  Some fits are so ill-conditioned (a thin pixel set, a
1:200 axis ratio, an affine fitted across an object boundary in a sliver of
border pixels) that the FP64 oracle itself moves by more than the tolerance under
those perturbations.  ``sensitivity`` measures both: (1) the oracle re-run with
tracks and opacities scaled by (1 + u), u ~ U(-1e-6, 1e-6); (2) the oracle's own
moments, expressed in the library's layout (origin mu_2D clamped to the image,
displacement about the track at that origin), each moved by 2^-21 of a bound on
the sum of its terms' magnitudes (the FP32 summation error; three random draws)
and rounded to FP32, re-solved in FP64 and carried through the oracle's
multi-view update.  A quantity is held to
its tolerance only where the oracle moved by less than half of it under both;
the others are checked for validity only and counted.
"""
from __future__ import annotations

import copy
import math

import numpy as np

import oracle


def to_device(scene):
    import torch
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return dict(means_opacity=t(scene.means_opacity), quats=t(scene.quats), scales=t(scene.scales),
                disp=[t(d) for d in scene.disp], vis=[t(v) for v in scene.vis])


def run_gpu(scene, ctx=None, inspect=True, **opts):
    """Fit on the GPU; returns numpy outputs, per-view outputs and intermediates."""
    import torch
    import paper_2604_02586_b300 as tsp
    own = ctx is None
    if own:
        ctx = tsp.Context(0, **opts)
    d = to_device(scene)
    out = ctx.fit_motion(d["means_opacity"], d["quats"], d["scales"], scene, d["disp"], d["vis"],
                         view_affine=True, view_moments=True, view_flags=True)
    ctx.sync()
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["status"] = res["status"].view(np.uint32)
    res["view_flags"] = res["view_flags"].view(np.uint32)
    if inspect:
        T = tsp.TSP
        res["rect"] = ctx.inspect(T.I_RECT).reshape(scene.num_views, scene.n, 4)
        res["depth"] = ctx.inspect(T.I_DEPTH).reshape(scene.num_views, scene.n)
        res["touched"] = ctx.inspect(T.I_TILES_TOUCHED).reshape(scene.num_views, scene.n)
        res["tile_off"] = ctx.inspect(T.I_TILE_OFFSETS)
        res["pairs"] = ctx.inspect(T.I_PAIRS)
        res["counts"] = ctx.inspect(T.I_COUNTS)
        res["view_means"] = ctx.inspect(T.I_VIEW_MEANS).reshape(scene.num_views, scene.n, 4)
        res["view_B"] = ctx.inspect(T.I_VIEW_COV).reshape(scene.num_views, scene.n, 8)
    if own:
        ctx.close()
    return res


def library_frame(scene, orc):
    """The oracle's per-view moments restated in the library's frame (FP64).

    The library sums each (view, Gaussian) record about the origin o = mu_2D
    clamped to the image rectangle [0, W] x [0, H], with displacements taken
    about the reference r = the track at the pixel holding o (Sec. 4.3.5 sums,
    shifted; the per-view solve undoes both shifts).  This is exact algebra on
    the oracle's sums about mu_2D.  Returns
      mom   [V, n, 15] slots 0-12: sum w, sum w x~ (2), sum w x~x~^T (xx, xy, yy),
            sum w d~ (2), sum w x~_i d~_j (xx, xy, yx, yy), sum w over static
            pixels; 13, 14 the pixel counts (x~ = x - o, d~ = d - r);
      mag   [V, n, 13] Cauchy-Schwarz bounds on the sum of the terms' magnitudes
            of slots 0-12 (sum w |x~_i| <= sqrt(sum w . sum w x~_i^2), ...), from
            the second moments and the oracle's sum w |d|^2 bookkeeping slot;
      dl, r [V, n, 2] the origin shift o - mu_2D and the reference displacement;
      r_ambiguous [V, n] where the oracle's centre lies within 1e-4 px of a pixel
            boundary, so the FP32 centre may pick the neighbouring pixel's track."""
    M = orc["moments"]
    V, n = M.shape[:2]
    mu = orc["mean2d"]
    W = np.asarray(scene.width, np.float64)[:, None]
    H = np.asarray(scene.height, np.float64)[:, None]
    o = np.stack([np.clip(mu[..., 0], 0, W), np.clip(mu[..., 1], 0, H)], -1)
    dl = o - mu
    r = np.zeros_like(mu)
    amb = np.zeros((V, n), bool)
    for v in range(V):
        ox = np.clip(np.floor(o[v, :, 0]).astype(np.int64), 0, int(W[v, 0]) - 1)
        oy = np.clip(np.floor(o[v, :, 1]).astype(np.int64), 0, int(H[v, 0]) - 1)
        r[v] = scene.disp[v][oy, ox].astype(np.float64)
        fr = np.abs(o[v] - np.round(o[v]))
        amb[v] = ((fr[:, 0] < 1e-4) & (o[v, :, 0] > 0) & (o[v, :, 0] < W[v, 0])) | \
                 ((fr[:, 1] < 1e-4) & (o[v, :, 1] > 0) & (o[v, :, 1] < H[v, 0]))
    sw = M[..., 5]
    S1 = np.stack([M[..., 2], M[..., 4]], -1)
    S2 = np.stack([np.stack([M[..., 0], M[..., 1]], -1), np.stack([M[..., 1], M[..., 3]], -1)], -2)
    D1 = np.stack([M[..., 10] - M[..., 2], M[..., 11] - M[..., 4]], -1)
    Dx = np.stack([np.stack([M[..., 6] - M[..., 0], M[..., 7] - M[..., 1]], -1),
                   np.stack([M[..., 8] - M[..., 1], M[..., 9] - M[..., 3]], -1)], -2)
    out = lambda a, b: a[..., :, None] * b[..., None, :]
    sw_ = sw[..., None]
    S1o = S1 - sw_ * dl
    S2o = S2 - out(S1, dl) - out(dl, S1) + sw_[..., None] * out(dl, dl)
    D1o = D1 - sw_ * r
    Dxo = Dx - out(dl, D1) - out(S1, r) + sw_[..., None] * out(dl, r)
    mom = np.zeros((V, n, 15))
    mom[..., 0] = sw
    mom[..., 1:3] = S1o
    mom[..., 3], mom[..., 4], mom[..., 5] = S2o[..., 0, 0], S2o[..., 0, 1], S2o[..., 1, 1]
    mom[..., 6:8] = D1o
    mom[..., 8], mom[..., 9], mom[..., 10], mom[..., 11] = Dxo[..., 0, 0], Dxo[..., 0, 1], Dxo[..., 1, 0], Dxo[..., 1, 1]
    mom[..., 12], mom[..., 13], mom[..., 14] = M[..., 12], M[..., 13], M[..., 14]
    E2 = np.maximum(M[..., 17] - 2 * (r[..., 0] * D1[..., 0] + r[..., 1] * D1[..., 1])
                    + sw * (r ** 2).sum(-1), 0.0)
    s2 = np.maximum(np.stack([S2o[..., 0, 0], S2o[..., 1, 1]], -1), 0.0)
    mag = np.zeros((V, n, 13))
    mag[..., 0] = sw
    mag[..., 1:3] = np.sqrt(sw_ * s2)
    mag[..., 3], mag[..., 5] = s2[..., 0], s2[..., 1]
    mag[..., 4] = np.sqrt(s2[..., 0] * s2[..., 1])
    mag[..., 6:8] = np.sqrt(sw * E2)[..., None]
    mag[..., 8:10] = np.sqrt(s2[..., 0] * E2)[..., None]
    mag[..., 10:12] = np.sqrt(s2[..., 1] * E2)[..., None]
    mag[..., 12] = M[..., 12]
    return dict(mom=mom, mag=mag, dl=dl, r=r, r_ambiguous=amb, E2=E2)


def oracle_record_from_library(lib, dl, r):
    """Inverse of ``library_frame``: records in the library's frame ([..., 15]
    slots, sums about the origin o = mu_2D + dl and the reference r) -> the
    oracle's record layout (sums about mu_2D, x' = x + d; [..., 18], the
    bookkeeping slots 15-17 zero).  Exact algebra, in FP64."""
    L = np.asarray(lib, np.float64)
    sw = L[..., 0]
    S1o = L[..., 1:3]
    S2o = _sym2(L[..., 3:6])
    D1o = L[..., 6:8]
    Dxo = np.stack([np.stack([L[..., 8], L[..., 9]], -1), np.stack([L[..., 10], L[..., 11]], -1)], -2)
    out = lambda a, b: a[..., :, None] * b[..., None, :]
    sw_ = sw[..., None]
    S1 = S1o + sw_ * dl
    S2 = S2o + out(S1o, dl) + out(dl, S1o) + sw_[..., None] * out(dl, dl)
    D1 = D1o + sw_ * r
    Dx = Dxo + out(dl, D1o) + out(S1o, r) + sw_[..., None] * out(dl, r)
    M = np.zeros(L.shape[:-1] + (18,))
    M[..., 5] = sw
    M[..., 2], M[..., 4] = S1[..., 0], S1[..., 1]
    M[..., 0], M[..., 1], M[..., 3] = S2[..., 0, 0], S2[..., 0, 1], S2[..., 1, 1]
    M[..., 6], M[..., 7] = Dx[..., 0, 0] + M[..., 0], Dx[..., 0, 1] + M[..., 1]
    M[..., 8], M[..., 9] = Dx[..., 1, 0] + M[..., 1], Dx[..., 1, 1] + M[..., 3]
    M[..., 10], M[..., 11] = D1[..., 0] + M[..., 2], D1[..., 1] + M[..., 4]
    M[..., 12], M[..., 13], M[..., 14] = L[..., 12], L[..., 13], L[..., 14]
    return M


def window_feature_bound(scene, orc, lf, pairs):
    """For the (view, Gaussian) pairs given as (v, g) index arrays: a bound on
    |f_q| over the pixels the Gaussian can reach, for each moment slot q's
    per-pixel feature f_q (1, x~, y~, x~^2, ... as in ``library_frame``).  A pixel
    contributes only where alpha >= 1/255, i.e. inside the ellipse
    (x - mu)^T (Sigma_2D + 0.3 I)^-1 (x - mu) <= 2 ln(255 o); the track deviation
    |d - r| is bounded by its maximum over that ellipse's bounding box."""
    V, n = orc["moments"].shape[:2]
    vv, gg = pairs
    F = np.zeros((len(vv), 13))
    op = scene.means_opacity[:, 3].astype(np.float64)
    for j, (v, g) in enumerate(zip(vv, gg)):
        q = 2.0 * math.log(max(255.0 * op[g], 1.0))
        c = orc["cov2d"][v, g]
        rx, ry = math.sqrt(q * (c[0] + 0.3)), math.sqrt(q * (c[2] + 0.3))
        mx, my = orc["mean2d"][v, g]
        Wv, Hv = int(scene.width[v]), int(scene.height[v])
        x0, x1 = max(int(math.floor(mx - rx - 0.5)), 0), min(int(math.ceil(mx + rx + 0.5)), Wv - 1)
        y0, y1 = max(int(math.floor(my - ry - 0.5)), 0), min(int(math.ceil(my + ry + 0.5)), Hv - 1)
        ox, oy = lf["dl"][v, g] + orc["mean2d"][v, g]
        ax = max(abs(x0 + 0.5 - ox), abs(x1 + 0.5 - ox))
        ay = max(abs(y0 + 0.5 - oy), abs(y1 + 0.5 - oy))
        if x1 >= x0 and y1 >= y0:
            d = scene.disp[v][y0:y1 + 1, x0:x1 + 1].astype(np.float64)
            ddx = float(np.abs(d[..., 0] - lf["r"][v, g, 0]).max())
            ddy = float(np.abs(d[..., 1] - lf["r"][v, g, 1]).max())
        else:
            ddx = ddy = 0.0
        F[j] = [1.0, ax, ay, ax * ax, ax * ay, ay * ay, ddx, ddy, ax * ddx, ax * ddy, ay * ddx, ay * ddy, 1.0]
    return F


def perturbed(scene, rel=1e-6, seed=2024):
    rng = np.random.default_rng(seed)
    s = copy.copy(scene)
    s.disp = [(d.astype(np.float64) * (1 + rel * rng.uniform(-1, 1, d.shape))).astype(np.float32)
              for d in scene.disp]
    mo = scene.means_opacity.astype(np.float64).copy()
    mo[:, 3] *= 1 + rel * rng.uniform(-1, 1, mo.shape[0])
    s.means_opacity = mo.astype(np.float32)
    return s


def quat_rot_batch(q):
    """Rotation matrices [m, 3, 3] of quaternions (w, x, y, z) [m, 4] (normalised)."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def cov_batch(q, s):
    """Sigma = R(q) diag(s^2) R(q)^T for [m] quaternions and scales."""
    R = quat_rot_batch(q)
    s2 = np.asarray(s, np.float64)[..., :3] ** 2
    return np.einsum("mij,mj,mkj->mik", R, s2, R)


def _cov_rel(Ca, Cb):
    den = np.linalg.norm(Cb.reshape(len(Cb), -1), axis=1)
    return np.linalg.norm((Ca - Cb).reshape(len(Ca), -1), axis=1) / np.maximum(den, 1e-300)


def _sym2(c):
    """[..., 3] (xx, xy, yy) -> [..., 2, 2]."""
    return np.stack([np.stack([c[..., 0], c[..., 1]], -1), np.stack([c[..., 1], c[..., 2]], -1)], -2)


def cov2_rel(ca, cb):
    """Relative Frobenius distance of 2x2 covariances given as (xx, xy, yy)."""
    A, B = _sym2(np.asarray(ca, np.float64)), _sym2(np.asarray(cb, np.float64))
    num = np.sqrt(((A - B) ** 2).sum((-1, -2)))
    den = np.sqrt((B ** 2).sum((-1, -2)))
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(den > 0, num / np.maximum(den, 1e-300), 0.0)


def _response(scene, orc, o2, ids):
    return dict(status_stable=(o2["out_status"][ids] == orc["out_status"][ids]),
                pos=np.linalg.norm(o2["out_mean"][ids] - orc["out_mean"][ids], axis=1) / scene.extent,
                scale=np.abs(o2["out_scale"][ids] / np.maximum(orc["out_scale"][ids], 1e-30) - 1).max(1),
                angle=rot_angle(o2["out_quat"][ids], orc["out_quat"][ids]),
                cov3=_cov_rel(cov_batch(o2["out_quat"][ids], o2["out_scale"][ids]),
                              cov_batch(orc["out_quat"][ids], orc["out_scale"][ids])))


def fp32_moment_rounding(scene, orc, ids, rel=2.0 ** -21, seed=7):
    """Oracle outputs when its per-view moments are FP32 sums in the library's
    frame (``library_frame``).  The library forms each sum from 32-term per-lane
    partial sums, one shuffle add and one atomic add per 8x8 block hit (some 20),
    so it is off by about sqrt(52) units in the last place -- 2^-21 -- of the sum
    of the terms' magnitudes, which for sums of mixed sign (first moments about
    the origin, displacement terms about the reference) is far larger than 2^-21
    of the sum itself.  Each sum therefore moves by rel * u * m, u ~ U(-1, 1),
    with m the slot's magnitude bound, and is rounded to FP32; the record is then
    taken back to the oracle's frame, re-solved in FP64 and carried through the
    oracle's multi-view update.  Needs per-view oracle outputs."""
    M = orc["moments"]
    V, n = M.shape[:2]
    mu = orc["mean2d"]
    lf = library_frame(scene, orc)
    dl, r, L, mag = lf["dl"], lf["r"], lf["mom"], lf["mag"]
    rng = np.random.default_rng(seed)
    f = lambda a, m: (a + rel * m * rng.uniform(-1, 1, a.shape)).astype(np.float32).astype(np.float64)
    Lb = L.copy()
    Lb[..., :12] = f(L[..., :12], mag[..., :12])
    Mb = M.copy()
    Mb[..., :12] = oracle_record_from_library(Lb, dl, r)[..., :12]
    flags = orc["view_flags"].copy()
    mu2 = orc["view_mean2d"].copy()
    cov2 = orc["view_cov2d"].copy()
    for g in ids:
        for v in range(V):
            if orc["view_flags"][v, g] & oracle.OV_CULLED:
                continue
            fl, _, m2, c2 = oracle.view_solve(Mb[v, g, :16], mu[v, g], orc["cov2d"][v, g])
            flags[v, g], mu2[v, g], cov2[v, g] = fl, m2, c2
    res = dict(out_status=orc["out_status"].copy(), out_mean=orc["out_mean"].copy(),
               out_quat=orc["out_quat"].copy(), out_scale=orc["out_scale"].copy())
    for g in ids:
        r_ = oracle.multiview(scene, int(g), flags[:, g], M[:, g, 5], M[:, g, 13], mu2[:, g], cov2[:, g])
        res["out_status"][g] = r_["status"]
        res["out_mean"][g], res["out_quat"][g], res["out_scale"][g] = r_["mean"], r_["quat"], r_["scale"]
    res["view_mean2d"], res["view_flags"], res["view_cov2d"] = mu2, flags, cov2
    return res


def sensitivity(scene, orc, sample=None, rel=1e-6, options=None):
    """Oracle response to FP32-sized perturbations (see the module docstring);
    ``options``: the oracle options ``orc`` was computed with (tile shape).
    Per Gaussian: status_stable, pos (/ extent), scale (relative), angle (rad),
    cov3 (relative Frobenius of Sigma_3D'); per (view, Gaussian), without a
    sample: view_flags_stable, mu (px), cov2 (relative Frobenius of Sigma_2D')."""
    n = scene.n
    ids = np.arange(n) if sample is None else np.asarray(sample)
    per_view = "view_mean2d" in orc
    o2 = oracle.fit_motion(perturbed(scene, rel), options, sample=sample, per_view=per_view)
    a = _response(scene, orc, o2, ids)
    if not per_view:
        return a
    # three draws of the rounding model: one random direction can miss a sensitive one
    o3s = [fp32_moment_rounding(scene, orc, ids, seed=sd) for sd in (7, 8, 9)]
    bs = [_response(scene, orc, o, ids) for o in o3s]
    keys = ("pos", "scale", "angle", "cov3")
    out = dict(status_stable=a["status_stable"] & np.logical_and.reduce([x["status_stable"] for x in bs]))
    for k in keys:
        out[k] = np.maximum(a[k], np.max([x[k] for x in bs], 0))
    if sample is None:
        m1 = np.linalg.norm(o2["view_mean2d"] - orc["view_mean2d"], axis=-1)
        m2 = np.max([np.linalg.norm(o["view_mean2d"] - orc["view_mean2d"], axis=-1) for o in o3s], 0)
        out["mu"] = np.maximum(m1, m2)
        c1 = cov2_rel(o2["view_cov2d"], orc["view_cov2d"])
        c2 = np.max([cov2_rel(o["view_cov2d"], orc["view_cov2d"]) for o in o3s], 0)
        out["cov2"] = np.maximum(c1, c2)
        out["view_flags_stable"] = (o2["view_flags"] == orc["view_flags"]) & \
            np.logical_and.reduce([o["view_flags"] == orc["view_flags"] for o in o3s])
    return out


def rot_angle(qa, qb):
    """Angle of the rotation between two quaternions (either sign).  Taken as
    4 asin(|qa - qb| / 2) with qb on qa's side: 2 acos(|qa . qb|) loses half the
    digits near 0 (the FP32 rounding of a unit quaternion alone reads as 6e-4 rad
    there)."""
    qa = np.asarray(qa, np.float64)
    qb = np.asarray(qb, np.float64)
    qa = qa / np.linalg.norm(qa, axis=-1, keepdims=True)
    qb = qb / np.linalg.norm(qb, axis=-1, keepdims=True)
    sgn = np.where((qa * qb).sum(-1) < 0, -1.0, 1.0)[..., None]
    return 4 * np.arcsin(np.clip(np.linalg.norm(qa - sgn * qb, axis=-1) / 2, 0, 1))


def quat_rot(q):
    return quat_rot_batch(np.asarray(q, np.float64)[None])[0]


def cov_from(q, s):
    return cov_batch(np.asarray(q, np.float64)[None], np.asarray(s, np.float64)[None])[0]


def compare_outputs(scene, gpu, orc, ids=None):
    """Per-Gaussian comparison; returns a dict of statistics and index sets."""
    n = scene.n
    ids = np.arange(n) if ids is None else np.asarray(ids)
    sg = gpu["status"][ids] & 0xFF
    so = orc["out_status"][ids] & 0xFF
    E = scene.extent
    both_pos = ((sg & 1) > 0) & ((so & 1) > 0)
    both_cov = ((sg & 2) > 0) & ((so & 2) > 0)
    pos_err = np.linalg.norm(gpu["means"][ids, :3].astype(np.float64) - orc["out_mean"][ids], axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        scale_rel = np.abs(gpu["scales"][ids, :3] / orc["out_scale"][ids] - 1).max(1)
    ang = rot_angle(gpu["quats"][ids], orc["out_quat"][ids])
    # eigen-gap: where two fitted eigenvalues (nearly) coincide the rotation is not
    # unique, so the fitted covariance is compared instead of the rotation
    lam = np.sort(orc["out_scale"][ids].astype(np.float64) ** 2, axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        gap = np.where(both_cov, np.minimum(lam[:, 1] - lam[:, 0], lam[:, 2] - lam[:, 1]) /
                       np.maximum(lam[:, 2], 1e-300), 1.0)
    cov_rel = np.zeros(len(ids))
    if both_cov.any():
        j = np.flatnonzero(both_cov)
        g = ids[j]
        cov_rel[j] = _cov_rel(cov_batch(gpu["quats"][g], gpu["scales"][g]),
                              cov_batch(orc["out_quat"][g], orc["out_scale"][g]))
    return dict(status_equal=float((sg == so).mean()), n=len(ids), status_equal_mask=(sg == so),
                status_mismatch=ids[sg != so], both_pos=both_pos, both_cov=both_cov,
                pos_err=pos_err / E, scale_rel=scale_rel, angle=ang, gap=gap, cov_rel=cov_rel,
                views=(orc["out_status"][ids] >> 16) & 0xFF)


# Gaussians whose oracle outputs move by more than half a tolerance under the
# FP32-sized perturbations of ``sensitivity`` are held to tol + K_SENS * (that
# movement) instead of tol, so no solved Gaussian goes unchecked.
K_SENS = 4.0
GAP_MIN, COV3_TOL = 1e-3, 2e-4


def summarize(cmp, sens=None, pos_tol=1e-4, scale_tol=1e-4, rot_tol=1e-3, cov3_tol=COV3_TOL, k_sens=K_SENS):
    """Statistics over the Gaussians the comparison applies to.  With ``sens``
    (from sensitivity), quantities the oracle cannot pin to half their tolerance
    are counted under excluded_* and held to tol + k_sens * sensitivity
    (*_excl_fail counts the ones over it).  Rotations are compared where the
    fitted eigenvalues are apart (relative gap >= 1e-3); elsewhere the fitted
    covariance is (relative Frobenius <= 2e-4).  "covall" compares the fitted
    covariance of every Gaussian with a fitted covariance the same way (the
    near-degenerate case is rare in these scenes, so this is what exercises
    that comparison)."""
    n = cmp["n"]
    z = np.zeros(n)
    sv = (lambda k: z) if sens is None else (lambda k: sens[k])
    stable = np.ones(n, bool) if sens is None else sens["status_stable"]
    bp, bc = cmp["both_pos"], cmp["both_cov"]
    big_gap = cmp["gap"] >= GAP_MIN
    res = dict(n=n, status_equal=cmp["status_equal"],
               status_equal_stable=float((np.asarray(cmp["status_equal_mask"]) | ~stable).mean()),
               status_mismatch_stable=int((~np.asarray(cmp["status_equal_mask"]) & stable).sum()),
               unstable_status=int((~stable).sum()),
               n_both_pos=int(bp.sum()), n_both_cov=int(bc.sum()),
               n_small_gap=int((bc & ~big_gap).sum()))
    worst = {}
    for name, err, tol, skey, base in (("pos", cmp["pos_err"], pos_tol, "pos", bp),
                                       ("scale", cmp["scale_rel"], scale_tol, "scale", bc),
                                       ("angle", cmp["angle"], rot_tol, "angle", bc & big_gap),
                                       ("cov", cmp["cov_rel"], cov3_tol, "cov3", bc & ~big_gap),
                                       ("covall", cmp["cov_rel"], cov3_tol, "cov3", bc)):
        s = sv(skey)
        tight = base & (s < tol / 2) & stable
        excl = base & ~tight
        bound = tol + k_sens * s
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = np.where(s > 0, err / np.maximum(s, 1e-300), np.inf)
        res[f"{name}_max"] = float(err[tight].max()) if tight.any() else 0.0
        res[f"{name}_fail"] = int((err[tight] > tol).sum())
        res[f"excluded_{name}"] = int(excl.sum())
        res[f"{name}_excl_fail"] = int((err[excl] > bound[excl]).sum())
        res[f"{name}_excl_err_max"] = float(err[excl].max()) if excl.any() else 0.0
        res[f"{name}_excl_ratio_max"] = float(ratio[excl].max()) if excl.any() else 0.0
        idx = np.flatnonzero(base)
        idx = idx[np.argsort((err[idx] / bound[idx]))[::-1][:3]]
        worst[name] = [(int(i), float(err[i]), float(s[i]), int(cmp["views"][i])) for i in idx]
    res["excluded_rot"] = res["excluded_angle"]
    res["worst"] = worst
    return res


def log_stats(tag, stats):
    """Append one JSON line of parity statistics to $TSP_PARITY_LOG, if set."""
    import json
    import os
    path = os.environ.get("TSP_PARITY_LOG")
    if not path:
        return
    clean = {k: v for k, v in stats.items() if not isinstance(v, np.ndarray)}
    with open(path, "a") as f:
        f.write(json.dumps({"case": tag, **clean}, default=float) + "\n")

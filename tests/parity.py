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


def oracle_moments_in_library_layout(om):
    """Oracle record (V1, V2 about mu_2D) -> library record (sum w d based)."""
    g = np.zeros(om.shape[:-1] + (16,))
    g[..., 0] = om[..., 5]
    g[..., 1] = om[..., 2]
    g[..., 2] = om[..., 4]
    g[..., 3] = om[..., 0]
    g[..., 4] = om[..., 1]
    g[..., 5] = om[..., 3]
    g[..., 6] = om[..., 10] - om[..., 2]
    g[..., 7] = om[..., 11] - om[..., 4]
    g[..., 8] = om[..., 6] - om[..., 0]
    g[..., 9] = om[..., 7] - om[..., 1]
    g[..., 10] = om[..., 8] - om[..., 1]
    g[..., 11] = om[..., 9] - om[..., 3]
    g[..., 12] = om[..., 12]
    g[..., 13] = om[..., 13]
    g[..., 14] = om[..., 14]
    return g


def perturbed(scene, rel=1e-6, seed=2024):
    rng = np.random.default_rng(seed)
    s = copy.copy(scene)
    s.disp = [(d.astype(np.float64) * (1 + rel * rng.uniform(-1, 1, d.shape))).astype(np.float32)
              for d in scene.disp]
    mo = scene.means_opacity.astype(np.float64).copy()
    mo[:, 3] *= 1 + rel * rng.uniform(-1, 1, mo.shape[0])
    s.means_opacity = mo.astype(np.float32)
    return s


def _response(scene, orc, o2, ids):
    return dict(status_stable=(o2["out_status"][ids] == orc["out_status"][ids]),
                pos=np.linalg.norm(o2["out_mean"][ids] - orc["out_mean"][ids], axis=1) / scene.extent,
                scale=np.abs(o2["out_scale"][ids] / np.maximum(orc["out_scale"][ids], 1e-30) - 1).max(1),
                angle=rot_angle(o2["out_quat"][ids], orc["out_quat"][ids]))


def fp32_moment_rounding(scene, orc, ids, rel=2.0 ** -21, seed=7):
    """Oracle outputs when its per-view moments are FP32 sums in the library's
    layout (see the module docstring).  The library forms each sum from 32-term
    per-lane partial sums, one shuffle add and one atomic add per 8x8 block hit
    (some 20), so it is off by about sqrt(52) units in the last place -- 2^-21 --
    of the sum of the terms' magnitudes, which for sums of mixed sign (first
    moments about the origin, displacement terms about the reference) is far
    larger than 2^-21 of the sum itself.  Each sum therefore
    moves by rel * u * m, u ~ U(-1, 1), with m a Cauchy-Schwarz bound on the
    magnitude sum built from the second moments (sum w |x~|^2 from the moment
    record, sum w |d - r|^2 from its bookkeeping slot), and is rounded to FP32.
    Needs per-view oracle outputs."""
    M = orc["moments"]
    V, n = M.shape[:2]
    mu = orc["mean2d"]
    W = scene.width.astype(np.float64)[:, None]
    H = scene.height.astype(np.float64)[:, None]
    o = np.stack([np.clip(mu[..., 0], 0, W), np.clip(mu[..., 1], 0, H)], -1)
    dl = o - mu
    r = np.zeros_like(mu)
    for v in range(V):
        ox = np.clip(np.floor(o[v, :, 0]).astype(np.int64), 0, int(W[v, 0]) - 1)
        oy = np.clip(np.floor(o[v, :, 1]).astype(np.int64), 0, int(H[v, 0]) - 1)
        r[v] = scene.disp[v][oy, ox].astype(np.float64)
    sw = M[..., 5]
    S1 = np.stack([M[..., 2], M[..., 4]], -1)
    S2 = np.stack([np.stack([M[..., 0], M[..., 1]], -1), np.stack([M[..., 1], M[..., 3]], -1)], -2)
    D1 = np.stack([M[..., 10] - M[..., 2], M[..., 11] - M[..., 4]], -1)
    Dx = np.stack([np.stack([M[..., 6] - M[..., 0], M[..., 7] - M[..., 1]], -1),
                   np.stack([M[..., 8] - M[..., 1], M[..., 9] - M[..., 3]], -1)], -2)
    out = lambda a, b: a[..., :, None] * b[..., None, :]
    sw_ = sw[..., None]
    # to the library's origin and reference, rounded to FP32, and back (FP64 algebra)
    S1o = S1 - sw_ * dl
    S2o = S2 - out(S1, dl) - out(dl, S1) + sw_[..., None] * out(dl, dl)
    D1o = D1 - sw_ * r
    Dxo = Dx - out(dl, D1) - out(S1, r) + sw_[..., None] * out(dl, r)
    # magnitude bounds: sum w |x~_i| <= sqrt(sw S2_ii), sum w |x~_i (d - r)_j| <= sqrt(S2_ii E2)
    E2 = np.maximum(M[..., 17] - 2 * (r[..., 0] * (M[..., 10] - M[..., 2]) + r[..., 1] * (M[..., 11] - M[..., 4]))
                    + sw * (r ** 2).sum(-1), 0.0)
    s2d = np.maximum(np.stack([S2o[..., 0, 0], S2o[..., 1, 1]], -1), 0.0)
    m_S1 = np.sqrt(sw_ * s2d)
    m_S2 = np.sqrt(s2d[..., :, None] * s2d[..., None, :])
    m_D1 = np.sqrt(sw_ * E2[..., None]) * np.ones(2)
    m_Dx = np.sqrt(s2d[..., :, None] * E2[..., None, None]) * np.ones((2, 2))
    rng = np.random.default_rng(seed)
    f = lambda a, m: (a + rel * m * rng.uniform(-1, 1, a.shape)).astype(np.float32).astype(np.float64)
    sw2, S1o, S2o, D1o, Dxo = f(sw, sw), f(S1o, m_S1), f(S2o, m_S2), f(D1o, m_D1), f(Dxo, m_Dx)
    sw2_ = sw2[..., None]
    S1b = S1o + sw2_ * dl
    S2b = S2o + out(S1o, dl) + out(dl, S1o) + sw2_[..., None] * out(dl, dl)
    D1b = D1o + sw2_ * r
    Dxb = Dxo + out(dl, D1o) + out(S1o, r) + sw2_[..., None] * out(dl, r)
    Mb = M.copy()
    Mb[..., 5] = sw2
    Mb[..., 2], Mb[..., 4] = S1b[..., 0], S1b[..., 1]
    Mb[..., 0], Mb[..., 1], Mb[..., 3] = S2b[..., 0, 0], S2b[..., 0, 1], S2b[..., 1, 1]
    Mb[..., 6], Mb[..., 7] = Dxb[..., 0, 0] + Mb[..., 0], Dxb[..., 0, 1] + Mb[..., 1]
    Mb[..., 8], Mb[..., 9] = Dxb[..., 1, 0] + Mb[..., 1], Dxb[..., 1, 1] + Mb[..., 3]
    Mb[..., 10], Mb[..., 11] = D1b[..., 0] + Mb[..., 2], D1b[..., 1] + Mb[..., 4]
    flags = orc["view_flags"].copy()
    mu2 = orc["view_mean2d"].copy()
    cov2 = orc["view_cov2d"].copy()
    touched = np.zeros((V, n), bool)
    for g in ids:
        for v in range(V):
            if orc["view_flags"][v, g] & oracle.OV_CULLED:
                continue
            fl, _, m2, c2 = oracle.view_solve(Mb[v, g, :16], mu[v, g], orc["cov2d"][v, g])
            flags[v, g], mu2[v, g], cov2[v, g] = fl, m2, c2
            touched[v, g] = True
    res = dict(out_status=orc["out_status"].copy(), out_mean=orc["out_mean"].copy(),
               out_quat=orc["out_quat"].copy(), out_scale=orc["out_scale"].copy())
    for g in ids:
        r_ = oracle.multiview(scene, int(g), flags[:, g], M[:, g, 5], M[:, g, 13], mu2[:, g], cov2[:, g])
        res["out_status"][g] = r_["status"]
        res["out_mean"][g], res["out_quat"][g], res["out_scale"][g] = r_["mean"], r_["quat"], r_["scale"]
    res["view_mean2d"], res["view_flags"] = mu2, flags
    return res


def sensitivity(scene, orc, sample=None, rel=1e-6, options=None):
    """Oracle response to FP32-sized perturbations (see the module docstring);
    ``options``: the oracle options ``orc`` was computed with (tile shape)."""
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
    b = dict(status_stable=np.logical_and.reduce([x["status_stable"] for x in bs]),
             pos=np.max([x["pos"] for x in bs], 0), scale=np.max([x["scale"] for x in bs], 0),
             angle=np.max([x["angle"] for x in bs], 0))
    o3 = o3s[0]
    out = dict(status_stable=a["status_stable"] & b["status_stable"],
               pos=np.maximum(a["pos"], b["pos"]), scale=np.maximum(a["scale"], b["scale"]),
               angle=np.maximum(a["angle"], b["angle"]))
    if sample is None:
        m1 = np.linalg.norm(o2["view_mean2d"] - orc["view_mean2d"], axis=-1)
        m2 = np.max([np.linalg.norm(o["view_mean2d"] - orc["view_mean2d"], axis=-1) for o in o3s], 0)
        out["mu"] = np.maximum(m1, m2)
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
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def cov_from(q, s):
    R = quat_rot(q)
    return R @ np.diag(np.asarray(s, np.float64)[:3] ** 2) @ R.T


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
    scale_rel = np.abs(gpu["scales"][ids, :3] / orc["out_scale"][ids] - 1).max(1)
    ang = rot_angle(gpu["quats"][ids], orc["out_quat"][ids])
    # eigen-gap: where two fitted eigenvalues (nearly) coincide the rotation is not
    # unique, so the fitted covariance is compared instead of the rotation
    gap = np.ones(len(ids))
    cov_rel = np.zeros(len(ids))
    for j, g in enumerate(ids):
        if not both_cov[j]:
            continue
        lam = np.sort(orc["out_scale"][g] ** 2)
        gap[j] = min(lam[1] - lam[0], lam[2] - lam[1]) / lam[2]
        Cg = cov_from(gpu["quats"][g], gpu["scales"][g])
        Co = cov_from(orc["out_quat"][g], orc["out_scale"][g])
        cov_rel[j] = np.linalg.norm(Cg - Co) / np.linalg.norm(Co)
    return dict(status_equal=float((sg == so).mean()), n=len(ids), status_equal_mask=(sg == so),
                status_mismatch=ids[sg != so], both_pos=both_pos, both_cov=both_cov,
                pos_err=pos_err / E, scale_rel=scale_rel, angle=ang, gap=gap, cov_rel=cov_rel,
                views=(orc["out_status"][ids] >> 16) & 0xFF)


def summarize(cmp, sens=None, pos_tol=1e-4, scale_tol=1e-4, rot_tol=1e-3):
    """Statistics over the Gaussians the comparison applies to.  With ``sens``
    (from sensitivity), quantities the oracle cannot pin to half their tolerance
    are left out and counted under excluded_*."""
    n = cmp["n"]
    ok_pos = np.ones(n, bool) if sens is None else (sens["pos"] < pos_tol / 2) & sens["status_stable"]
    ok_scale = np.ones(n, bool) if sens is None else (sens["scale"] < scale_tol / 2) & sens["status_stable"]
    ok_rot = np.ones(n, bool) if sens is None else (sens["angle"] < rot_tol / 2) & sens["status_stable"]
    stable = np.ones(n, bool) if sens is None else sens["status_stable"]
    pe = cmp["pos_err"][cmp["both_pos"] & ok_pos]
    bc = cmp["both_cov"]
    sr = cmp["scale_rel"][bc & ok_scale]
    ok_gap = bc & (cmp["gap"] >= 1e-3) & ok_rot
    an = cmp["angle"][ok_gap]
    status_eq = (np.asarray(cmp["status_equal_mask"]) | ~stable)
    q = lambda a, p: float(np.quantile(a, p)) if a.size else 0.0
    return dict(n=n, status_equal=cmp["status_equal"], status_equal_stable=float(status_eq.mean()),
                excluded_pos=int((cmp["both_pos"] & ~ok_pos).sum()),
                excluded_scale=int((bc & ~ok_scale).sum()), excluded_rot=int((bc & ~ok_rot).sum()),
                unstable_status=int((~stable).sum()),
                pos_max=float(pe.max()) if pe.size else 0.0, pos_p99=q(pe, 0.99),
                pos_fail=int((pe > 1e-4).sum()),
                scale_max=float(sr.max()) if sr.size else 0.0, scale_p99=q(sr, 0.99),
                scale_fail=int((sr > 1e-4).sum()),
                angle_max=float(an.max()) if an.size else 0.0, angle_fail=int((an > 1e-3).sum()),
                cov_rel_max=float(cmp["cov_rel"][bc].max()) if bc.any() else 0.0,
                n_both_pos=int(cmp["both_pos"].sum()), n_both_cov=int(bc.sum()),
                worst=_worst(cmp, sens, bc & ok_scale, ok_gap, cmp["both_pos"] & ok_pos))


def _worst(cmp, sens, m_scale, m_rot, m_pos, k=3):
    """The k largest errors of each kind with their oracle sensitivity and the
    number of views, for failure messages."""
    out = {}
    for name, err, m, key in (("scale", cmp["scale_rel"], m_scale, "scale"),
                              ("angle", cmp["angle"], m_rot, "angle"),
                              ("pos", cmp["pos_err"], m_pos, "pos")):
        idx = np.flatnonzero(m)
        idx = idx[np.argsort(err[idx])[::-1][:k]]
        out[name] = [(int(i), float(err[i]), float(sens[key][i]) if sens is not None else None,
                      int(cmp["views"][i])) for i in idx]
    return out

"""Run the CUDA path through the C ABI and compare it with the oracle.

Tolerances (per solvable Gaussian, from the motion-fit target): position
1e-4 of the scene extent, rotation 1e-3 rad, scale 1e-4 relative; rendered
colour and transmittance 1e-4 absolute.  Per-view intermediates get bounds that
keep those: mean shift 1e-3 px, affine 1e-4, Sigma_2D' 1e-3 of its largest
eigenvalue.  Items whose oracle value sits within a threshold margin are
compared only for validity and counted.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

O2G = None  # filled lazily: oracle moment layout -> library moment layout


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


def rot_angle(qa, qb):
    qa = np.asarray(qa, np.float64)
    qb = np.asarray(qb, np.float64)
    qa = qa / np.linalg.norm(qa, axis=-1, keepdims=True)
    qb = qb / np.linalg.norm(qb, axis=-1, keepdims=True)
    d = np.abs((qa * qb).sum(-1)).clip(0, 1)
    return 2 * np.arccos(d)


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
    return dict(status_equal=float((sg == so).mean()), n=len(ids),
                status_mismatch=ids[sg != so], both_pos=both_pos, both_cov=both_cov,
                pos_err=pos_err / E, scale_rel=scale_rel, angle=ang, gap=gap, cov_rel=cov_rel)


def summarize(cmp):
    pe = cmp["pos_err"][cmp["both_pos"]]
    bc = cmp["both_cov"]
    sr = cmp["scale_rel"][bc]
    ok_gap = bc & (cmp["gap"] >= 1e-3)
    an = cmp["angle"][ok_gap]
    q = lambda a, p: float(np.quantile(a, p)) if a.size else 0.0
    return dict(n=cmp["n"], status_equal=cmp["status_equal"],
                pos_max=float(pe.max()) if pe.size else 0.0, pos_p99=q(pe, 0.99),
                pos_fail=int((pe > 1e-4).sum()),
                scale_max=float(sr.max()) if sr.size else 0.0, scale_p99=q(sr, 0.99),
                scale_fail=int((sr > 1e-4).sum()),
                angle_max=float(an.max()) if an.size else 0.0, angle_fail=int((an > 1e-3).sum()),
                cov_rel_max=float(cmp["cov_rel"][bc].max()) if bc.any() else 0.0,
                n_both_pos=int(cmp["both_pos"].sum()), n_both_cov=int(bc.sum()))

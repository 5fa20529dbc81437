"""Seeded synthetic multi-view inputs for the track-to-Gaussian motion fit.

This module only draws random numbers and shapes them into inputs: 3D Gaussians,
pinhole cameras, a ground-truth rigid motion per Gaussian and dense per-view
pixel tracks with a visibility flag.  It is shared by the oracle tests, the GPU
parity tests and the benchmark, and it holds none of the method's arithmetic:
no covariance projection, no alpha blending, no least squares, no triangulation
and no eigen decomposition.

Tracks stand in for the output of a dense point tracker (the paper uses DOT,
Sec. 3.2).  They are made the way such a tracker sees a scene of opaque points:
a point-splat z-buffer keeps, per pixel, the nearest Gaussian centre whose disc
(radius 1.5 x its largest scale, in pixels) covers the pixel; the pixel is lifted
to that centre's depth, moved with that Gaussian's rigid motion and re-imaged.
The displacement x' - x gets i.i.d. Gaussian noise; pixels with no z-buffer hit
carry noise only and vis = 0.

Workload shapes follow the paper's captures (Sec. 5.1: 13-27 fixed views,
640x360 to 2704x2028 frames, 1-8 frame clips).  Two presets:

* ``tiny``: 2,000 Gaussians in the unit cube, 4 cameras at 128x128, one rigid
  motion (rotation <= 20 deg, translation <= 0.1), noise 0.3 px.
* ``capture``: 200,000 Gaussians in a 4-unit box, 18 cameras at 1352x1014 on a
  hemisphere (half the 2704x2028 frames of the paper's 18-view captures),
  piecewise-rigid motion over 8 k-means clusters (rotation <= 30 deg,
  translation <= 0.15 of the box), noise 0.5 px.

Both accept ``n`` and ``views`` overrides for smaller cases of the same shape.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = ["Scene", "make_scene", "PRESETS", "look_at", "motion_pair"]


@dataclass
class Scene:
    """One frame pair: frame-0 Gaussians, cameras, ground-truth motion, tracks."""

    name: str
    seed: int
    extent: float                 # side of the box the means are drawn in
    means_opacity: np.ndarray     # [N,4] f32: x, y, z, opacity in (0,1)
    quats: np.ndarray             # [N,4] f32: w, x, y, z (unit)
    scales: np.ndarray            # [N,4] f32: sx, sy, sz (linear, > 0), 0
    sh_degree: int
    sh: np.ndarray                # [N,(d+1)^2,3] f32 colour coefficients
    width: np.ndarray             # [V] i32
    height: np.ndarray            # [V] i32
    fx: np.ndarray                # [V] f32
    fy: np.ndarray
    cx: np.ndarray
    cy: np.ndarray
    R: np.ndarray                 # [V,3,3] f32 world -> camera rotation
    t: np.ndarray                 # [V,3] f32 world -> camera translation
    labels: np.ndarray            # [N] i32 motion cluster of each Gaussian
    motion_R: np.ndarray          # [K,3,3] f64 rotation of each cluster
    motion_c: np.ndarray          # [K,3] f64 rotation centre
    motion_t: np.ndarray          # [K,3] f64 translation
    disp: list = field(default_factory=list)   # V x [H,W,2] f32 tracked x' - x (px)
    vis: list = field(default_factory=list)    # V x [H,W] u8 1 = tracked/visible
    noise_px: float = 0.0

    @property
    def n(self) -> int:
        return int(self.means_opacity.shape[0])

    @property
    def num_views(self) -> int:
        return int(self.width.shape[0])

    def gt_means(self) -> np.ndarray:
        """Ground-truth moved means (f64) under each Gaussian's rigid motion."""
        X = self.means_opacity[:, :3].astype(np.float64)
        lab = self.labels
        c = self.motion_c[lab]
        return np.einsum("nij,nj->ni", self.motion_R[lab], X - c) + c + self.motion_t[lab]

    def subset_views(self, idx) -> "Scene":
        """The same scene restricted to some views (tracks included)."""
        idx = list(idx)
        s = Scene(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        for k in ("width", "height", "fx", "fy", "cx", "cy", "R", "t"):
            setattr(s, k, getattr(self, k)[idx].copy())
        s.disp = [self.disp[i] for i in idx] if self.disp else []
        s.vis = [self.vis[i] for i in idx] if self.vis else []
        return s


PRESETS = {
    "tiny": dict(n=2000, box=1.0, logs_mu=-4.0, logs_sd=0.5, opacity="sigmoid",
                 sh_degree=0, views=4, rig="ring", radius=3.0, W=128, H=128, f=128.0,
                 clusters=1, max_deg=20.0, max_trans=0.1, noise=0.3),
    "capture": dict(n=200_000, box=4.0, logs_mu=-5.0, logs_sd=0.7, opacity="beta22",
                    sh_degree=3, views=18, rig="hemisphere", radius=4.0, W=1352, H=1014,
                    f=1000.0, clusters=8, max_deg=30.0, max_trans=0.6, noise=0.5),
    # one frame of a batch: the capture scene's Gaussians and rig, the tiny preset's
    # motion (one rigid transform, <= 20 deg, translation <= 0.1 of the box)
    "frame": dict(n=200_000, box=4.0, logs_mu=-5.0, logs_sd=0.7, opacity="beta22",
                  sh_degree=3, views=18, rig="hemisphere", radius=4.0, W=1352, H=1014,
                  f=1000.0, clusters=1, max_deg=20.0, max_trans=0.4, noise=0.5),
}


def look_at(pos, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)):
    """World->camera (R, t) for a camera at ``pos`` looking at ``target``.

    Camera axes: +z forward, +x right, +y down in the image.
    """
    pos = np.asarray(pos, np.float64)
    f = np.asarray(target, np.float64) - pos
    f /= np.linalg.norm(f)
    x = np.cross(f, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    return R, -R @ pos


def _ring_positions(v, radius, elev_deg=30.0):
    # Equally spaced azimuths on a ring raised 30 deg above the equator.  Opposite
    # cameras then look along distinct directions, so the 6-unknown covariance fit
    # is not rank-deficient (it would be for a ring in the plane of the target).
    e = math.radians(elev_deg)
    return [radius * np.array([math.cos(e) * math.cos(2 * math.pi * k / v),
                               math.cos(e) * math.sin(2 * math.pi * k / v),
                               math.sin(e)]) for k in range(v)]


def _hemisphere_positions(v, radius):
    # Fibonacci points on the upper hemisphere, height fraction in [0.1, 1).
    golden = math.pi * (3.0 - math.sqrt(5.0))
    out = []
    for k in range(v):
        z = 0.1 + 0.9 * (k + 0.5) / v
        r = math.sqrt(max(0.0, 1.0 - z * z))
        out.append(radius * np.array([r * math.cos(golden * k), r * math.sin(golden * k), z]))
    return out


def _rodrigues(axis, ang):
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)


def _kmeans(rng, X, k, iters=20):
    """k-means++ seeding from ``rng`` followed by Lloyd iterations."""
    n = X.shape[0]
    sub = X if n <= 50_000 else X[rng.choice(n, 50_000, replace=False)]
    cent = [sub[rng.integers(sub.shape[0])]]
    d2 = ((sub - cent[0]) ** 2).sum(1)
    for _ in range(1, k):
        p = d2 / d2.sum()
        cent.append(sub[rng.choice(sub.shape[0], p=p)])
        d2 = np.minimum(d2, ((sub - cent[-1]) ** 2).sum(1))
    C = np.array(cent)
    for _ in range(iters):
        lab = np.argmin(((X[:, None, :] - C[None]) ** 2).sum(2), axis=1)
        for j in range(k):
            m = lab == j
            if m.any():
                C[j] = X[m].mean(0)
    lab = np.argmin(((X[:, None, :] - C[None]) ** 2).sum(2), axis=1)
    return lab.astype(np.int32), C


def make_scene(preset: str = "tiny", seed: int = 1, n: int | None = None,
               views: int | None = None, width: int | None = None,
               height: int | None = None, focal: float | None = None,
               noise: float | None = None, tracks: bool = True) -> Scene:
    """Draw one frame pair of the given preset (see the module docstring)."""
    p = dict(PRESETS[preset])
    if n is not None:
        p["n"] = n
    if views is not None:
        p["views"] = views
    if width is not None:
        p["W"] = width
    if height is not None:
        p["H"] = height
    if focal is not None:
        p["f"] = focal
    if noise is not None:
        p["noise"] = noise
    rng = np.random.default_rng(seed)
    N, V = p["n"], p["views"]
    box = p["box"]

    means = rng.uniform(-box / 2, box / 2, size=(N, 3))
    logs = rng.normal(p["logs_mu"], p["logs_sd"], size=(N, 3))
    q = rng.normal(size=(N, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    if p["opacity"] == "sigmoid":
        op = 1.0 / (1.0 + np.exp(-rng.normal(size=N)))
    else:
        op = rng.beta(2.0, 2.0, size=N)
    op = np.clip(op, 1e-4, 1.0 - 1e-4)
    d = p["sh_degree"]
    if d == 0:
        # RGB ~ U[0,1] given directly: coefficient = (rgb - 0.5) / Y00.
        rgb = rng.uniform(0.0, 1.0, size=(N, 1, 3))
        sh = (rgb - 0.5) / (0.5 / math.sqrt(math.pi))
    else:
        sh = rng.normal(0.0, 0.2, size=(N, (d + 1) ** 2, 3))

    mo = np.zeros((N, 4), np.float32)
    mo[:, :3] = means
    mo[:, 3] = op
    sc = np.zeros((N, 4), np.float32)
    sc[:, :3] = np.exp(logs)

    if p["rig"] == "ring":
        pos = _ring_positions(V, p["radius"])
    else:
        pos = _hemisphere_positions(V, p["radius"])
    Rs, ts = zip(*[look_at(x) for x in pos]) if V > 0 else ((), ())
    W, H, f = p["W"], p["H"], p["f"]

    k = p["clusters"]
    if k == 1 or N < k:
        k = 1
        labels = np.zeros(N, np.int32)
        centres = np.zeros((1, 3))
    else:
        labels, centres = _kmeans(rng, means, k)
    mR, mt = [], []
    for _ in range(k):
        axis = rng.normal(size=3)
        ang = math.radians(rng.uniform(0.0, p["max_deg"]))
        mR.append(_rodrigues(axis, ang))
        dirn = rng.normal(size=3)
        mt.append(dirn / np.linalg.norm(dirn) * rng.uniform(0.0, p["max_trans"]))

    s = Scene(name=preset, seed=seed, extent=box,
              means_opacity=mo, quats=q.astype(np.float32), scales=sc,
              sh_degree=d, sh=sh.astype(np.float32),
              width=np.full(V, W, np.int32), height=np.full(V, H, np.int32),
              fx=np.full(V, f, np.float32), fy=np.full(V, f, np.float32),
              cx=np.full(V, W / 2, np.float32), cy=np.full(V, H / 2, np.float32),
              R=np.array(Rs, np.float32).reshape(V, 3, 3), t=np.array(ts, np.float32).reshape(V, 3),
              labels=labels, motion_R=np.array(mR), motion_c=centres,
              motion_t=np.array(mt), noise_px=p["noise"])
    if tracks:
        trng = np.random.default_rng([seed, 7919])
        for v in range(V):
            dv, vv = _view_tracks(s, v, trng)
            s.disp.append(dv)
            s.vis.append(vv)
    return s


def _disc_offsets(r):
    o = np.arange(-r, r + 1)
    dx, dy = np.meshgrid(o, o)
    m = dx * dx + dy * dy <= r * r
    return dx[m].astype(np.int64), dy[m].astype(np.int64)


def _view_tracks(s: Scene, v: int, rng) -> tuple[np.ndarray, np.ndarray]:
    W, H = int(s.width[v]), int(s.height[v])
    fx, fy, cx, cy = (float(a[v]) for a in (s.fx, s.fy, s.cx, s.cy))
    R = s.R[v].astype(np.float64)
    t = s.t[v].astype(np.float64)
    X = s.means_opacity[:, :3].astype(np.float64)
    P = X @ R.T + t
    z = P[:, 2]
    ok = z > 0.2
    zs = np.where(ok, z, 1.0)
    u = fx * P[:, 0] / zs + cx
    w = fy * P[:, 1] / zs + cy
    smax = s.scales[:, :3].max(1).astype(np.float64)
    rad = np.clip(np.ceil(1.5 * smax * fx / zs), 1, 48).astype(np.int64)
    ok &= (u + rad >= 0) & (u - rad < W) & (w + rad >= 0) & (w - rad < H)

    empty = np.iinfo(np.uint64).max
    zbuf = np.full(H * W, empty, np.uint64)
    key = (z.astype(np.float32).view(np.uint32).astype(np.uint64) << np.uint64(32)) | \
        np.arange(s.n, dtype=np.uint64)
    ui = np.floor(u).astype(np.int64)
    wi = np.floor(w).astype(np.int64)
    for r in np.unique(rad[ok]):
        ids = np.nonzero(ok & (rad == r))[0]
        ox, oy = _disc_offsets(int(r))
        step = max(1, 8_000_000 // ox.size)
        for a in range(0, ids.size, step):
            b = ids[a:a + step]
            px = ui[b, None] + ox[None, :]
            py = wi[b, None] + oy[None, :]
            inb = (px >= 0) & (px < W) & (py >= 0) & (py < H)
            kk = np.broadcast_to(key[b, None], px.shape)
            np.minimum.at(zbuf, (py * W + px)[inb], kk[inb])

    noise = rng.normal(0.0, s.noise_px, size=(H * W, 2))
    hit = zbuf != empty
    g = (zbuf[hit] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    pix = np.nonzero(hit)[0]
    pxc = (pix % W).astype(np.float64) + 0.5
    pyc = (pix // W).astype(np.float64) + 0.5
    depth = z[g]
    Pc = np.stack([(pxc - cx) / fx * depth, (pyc - cy) / fy * depth, depth], 1)
    Xw = (Pc - t) @ R                       # R^T (Pc - t), row form
    lab = s.labels[g]
    c = s.motion_c[lab]
    Xm = np.einsum("nij,nj->ni", s.motion_R[lab], Xw - c) + c + s.motion_t[lab]
    Pm = Xm @ R.T + t
    front = Pm[:, 2] > 0.2
    zm = np.where(front, Pm[:, 2], 1.0)
    du = fx * Pm[:, 0] / zm + cx - pxc
    dv = fy * Pm[:, 1] / zm + cy - pyc
    disp = noise.copy()
    disp[pix[front], 0] += du[front]
    disp[pix[front], 1] += dv[front]
    vis = np.zeros(H * W, np.uint8)
    vis[pix[front]] = 1
    return disp.astype(np.float32).reshape(H, W, 2), vis.reshape(H, W)


def motion_pair(n: int, views: int = 4, seed: int = 0, extent: float = 4.0, p_pos: float = 0.85,
                p_cov: float = 0.6, p_static: float = 0.15, outliers: float = 0.05, max_rot: float = 0.2,
                lattice: bool = False):
    """Inputs of the motion regularization (Sec. 4.5) without running a fit.

    First-frame Gaussians (``lattice``: on an integer grid scaled by ``extent``/side,
    so that many neighbour distances tie; else a mix of a uniform box and dense
    blobs, with a few exact duplicates), a motion per Gaussian (a smooth field
    plus noise, ``outliers`` of them thrown far, rotations up to ``max_rot``
    radians, scale changes of a few per cent), fit status bits (position solved
    with probability ``p_pos``, covariance with ``p_cov``), and per-view pixel
    counters [views, n] (pixels, static pixels) in which about ``p_static`` of
    the Gaussians are static in most views and some sit exactly on the rule's
    thresholds.  Returns dict(before=(mo, q, s), after=(mo, q, s), status,
    npix, nstat), all float32 except status (uint32)."""
    rng = np.random.default_rng(seed)
    if lattice:
        side = max(2, int(round(n ** (1.0 / 3.0))) + 1)
        grid = np.stack(np.meshgrid(*[np.arange(side)] * 3, indexing="ij"), -1).reshape(-1, 3)
        X = grid[rng.permutation(grid.shape[0])[:n]] * (extent / side)
    else:
        nb = n // 2
        X = rng.uniform(-0.5 * extent, 0.5 * extent, (n, 3))
        centres = rng.uniform(-0.4 * extent, 0.4 * extent, (8, 3))
        X[:nb] = centres[rng.integers(0, 8, nb)] + rng.normal(0, 0.03 * extent, (nb, 3))
        dup = rng.integers(0, n, max(1, n // 200))
        X[rng.integers(0, n, dup.shape[0])] = X[dup]
    mo = np.empty((n, 4), np.float32)
    mo[:, :3] = X
    mo[:, 3] = rng.uniform(0.05, 0.99, n)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    s = np.zeros((n, 4), np.float32)
    s[:, :3] = np.exp(rng.normal(-4.0, 0.5, (n, 3)))
    # motion: a smooth field plus noise
    field_t = 0.02 * extent * np.sin(X[:, [1, 2, 0]] * (2.0 / extent))
    dmu = field_t + rng.normal(0, 0.002 * extent, (n, 3))
    far = rng.random(n) < outliers
    dmu[far] += rng.normal(0, 0.2 * extent, (int(far.sum()), 3))
    axis = rng.normal(size=(n, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    ang = rng.uniform(0, max_rot, n)
    dq = np.concatenate([np.cos(ang / 2)[:, None], np.sin(ang / 2)[:, None] * axis], 1)
    w1, v1 = dq[:, :1], dq[:, 1:]
    w2, v2 = q[:, :1], q[:, 1:]
    q1 = np.concatenate([w1 * w2 - (v1 * v2).sum(1, keepdims=True),
                         w1 * v2 + w2 * v1 + np.cross(v1, v2)], 1)       # dq * q
    mo1 = mo.copy()
    mo1[:, :3] = X + dmu
    s1 = s.copy()
    s1[:, :3] = s[:, :3] * rng.uniform(0.95, 1.05, (n, 3))
    status = np.zeros(n, np.uint32)
    status[rng.random(n) < p_pos] |= 1
    status[rng.random(n) < p_cov] |= 2
    # pixel counters: integers, a static group, and rows on the thresholds
    npix = rng.integers(0, 40, (views, n)).astype(np.float32)
    frac = rng.uniform(0, 1, (views, n))
    stat_g = rng.random(n) < p_static
    frac[:, stat_g] = rng.uniform(0.9, 1.0, (views, int(stat_g.sum())))
    nstat = np.floor(npix * frac).astype(np.float32)
    edge = rng.random((views, n)) < 0.05
    npix[edge] = 10.0
    nstat[edge] = 9.0                                                   # 9 > 0.9 * 10 is false in FP32
    edge2 = rng.random((views, n)) < 0.03
    npix[edge2] = 9.0                                                   # not more than 9 pixels
    nstat[edge2] = 9.0
    return dict(before=(mo, q.astype(np.float32), s), after=(mo1, q1.astype(np.float32), s1),
                status=status, npix=npix, nstat=nstat)


def point_set(kind: str, n: int, rng) -> np.ndarray:
    """Point sets for the neighbour search (float32 [n, 4]: x, y, z, 0.5), drawn
    from the numpy Generator ``rng``: "uniform" (a 4-unit box), "clustered" (six
    tight clusters and a sparse far field), "lattice" (an integer grid, many
    distance ties), "flat" (a plane), "duplicates" (exact repeats), "offset" (far
    from the origin), "spheres_far" (20 sphere surfaces and 5 % far floaters),
    "blobs" (20 tight Gaussian blobs)."""
    mo = np.zeros((n, 4), np.float32)
    if kind == "uniform":
        mo[:, :3] = rng.uniform(-2, 2, (n, 3))
    elif kind == "clustered":
        c = rng.uniform(-2, 2, (6, 3))
        mo[:, :3] = c[rng.integers(0, 6, n)] + rng.normal(0, 0.02, (n, 3))
        mo[: n // 10, :3] = rng.uniform(-20, 20, (n // 10, 3))        # a sparse far field
    elif kind == "lattice":
        side = int(np.ceil(n ** (1 / 3))) + 1
        g = np.stack(np.meshgrid(*[np.arange(side)] * 3, indexing="ij"), -1).reshape(-1, 3)
        mo[:, :3] = g[rng.permutation(len(g))[:n]] * 0.25
    elif kind == "flat":
        mo[:, :2] = rng.uniform(-1, 1, (n, 2))
        mo[:, 2] = 0.5
    elif kind == "duplicates":
        base = rng.uniform(-1, 1, (max(1, n // 4), 3))
        mo[:, :3] = base[rng.integers(0, len(base), n)]
    elif kind == "offset":                                            # far from the origin
        mo[:, :3] = 1000.0 + rng.uniform(0, 1, (n, 3))
    elif kind in ("spheres_far", "blobs"):
        c = rng.uniform(-2, 2, (20, 3))
        if kind == "blobs":
            mo[:, :3] = c[rng.integers(0, 20, n)] + rng.normal(0, 0.02, (n, 3))
        else:                                                         # surfaces and floaters
            d = rng.normal(size=(n, 3))
            d /= np.linalg.norm(d, axis=1, keepdims=True)
            mo[:, :3] = c[rng.integers(0, 20, n)] + 0.3 * d
            mo[: n // 20, :3] = rng.uniform(-20, 20, (n // 20, 3))
    mo[:, 3] = 0.5
    return mo

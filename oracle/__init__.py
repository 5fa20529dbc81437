"""FP64 CPU oracle of the TrackerSplat motion-compensation path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product path.  The C source
``oracle.c`` states, function by function, which passage of the paper it follows.
It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# Per-view flags and per-Gaussian status bits.
OV_OK, OV_FEW_PX, OV_LOW_ALPHA, OV_SINGULAR, OV_CULLED = 1, 2, 4, 8, 16
OS_POS_OK, OS_COV_OK, OS_NEG_EIG, OS_FEW_VIEWS = 1, 2, 4, 8
OS_LOW_ALPHA, OS_FEW_PX, OS_COV_SINGULAR, OS_TRI_SINGULAR = 16, 32, 64, 128


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, FP contraction off, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("R", C.c_float * 9), ("t", C.c_float * 3)]


class Options(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("det_min", C.c_double),
                ("sumw_min_view", C.c_double), ("min_px_view", C.c_int32),
                ("lam_min_px2", C.c_double), ("min_views", C.c_int32),
                ("sumw_min_total", C.c_double), ("min_px_total", C.c_int32),
                ("cov_rcond_min", C.c_double)]


class Tracks(C.Structure):
    _fields_ = [("disp", C.c_void_p), ("vis", C.c_void_p)]


_OUT_FIELDS = ["moments", "mean2d", "cov2d", "view_flags", "view_affine", "view_mean2d",
               "view_cov2d", "out_mean", "out_quat", "out_scale", "out_cov3d", "out_status"]


class Outputs(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in _OUT_FIELDS]


def default_options(tile=(16, 16)) -> Options:
    """Sec. 5.1 thresholds plus the two added guards (lambda_min, covariance rcond)."""
    return Options(tile[0], tile[1], 1e-12, 1e-3, 2, 1e-4, 2, 1e-3, 3, 1e-6)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.orc_keys.argtypes = [C.c_int, C.c_int, P, P, P, P, C.c_int, C.c_int, P, P, P, P]
        _lib.orc_count_pairs.argtypes = [C.c_int, C.c_int, P, P, P, P, C.c_int, C.c_int]
        _lib.orc_count_pairs.restype = C.c_int64
        _lib.orc_bin.argtypes = [C.c_int, C.c_int, P, P, P, P, C.c_int, C.c_int, P, P]
        _lib.orc_fit_motion.argtypes = [C.c_int, C.c_int, P, P, P, P, P, P, P, C.c_int, P]
        _lib.orc_render.argtypes = [C.c_int, C.c_int, P, P, P, P, C.c_int, P, C.c_int, C.c_int,
                                    P, P, P]
        _lib.orc_render_bruteforce.argtypes = [C.c_int, P, P, P, P, C.c_int, P, C.c_int, C.c_int,
                                               C.c_int, P, P]
        _lib.orc_render_grad.argtypes = [C.c_int, C.c_int, P, P, P, P, C.c_int, P, C.c_int, C.c_int,
                                         P, P, P, P, P, P, P]
        _lib.orc_static_flags.argtypes = [C.c_int, C.c_int, P, P, C.c_float, C.c_float, C.c_int, P]
        _lib.orc_knn.argtypes = [C.c_int, P, P, C.c_int, P]
        _lib.orc_regularize.argtypes = [C.c_int, P, P, P, P, P, P, P, P, C.c_int, P, P, P, P]
        _lib.orc_naive_ls.argtypes = [C.c_int, P, P, P, P]
        _lib.orc_project.argtypes = [P, P, P, P, P, P, P]
        _lib.orc_eig3.argtypes = [P, P, P]
        _lib.orc_lstsq.argtypes = [C.c_int, C.c_int, P, P, P]
        _lib.orc_lstsq.restype = C.c_double
        _lib.orc_view_solve.argtypes = [P, P, P, P, P, P, P, P]
        _lib.orc_multiview.argtypes = [C.c_int, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
        _lib.orc_sh_basis.argtypes = [C.c_double, C.c_double, C.c_double, P]
        _lib.orc_max_threads.restype = C.c_int
        _lib.orc_set_threads.argtypes = [C.c_int]
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def cameras(scene) -> "C.Array":
    V = scene.num_views
    arr = (Camera * max(V, 1))()
    for v in range(V):
        c = arr[v]
        c.width, c.height = int(scene.width[v]), int(scene.height[v])
        c.fx, c.fy, c.cx, c.cy = (float(a[v]) for a in (scene.fx, scene.fy, scene.cx, scene.cy))
        c.R[:] = [float(x) for x in np.asarray(scene.R[v], np.float32).ravel()]
        c.t[:] = [float(x) for x in np.asarray(scene.t[v], np.float32).ravel()]
    return arr


def _gauss(scene):
    mo = np.ascontiguousarray(scene.means_opacity, np.float32)
    q = np.ascontiguousarray(scene.quats, np.float32)
    s = np.ascontiguousarray(scene.scales, np.float32)
    return mo, q, s


def keys(scene, tile=(16, 16)) -> dict:
    """Key path per (view, Gaussian): visible, depth bits, tile rect, tiles touched."""
    mo, q, s = _gauss(scene)
    n, V = scene.n, scene.num_views
    out = dict(visible=np.zeros((V, n), np.int32), depth_bits=np.zeros((V, n), np.uint32),
               rect=np.zeros((V, n, 4), np.int32), tiles_touched=np.zeros((V, n), np.uint32))
    lib().orc_keys(n, V, _ptr(mo), _ptr(q), _ptr(s), C.cast(cameras(scene), C.c_void_p),
                   tile[0], tile[1], _ptr(out["visible"]), _ptr(out["depth_bits"]),
                   _ptr(out["rect"]), _ptr(out["tiles_touched"]))
    return out


def bin_lists(scene, tile=(16, 16)):
    """Per-tile lists: (offsets [NT+1] i64, entries [K] u64 = depth_bits << 32 | g)."""
    mo, q, s = _gauss(scene)
    n, V = scene.n, scene.num_views
    cams = cameras(scene)
    K = lib().orc_count_pairs(n, V, _ptr(mo), _ptr(q), _ptr(s), C.cast(cams, C.c_void_p),
                              tile[0], tile[1])
    NT = sum(((int(scene.width[v]) + tile[0] - 1) // tile[0]) *
             ((int(scene.height[v]) + tile[1] - 1) // tile[1]) for v in range(V))
    offsets = np.zeros(NT + 1, np.int64)
    entries = np.zeros(max(K, 1), np.uint64)
    lib().orc_bin(n, V, _ptr(mo), _ptr(q), _ptr(s), C.cast(cams, C.c_void_p), tile[0], tile[1],
                  _ptr(offsets), _ptr(entries))
    return offsets, entries[:K]


def fit_motion(scene, options: Options | None = None, sample=None, per_view=True) -> dict:
    """Run the whole path.  ``sample``: optional Gaussian ids to fit (others untouched)."""
    opt = options or default_options()
    mo, q, s = _gauss(scene)
    n, V = scene.n, scene.num_views
    tr = (Tracks * max(V, 1))()
    keep = []
    for v in range(V):
        d = np.ascontiguousarray(scene.disp[v], np.float32)
        m = np.ascontiguousarray(scene.vis[v], np.uint8)
        keep += [d, m]
        tr[v].disp, tr[v].vis = d.ctypes.data, m.ctypes.data
    res = {}
    if per_view:
        res.update(moments=np.zeros((V, n, 18)), mean2d=np.zeros((V, n, 2)),
                   cov2d=np.zeros((V, n, 3)), view_flags=np.zeros((V, n), np.uint32),
                   view_affine=np.zeros((V, n, 6)), view_mean2d=np.zeros((V, n, 2)),
                   view_cov2d=np.zeros((V, n, 3)))
    res.update(out_mean=np.zeros((n, 3)), out_quat=np.zeros((n, 4)), out_scale=np.zeros((n, 3)),
               out_cov3d=np.zeros((n, 6)), out_status=np.zeros(n, np.uint32))
    o = Outputs(**{k: (res[k].ctypes.data if k in res else None) for k in _OUT_FIELDS})
    smp = None if sample is None else np.ascontiguousarray(sample, np.int32)
    t0 = time.perf_counter()
    nthreads = lib().orc_fit_motion(n, V, _ptr(mo), _ptr(q), _ptr(s),
                                    C.cast(cameras(scene), C.c_void_p), C.cast(tr, C.c_void_p),
                                    C.byref(opt), _ptr(smp), 0 if smp is None else smp.size,
                                    C.byref(o))
    res["seconds"] = time.perf_counter() - t0
    res["threads"] = nthreads
    return res


def render(scene, tile=(16, 16)):
    """Colour [V] x [H,W,3], transmittance [V] x [H,W] and threshold-window flags."""
    mo, q, s = _gauss(scene)
    n, V = scene.n, scene.num_views
    rgb = [np.zeros((int(scene.height[v]), int(scene.width[v]), 3), np.float32) for v in range(V)]
    T = [np.zeros((int(scene.height[v]), int(scene.width[v])), np.float32) for v in range(V)]
    fl = [np.zeros((int(scene.height[v]), int(scene.width[v])), np.uint8) for v in range(V)]
    pa = (C.c_void_p * max(V, 1))(*[a.ctypes.data for a in rgb])
    pt = (C.c_void_p * max(V, 1))(*[a.ctypes.data for a in T])
    pf = (C.c_void_p * max(V, 1))(*[a.ctypes.data for a in fl])
    sh = np.ascontiguousarray(scene.sh, np.float32)
    lib().orc_render(n, V, _ptr(mo), _ptr(q), _ptr(s), _ptr(sh), int(scene.sh_degree),
                     C.cast(cameras(scene), C.c_void_p), tile[0], tile[1],
                     C.cast(pa, C.c_void_p), C.cast(pt, C.c_void_p), C.cast(pf, C.c_void_p))
    return rgb, T, fl


def render_grad(scene, W, tile=(16, 16), gradient=True):
    """L = sum over views, pixels and channels of W[v] * colour (float32 weights
    [V] x [H,W,3]) and, with gradient=True, dL/d(means [n,3], linear scales [n,3],
    raw quaternions [n,4], opacity [n], colour coefficients [n, (deg+1)^2, 3]),
    in FP64 with the blend's decisions held fixed."""
    mo, q, s = _gauss(scene)
    n, V = scene.n, scene.num_views
    nb = (int(scene.sh_degree) + 1) ** 2
    Ws = [np.ascontiguousarray(w, np.float32) for w in W]
    pw = (C.c_void_p * max(V, 1))(*[w.ctypes.data for w in Ws])
    sh = np.ascontiguousarray(scene.sh, np.float32)
    loss = np.zeros(1)
    out = dict(means=np.zeros((n, 3)), scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               opacity=np.zeros(n), sh=np.zeros((n, nb, 3))) if gradient else None
    g = (lambda k: _ptr(out[k])) if gradient else (lambda k: None)
    lib().orc_render_grad(n, V, _ptr(mo), _ptr(q), _ptr(s), _ptr(sh), int(scene.sh_degree),
                          C.cast(cameras(scene), C.c_void_p), tile[0], tile[1], C.cast(pw, C.c_void_p),
                          _ptr(loss), g("means"), g("scales"), g("quats"), g("opacity"), g("sh"))
    if not gradient:
        return float(loss[0])
    out["loss"] = float(loss[0])
    return out


def render_bruteforce(scene, view: int, use_rect: bool, tile=(16, 16)):
    mo, q, s = _gauss(scene)
    H, W = int(scene.height[view]), int(scene.width[view])
    rgb = np.zeros((H, W, 3), np.float32)
    T = np.zeros((H, W), np.float32)
    cams = cameras(scene)
    sh = np.ascontiguousarray(scene.sh, np.float32)
    lib().orc_render_bruteforce(scene.n, _ptr(mo), _ptr(q), _ptr(s), _ptr(sh), int(scene.sh_degree),
                                C.cast(C.byref(cams[view]), C.c_void_p), tile[0], tile[1],
                                int(use_rect), _ptr(rgb), _ptr(T))
    return rgb, T


def naive_ls(x, xp, w=None):
    """Eq. 3 with explicit X and Y (Householder QR); returns A (2x2), b (2)."""
    x = np.ascontiguousarray(x, np.float64)
    xp = np.ascontiguousarray(xp, np.float64)
    wv = None if w is None else np.ascontiguousarray(w, np.float64)
    out = np.zeros(6)
    ok = lib().orc_naive_ls(x.shape[0], _ptr(x), _ptr(xp), _ptr(wv), _ptr(out))
    if not ok:
        raise ValueError("singular")
    return out[:4].reshape(2, 2), out[4:]


def project(mo, q, s, cam: Camera):
    m2 = np.zeros(2)
    c2 = np.zeros(3)
    cn = np.zeros(3)
    lib().orc_project(_ptr(np.ascontiguousarray(mo, np.float32)),
                      _ptr(np.ascontiguousarray(q, np.float32)),
                      _ptr(np.ascontiguousarray(s, np.float32)), C.cast(C.byref(cam), C.c_void_p),
                      _ptr(m2), _ptr(c2), _ptr(cn))
    return m2, c2, cn


def eig3(S):
    S = np.ascontiguousarray(S, np.float64)
    lam = np.zeros(3)
    E = np.zeros((3, 3))
    lib().orc_eig3(_ptr(S), _ptr(lam), _ptr(E))
    return lam, E


def lstsq(A, b):
    A = np.ascontiguousarray(A, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros(A.shape[1])
    rc = lib().orc_lstsq(A.shape[0], A.shape[1], _ptr(A), _ptr(b), _ptr(x))
    return x, rc


def view_solve(mom16, mean2d, cov2d, options: Options | None = None):
    """Per-view solve of one moment record -> (flags, affine[6], mean2d', cov2d')."""
    opt = options or default_options()
    m = np.ascontiguousarray(mom16, np.float64)
    mu = np.ascontiguousarray(mean2d, np.float64)
    cv = np.ascontiguousarray(cov2d, np.float64)
    fl = np.zeros(1, np.uint32)
    aff, mn, cn = np.zeros(6), np.zeros(2), np.zeros(3)
    lib().orc_view_solve(_ptr(m), _ptr(mu), _ptr(cv), C.byref(opt), _ptr(fl), _ptr(aff),
                         _ptr(mn), _ptr(cn))
    return int(fl[0]), aff, mn, cn


def multiview(scene, g, flags, sumw, npix, mean2d_new, cov2d_new, options: Options | None = None):
    """Multi-view update of Gaussian ``g`` of ``scene`` from given per-view results."""
    opt = options or default_options()
    V = scene.num_views
    mo, q, s = _gauss(scene)
    fl = np.ascontiguousarray(flags, np.uint32)
    sw = np.ascontiguousarray(sumw, np.float64)
    npx = np.ascontiguousarray(npix, np.float64)
    mn = np.ascontiguousarray(mean2d_new, np.float64)
    cn = np.ascontiguousarray(cov2d_new, np.float64)
    mean, quat, scale, cov = np.zeros(3), np.zeros(4), np.zeros(3), np.zeros(6)
    st = np.zeros(1, np.uint32)
    mog, qg, sg = (np.ascontiguousarray(a[g]) for a in (mo, q, s))
    lib().orc_multiview(V, C.cast(cameras(scene), C.c_void_p), _ptr(fl), _ptr(sw), _ptr(npx),
                        _ptr(mn), _ptr(cn), _ptr(mog), _ptr(qg), _ptr(sg), C.byref(opt),
                        _ptr(mean), _ptr(quat), _ptr(scale), _ptr(cov), _ptr(st))
    return dict(mean=mean, quat=quat, scale=scale, cov3d=cov, status=int(st[0]))


def sh_basis(d):
    """The 16 colour basis functions at the unit direction d."""
    Y = np.zeros(16)
    lib().orc_sh_basis(float(d[0]), float(d[1]), float(d[2]), _ptr(Y))
    return Y


def max_threads() -> int:
    return int(lib().orc_max_threads())


def set_threads(n: int) -> None:
    """Threads the oracle's parallel regions use from now on (<= 0: the default)."""
    lib().orc_set_threads(int(n))


REG_STATIC, REG_POS_MEDIAN, REG_POS_PROPAGATED, REG_COV_MEDIAN, REG_COV_PROPAGATED = 1, 2, 4, 8, 16


def static_flags(npix, nstat, min_px=9.0, frac=0.9, min_views=2):
    """Sec. 4.5.2 static Gaussians from per-view pixel counts [V, n] (float)."""
    npix = np.ascontiguousarray(npix, np.float32)
    nstat = np.ascontiguousarray(nstat, np.float32)
    V, n = npix.shape
    out = np.zeros(n, np.uint8)
    lib().orc_static_flags(n, V, _ptr(npix), _ptr(nstat), float(min_px), float(frac), int(min_views), _ptr(out))
    return out


def knn(means_opacity, mask, k=8):
    """The k nearest members of mask (other than the point) of every point, by
    FP32 squared distance then index; -1 pads."""
    mo = np.ascontiguousarray(means_opacity, np.float32)
    m = np.ascontiguousarray(mask, np.uint8)
    n = mo.shape[0]
    out = np.zeros((n, k), np.int32)
    lib().orc_knn(n, _ptr(mo), _ptr(m), int(k), _ptr(out))
    return out


def regularize(before, after, status, is_static, k=8):
    """Motion regularization (Sec. 4.5): before/after = (means_opacity, quats,
    scales) [n, 4] float32 of the first frame and of the fit; status the fit's
    status bits.  Returns dict(means_opacity, quats, scales, flags)."""
    b = [np.ascontiguousarray(a, np.float32) for a in before]
    a = [np.ascontiguousarray(x, np.float32) for x in after]
    st = np.ascontiguousarray(status, np.uint32)
    stat = np.ascontiguousarray(is_static, np.uint8)
    n = b[0].shape[0]
    mo, q, sc = np.zeros((n, 4), np.float32), np.zeros((n, 4), np.float32), np.zeros((n, 4), np.float32)
    fl = np.zeros(n, np.uint32)
    lib().orc_regularize(n, _ptr(b[0]), _ptr(b[1]), _ptr(b[2]), _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(st),
                         _ptr(stat), int(k), _ptr(mo), _ptr(q), _ptr(sc), _ptr(fl))
    return dict(means_opacity=mo, quats=q, scales=sc, flags=fl)

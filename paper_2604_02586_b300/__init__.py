"""Python binding of libtsplat.so, the B300 motion-compensation path of TrackerSplat.

Argument marshalling only: every step runs in the library's CUDA kernels.  The
C functions are exported under their C names (``tsp_create``, ``tsp_fit_motion``,
``tsp_fit_motion_host``, ``tsp_render``, ``tsp_sync``, ``tsp_inspect`` ...) and
wrapped by :class:`Context`, whose methods take torch CUDA tensors (device path)
or numpy arrays (host path).  Loading fails loudly if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = ["Context", "Camera", "Options", "TSP", "lib", "LIB_PATH", "cameras_from"]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtsplat.so")


class TSP:
    """Status codes and flag bits of include/tsplat.h."""
    OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_BUDGET, ERR_OVERFLOW = range(7)
    VIEW_OK, VIEW_FEW_PX, VIEW_LOW_ALPHA, VIEW_SINGULAR, VIEW_CULLED = 1, 2, 4, 8, 16
    POS_OK, COV_OK, NEG_EIG, FEW_VIEWS, LOW_ALPHA, FEW_PX, COV_SINGULAR, TRI_SINGULAR = \
        1, 2, 4, 8, 16, 32, 64, 128
    I_COUNTS, I_RECT, I_DEPTH, I_TILES_TOUCHED, I_TILE_OFFSETS, I_PAIRS, I_MOMENTS, I_STATS, \
        I_VIEW_MEANS, I_VIEW_COV, I_KNN_PATH = range(11)
    STAGES = ("project", "scan", "emit", "tile_sort", "raster", "view_solve", "multiview")
    MAX_VIEWS = 32
    REG_STATIC, REG_POS_MEDIAN, REG_POS_PROPAGATED, REG_COV_MEDIAN, REG_COV_PROPAGATED = 1, 2, 4, 8, 16
    REG_MAX_K = 16


class Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("R", C.c_float * 9), ("t", C.c_float * 3)]


class Gaussians(C.Structure):
    _fields_ = [("n", C.c_int32), ("means_opacity", C.c_void_p), ("quats", C.c_void_p),
                ("scales", C.c_void_p)]


class ViewTracks(C.Structure):
    _fields_ = [("disp", C.c_void_p), ("vis", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("means", C.c_void_p), ("quats", C.c_void_p), ("scales", C.c_void_p),
                ("status", C.c_void_p), ("view_affine", C.c_void_p), ("view_moments", C.c_void_p),
                ("view_flags", C.c_void_p)]


class Frame(C.Structure):
    _fields_ = [("g", Gaussians), ("cams", C.c_void_p), ("num_views", C.c_int32),
                ("tracks", C.c_void_p), ("out", Result)]


class RenderGrads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p), ("sh", C.c_void_p)]


class RegOptions(C.Structure):
    _fields_ = [("k", C.c_int32), ("static_min_px", C.c_float), ("static_frac", C.c_float),
                ("static_min_views", C.c_int32)]


class RegResult(C.Structure):
    _fields_ = [("means_opacity", C.c_void_p), ("quats", C.c_void_p), ("scales", C.c_void_p),
                ("flags", C.c_void_p), ("nbr_pos", C.c_void_p), ("nbr_cov", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("det_min", C.c_float),
                ("sumw_min_view", C.c_float), ("min_px_view", C.c_int32), ("lam_min_px2", C.c_float),
                ("min_views", C.c_int32), ("sumw_min_total", C.c_float), ("min_px_total", C.c_int32),
                ("cov_rcond_min", C.c_float), ("async_pairs", C.c_int32), ("stage_timing", C.c_int32),
                ("collect_stats", C.c_int32), ("raster_variant", C.c_int32),
                ("pair_capacity", C.c_int64), ("budget_bytes", C.c_int64), ("checked", C.c_int32)]


# tsp_alloc_fn / tsp_free_fn
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_int, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_int, C.c_void_p)

_lib = None


def lib():
    """The loaded library (raises if libtsplat.so has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2604_02586_b300.build`")
        L = C.CDLL(LIB_PATH)
        P, I = C.c_void_p, C.c_int
        L.tsp_default_options.argtypes = [P]
        L.tsp_create.argtypes = [I, P, P]
        L.tsp_destroy.argtypes = [P]
        L.tsp_fit_motion.argtypes = [P, P, P, I, P, P, P]
        L.tsp_fit_motion_host.argtypes = [P, P, P, I, P, P, P]
        L.tsp_fit_motion_batch.argtypes = [P, P, I, P]
        L.tsp_autotune.argtypes = [P, P, I, I, P, P, P]
        L.tsp_autotune_cached.argtypes = [P, P, I, I, P, C.c_char_p, P, P, P]
        L.tsp_render.argtypes = [P, P, P, I, P, I, P, P, P]
        L.tsp_render_backward.argtypes = [P, P, P, I, P, I, P, P, P, P]
        L.tsp_default_reg_options.argtypes = [P]
        L.tsp_regularize.argtypes = [P, P, P, P, I, P, P, P]
        L.tsp_knn.argtypes = [P, P, P, I, I, P, P]
        L.tsp_sync.argtypes = [P, P, I]
        L.tsp_inspect.argtypes = [P, I, P, C.c_size_t, P]
        L.tsp_workspace_bytes.argtypes = [P, P]
        L.tsp_stage_times.argtypes = [P, P, I, P]
        L.tsp_set_allocator.argtypes = [P, ALLOC_FN, FREE_FN, P]
        L.tsp_set_budget.argtypes = [P, C.c_int64]
        L.tsp_set_track_gate.argtypes = [P, P, C.c_uint32, C.c_int64]
        L.tsp_sort_tiles_noalloc.argtypes = [P, P, C.c_uint32, C.c_uint32, P]
        L.tsp_sort_tiles_noalloc.restype = I
        L.tsp_status_string.argtypes = [I]
        L.tsp_status_string.restype = C.c_char_p
        L.tsp_last_error.argtypes = [P]
        L.tsp_last_error.restype = C.c_char_p
        L.tsp_version.restype = I
        for name in ("tsp_default_options", "tsp_create", "tsp_destroy", "tsp_fit_motion",
                     "tsp_fit_motion_host", "tsp_fit_motion_batch", "tsp_autotune", "tsp_autotune_cached", "tsp_render",
                     "tsp_render_backward", "tsp_sync", "tsp_inspect", "tsp_default_reg_options",
                     "tsp_regularize", "tsp_knn", "tsp_set_allocator", "tsp_set_budget", "tsp_set_track_gate",
                     "tsp_workspace_bytes", "tsp_stage_times"):
            getattr(L, name).restype = I
        _lib = L
    return _lib


def __getattr__(name):
    if name.startswith("tsp_"):
        return getattr(lib(), name)
    raise AttributeError(name)


class TspError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def cameras_from(width, height, fx, fy, cx, cy, R, t):
    """ctypes array of tsp_camera from per-view arrays."""
    V = len(width)
    arr = (Camera * max(V, 1))()
    for v in range(V):
        c = arr[v]
        c.width, c.height = int(width[v]), int(height[v])
        c.fx, c.fy, c.cx, c.cy = float(fx[v]), float(fy[v]), float(cx[v]), float(cy[v])
        c.R[:] = [float(x) for x in np.asarray(R[v], np.float32).ravel()]
        c.t[:] = [float(x) for x in np.asarray(t[v], np.float32).ravel()]
    return arr, V


def _cams(cams):
    if isinstance(cams, tuple):
        return cams
    return cameras_from(cams.width, cams.height, cams.fx, cams.fy, cams.cx, cams.cy, cams.R, cams.t)


def cameras(cam_set):
    """The (tsp_camera array, view count) pair of a camera set (an object with
    per-view width, height, fx, fy, cx, cy, R, t).  Every call taking ``cams``
    accepts either form; a caller that fits the same views repeatedly builds the
    pair once and saves rebuilding it (~0.13 ms for 18 views) on every call."""
    return _cams(cam_set)


def _dptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _hptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _need(t, shape, dtype, device=None, name="tensor"):
    """Check a torch tensor's shape, dtype, contiguity and device before its
    pointer is handed to the library (the kernels trust these sizes)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if t.dtype != dtype:
        raise ValueError(f"{name} has dtype {t.dtype}, expected {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")


def _need_np(a, shape, name):
    if tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(a.shape)}, expected {tuple(shape)}")


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Context:
    """A libtsplat context on one CUDA device (owns the device workspace)."""

    def __init__(self, device: int = 0, **options):
        self.opt = Options()
        lib().tsp_default_options(C.byref(self.opt))
        for k, v in options.items():
            setattr(self.opt, k, v)
        self.device = device
        self._h = C.c_void_p()
        self._check(lib().tsp_create(device, C.byref(self.opt), C.byref(self._h)), "tsp_create")

    # -- helpers -------------------------------------------------------------
    def _check(self, status, what):
        if status != TSP.OK:
            msg = lib().tsp_last_error(self._h).decode() if self._h else ""
            raise TspError(status, f"{what}: {lib().tsp_status_string(status).decode()}: {msg}")

    def close(self):
        if self._h:
            lib().tsp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def set_allocator(self, alloc=None, free=None):
        """Route the workspace through alloc(bytes, device) -> int device pointer
        (256-byte aligned) or None to refuse, and free(ptr, bytes, device);
        both None restores cudaMalloc / cudaFree (tsp_set_allocator)."""
        if (alloc is None) != (free is None):
            raise ValueError("give both alloc and free, or neither")
        if alloc is None:
            self._alloc_cb = self._free_cb = None
            self._check(lib().tsp_set_allocator(self._h, ALLOC_FN(), FREE_FN(), None), "tsp_set_allocator")
            return
        a = ALLOC_FN(lambda nbytes, device, user: alloc(int(nbytes), int(device)))
        f = FREE_FN(lambda ptr, nbytes, device, user: free(int(ptr), int(nbytes), int(device)))
        self._check(lib().tsp_set_allocator(self._h, a, f, None), "tsp_set_allocator")
        self._alloc_cb, self._free_cb = a, f          # the library keeps calling these

    def set_track_gate(self, flag=None, value: int = 1, timeout_us: int = 1_000_000):
        """Make device-track calls wait on the device until the int32 CUDA tensor
        ``flag`` (one element) reaches ``value``, for at most ``timeout_us``;
        None removes the gate (tsp_set_track_gate)."""
        import torch
        if flag is None:
            self._gate = None
            self._check(lib().tsp_set_track_gate(self._h, None, 0, 0), "tsp_set_track_gate")
            return
        _need(flag, (1,), torch.int32, None, "flag")
        self._check(lib().tsp_set_track_gate(self._h, C.c_void_p(flag.data_ptr()), int(value), int(timeout_us)),
                    "tsp_set_track_gate")
        self._gate = flag                           # the library keeps the pointer

    def set_budget(self, budget_bytes: int):
        """Workspace ceiling in bytes, 0 = unlimited (tsp_set_budget)."""
        self._check(lib().tsp_set_budget(self._h, int(budget_bytes)), "tsp_set_budget")
        self.opt.budget_bytes = int(budget_bytes)

    def __exit__(self, *exc):
        self.close()

    # -- the motion fit --------------------------------------------------------
    def _frame(self, means_opacity, quats, scales, cams, disp, vis, out=None,
               view_affine=False, view_moments=False, view_flags=False):
        """Check one frame's tensors and build its C structures (kept alive by the
        returned tuple: Gaussians, camera array, view count, tracks, Result, out)."""
        import torch
        n = int(means_opacity.shape[0])
        carr, V = _cams(cams)
        dev = means_opacity.device
        if out is None:
            out = dict(means=torch.empty((n, 4), dtype=torch.float32, device=dev),
                       quats=torch.empty((n, 4), dtype=torch.float32, device=dev),
                       scales=torch.empty((n, 4), dtype=torch.float32, device=dev),
                       status=torch.empty((n,), dtype=torch.int32, device=dev))
            if view_affine:
                out["view_affine"] = torch.empty((V, n, 6), dtype=torch.float32, device=dev)
            if view_moments:
                out["view_moments"] = torch.empty((V, n, 16), dtype=torch.float32, device=dev)
            if view_flags:
                out["view_flags"] = torch.empty((V, n), dtype=torch.int32, device=dev)
        f32 = torch.float32
        for name, t in (("means_opacity", means_opacity), ("quats", quats), ("scales", scales)):
            _need(t, (n, 4), f32, dev, name)
        if len(disp) < V or len(vis) < V:
            raise ValueError("need one disp and one vis tensor per camera")
        for v in range(V):
            H, W = carr[v].height, carr[v].width
            _need(disp[v], (H, W, 2), f32, dev, f"disp[{v}]")
            _need(vis[v], (H, W), torch.uint8, dev, f"vis[{v}]")
        shapes = dict(means=((n, 4), f32), quats=((n, 4), f32), scales=((n, 4), f32),
                      status=((n,), torch.int32), view_affine=((V, n, 6), f32),
                      view_moments=((V, n, 16), f32), view_flags=((V, n), torch.int32))
        for k, t in out.items():
            _need(t, shapes[k][0], shapes[k][1], dev, f"out[{k}]")
        g = Gaussians(n, means_opacity.data_ptr(), quats.data_ptr(), scales.data_ptr())
        tr = (ViewTracks * max(V, 1))()
        for v in range(V):
            tr[v].disp, tr[v].vis = disp[v].data_ptr(), vis[v].data_ptr()
        r = Result(*[(out[k].data_ptr() if k in out else None) for k in
                     ("means", "quats", "scales", "status", "view_affine", "view_moments", "view_flags")])
        return g, carr, V, tr, r, out

    def fit_motion(self, means_opacity, quats, scales, cams, disp, vis, *, out=None,
                   view_affine=False, view_moments=False, view_flags=False, stream=None,
                   sync=False):
        """Device path.  Tensors are CUDA tensors on the context's device:
        means_opacity/quats/scales [n,4] f32, disp [V] x [H,W,2] f32, vis [V] x [H,W] u8.
        Returns a dict of output tensors (allocated here unless ``out`` is given)."""
        g, carr, V, tr, r, out = self._frame(means_opacity, quats, scales, cams, disp, vis, out,
                                             view_affine, view_moments, view_flags)
        self._check(lib().tsp_fit_motion(self._h, C.byref(g), carr, V, tr, C.byref(r),
                                         _stream_handle(stream)), "tsp_fit_motion")
        if sync:
            self.sync(stream)
        return out

    def fit_motion_batch(self, frames, *, stream=None, sync=False):
        """Several frame pairs in one launch of each step.  ``frames`` is a list of
        dicts with the arguments of fit_motion (means_opacity, quats, scales, cams,
        disp, vis and optionally out, view_affine, view_moments, view_flags).
        Returns the list of per-frame output dicts."""
        keys = ("means_opacity", "quats", "scales", "cams", "disp", "vis")
        prep = [self._frame(*[f[k] for k in keys], f.get("out"), f.get("view_affine", False),
                            f.get("view_moments", False), f.get("view_flags", False)) for f in frames]
        arr = (Frame * max(len(prep), 1))()
        for k, (g, carr, V, tr, r, _) in enumerate(prep):
            arr[k].g = g
            arr[k].cams = C.cast(carr, C.c_void_p)
            arr[k].num_views = V
            arr[k].tracks = C.cast(tr, C.c_void_p)
            arr[k].out = r
        self._check(lib().tsp_fit_motion_batch(self._h, arr, len(prep), _stream_handle(stream)),
                    "tsp_fit_motion_batch")
        if sync:
            self.sync(stream)
        return [p[5] for p in prep]

    # (tile_w, tile_h, raster_variant), in the order of tsp_autotune's candidates
    TUNE_CANDIDATES = ((16, 16, 0), (16, 16, 5), (16, 16, 2), (16, 16, 1), (16, 16, 4), (32, 8, 0), (32, 8, 5))

    def _tune_frames(self, frames):
        keys = ("means_opacity", "quats", "scales", "cams", "disp", "vis")
        prep = [self._frame(*[f[k] for k in keys], f.get("out")) for f in frames]
        arr = (Frame * max(len(prep), 1))()
        for k, (g, carr, V, tr, r, _) in enumerate(prep):
            arr[k].g, arr[k].cams, arr[k].num_views = g, C.cast(carr, C.c_void_p), V
            arr[k].tracks, arr[k].out = C.cast(tr, C.c_void_p), r
        return prep, arr

    def autotune(self, frames, repeats=3, stream=None):
        """Time each candidate (tile shape, raster kernel) on ``frames``
        (fit_motion_batch arguments) by the whole fit and keep the fastest.
        Returns (candidate, {candidate: median ms}), candidates as in
        TUNE_CANDIDATES."""
        prep, arr = self._tune_frames(frames)
        chosen = C.c_int(0)
        ms = (C.c_float * len(self.TUNE_CANDIDATES))()
        self._check(lib().tsp_autotune(self._h, arr, len(prep), int(repeats), _stream_handle(stream),
                                       C.byref(chosen), ms), "tsp_autotune")
        best = self.TUNE_CANDIDATES[chosen.value]
        self.opt.tile_w, self.opt.tile_h, self.opt.raster_variant = best
        return best, dict(zip(self.TUNE_CANDIDATES, [float(x) for x in ms]))

    def autotune_cached(self, frames, cache_path, repeats=3, stream=None):
        """tsp_autotune_cached: the choice for this workload's key from the cache
        file if it holds one, else tuned as ``autotune`` and appended.  Returns
        (candidate, {candidate: median ms, -1 where not timed}, from_cache)."""
        prep, arr = self._tune_frames(frames)
        chosen, hit = C.c_int(0), C.c_int(0)
        ms = (C.c_float * len(self.TUNE_CANDIDATES))()
        self._check(lib().tsp_autotune_cached(self._h, arr, len(prep), int(repeats), _stream_handle(stream),
                                              os.fsencode(cache_path), C.byref(chosen), ms, C.byref(hit)),
                    "tsp_autotune_cached")
        best = self.TUNE_CANDIDATES[chosen.value]
        self.opt.tile_w, self.opt.tile_h, self.opt.raster_variant = best
        return best, dict(zip(self.TUNE_CANDIDATES, [float(x) for x in ms])), bool(hit.value)

    def fit_motion_host(self, means_opacity, quats, scales, cams, disp, vis, out=None, stream=None):
        """Host path: numpy inputs and outputs; copies happen inside the library."""
        n = int(means_opacity.shape[0])
        carr, V = _cams(cams)
        mo = np.ascontiguousarray(means_opacity, np.float32)
        q = np.ascontiguousarray(quats, np.float32)
        s = np.ascontiguousarray(scales, np.float32)
        if out is None:
            out = dict(means=np.empty((n, 4), np.float32), quats=np.empty((n, 4), np.float32),
                       scales=np.empty((n, 4), np.float32), status=np.empty(n, np.uint32))
        for name, a in (("means_opacity", mo), ("quats", q), ("scales", s)):
            _need_np(a, (n, 4), name)
        for k, shp in (("means", (n, 4)), ("quats", (n, 4)), ("scales", (n, 4)), ("status", (n,))):
            _need_np(out[k], shp, f"out[{k}]")
            if not out[k].flags.c_contiguous:
                raise ValueError(f"out[{k}] must be contiguous")
        if len(disp) < V or len(vis) < V:
            raise ValueError("need one disp and one vis array per camera")
        g = Gaussians(n, mo.ctypes.data, q.ctypes.data, s.ctypes.data)
        tr = (ViewTracks * max(V, 1))()
        keep = []
        for v in range(V):
            d = np.ascontiguousarray(disp[v], np.float32)
            m = np.ascontiguousarray(vis[v], np.uint8)
            _need_np(d, (carr[v].height, carr[v].width, 2), f"disp[{v}]")
            _need_np(m, (carr[v].height, carr[v].width), f"vis[{v}]")
            keep += [d, m]
            tr[v].disp, tr[v].vis = d.ctypes.data, m.ctypes.data
        r = Result(out["means"].ctypes.data, out["quats"].ctypes.data, out["scales"].ctypes.data,
                   out["status"].ctypes.data, None, None, None)
        st = C.c_void_p(0) if stream is None else _stream_handle(stream)
        self._check(lib().tsp_fit_motion_host(self._h, C.byref(g), carr, V, tr, C.byref(r), st),
                    "tsp_fit_motion_host")
        return out

    def render(self, means_opacity, quats, scales, sh, sh_degree, cams, stream=None, sync=False):
        """Colour [V] x [H,W,3] and final transmittance [V] x [H,W] (CUDA tensors)."""
        import torch
        n = int(means_opacity.shape[0])
        carr, V = _cams(cams)
        dev = means_opacity.device
        rgb = [torch.empty((carr[v].height, carr[v].width, 3), dtype=torch.float32, device=dev)
               for v in range(V)]
        T = [torch.empty((carr[v].height, carr[v].width), dtype=torch.float32, device=dev)
             for v in range(V)]
        for name, t in (("means_opacity", means_opacity), ("quats", quats), ("scales", scales)):
            _need(t, (n, 4), torch.float32, dev, name)
        _need(sh, (n, (int(sh_degree) + 1) ** 2, 3), torch.float32, dev, "sh")
        g = Gaussians(n, means_opacity.data_ptr(), quats.data_ptr(), scales.data_ptr())
        pr = (C.c_void_p * max(V, 1))(*[x.data_ptr() for x in rgb])
        pt = (C.c_void_p * max(V, 1))(*[x.data_ptr() for x in T])
        self._check(lib().tsp_render(self._h, C.byref(g), C.c_void_p(sh.data_ptr()), int(sh_degree),
                                     carr, V, pr, pt, _stream_handle(stream)), "tsp_render")
        if sync:
            self.sync(stream)
        return rgb, T

    def render_backward(self, means_opacity, quats, scales, sh, sh_degree, cams, rgb, grad_rgb, stream=None,
                        sync=False):
        """Adjoint of render: given its colour images ``rgb`` and dL/dcolour
        ``grad_rgb`` ([V] x [H,W,3] CUDA tensors), returns dL/d(means_opacity,
        quats, scales, sh) with the shapes of those inputs (scales' w = 0)."""
        import torch
        n = int(means_opacity.shape[0])
        carr, V = _cams(cams)
        dev = means_opacity.device
        for name, t in (("means_opacity", means_opacity), ("quats", quats), ("scales", scales)):
            _need(t, (n, 4), torch.float32, dev, name)
        nb = (int(sh_degree) + 1) ** 2
        _need(sh, (n, nb, 3), torch.float32, dev, "sh")
        if len(rgb) < V or len(grad_rgb) < V:
            raise ValueError("need one colour and one gradient image per camera")
        for v in range(V):
            shp = (carr[v].height, carr[v].width, 3)
            _need(rgb[v], shp, torch.float32, dev, f"rgb[{v}]")
            _need(grad_rgb[v], shp, torch.float32, dev, f"grad_rgb[{v}]")
        out = dict(means_opacity=torch.empty((n, 4), dtype=torch.float32, device=dev),
                   quats=torch.empty((n, 4), dtype=torch.float32, device=dev),
                   scales=torch.empty((n, 4), dtype=torch.float32, device=dev),
                   sh=torch.empty((n, nb, 3), dtype=torch.float32, device=dev))
        g = Gaussians(n, means_opacity.data_ptr(), quats.data_ptr(), scales.data_ptr())
        pr = (C.c_void_p * max(V, 1))(*[x.data_ptr() for x in rgb[:V]])
        pg = (C.c_void_p * max(V, 1))(*[x.data_ptr() for x in grad_rgb[:V]])
        r = RenderGrads(out["means_opacity"].data_ptr(), out["scales"].data_ptr(), out["quats"].data_ptr(),
                        out["sh"].data_ptr())
        self._check(lib().tsp_render_backward(self._h, C.byref(g), C.c_void_p(sh.data_ptr()), int(sh_degree),
                                              carr, V, pr, pg, C.byref(r), _stream_handle(stream)),
                    "tsp_render_backward")
        if sync:
            self.sync(stream)
        return out

    # -- motion regularization (Sec. 4.5) ---------------------------------------
    def regularize(self, before, fitted, num_views, *, view_moments=None, k=8, static_min_px=9.0,
                   static_frac=0.9, static_min_views=2, neighbours=False, stream=None, sync=False):
        """Median filter and propagation of a fit's motion.  ``before`` =
        (means_opacity, quats, scales) the fit started from, ``fitted`` its output
        dict (means, quats, scales, status), CUDA tensors.  ``view_moments``
        [V, n, 16] or None for the moments of this context's last fit_motion
        (same n and ``num_views``).  Returns dict(means_opacity, quats, scales,
        flags) and, with ``neighbours``, nbr_pos / nbr_cov [n, k]."""
        import torch
        mo, q, sc = before
        n = int(mo.shape[0])
        dev = mo.device
        f32 = torch.float32
        for name, t in (("means_opacity", mo), ("quats", q), ("scales", sc)):
            _need(t, (n, 4), f32, dev, name)
        for name in ("means", "quats", "scales"):
            _need(fitted[name], (n, 4), f32, dev, f"fitted[{name}]")
        _need(fitted["status"], (n,), torch.int32, dev, "fitted[status]")
        if view_moments is not None:
            _need(view_moments, (int(num_views), n, 16), f32, dev, "view_moments")
        out = dict(means_opacity=torch.empty((n, 4), dtype=f32, device=dev),
                   quats=torch.empty((n, 4), dtype=f32, device=dev),
                   scales=torch.empty((n, 4), dtype=f32, device=dev),
                   flags=torch.empty((n,), dtype=torch.int32, device=dev))
        if neighbours:
            out["nbr_pos"] = torch.empty((n, int(k)), dtype=torch.int32, device=dev)
            out["nbr_cov"] = torch.empty((n, int(k)), dtype=torch.int32, device=dev)
        g = Gaussians(n, mo.data_ptr(), q.data_ptr(), sc.data_ptr())
        r = Result(fitted["means"].data_ptr(), fitted["quats"].data_ptr(), fitted["scales"].data_ptr(),
                   fitted["status"].data_ptr(), None, None, None)
        o = RegOptions(int(k), float(static_min_px), float(static_frac), int(static_min_views))
        rr = RegResult(*[(out[x].data_ptr() if x in out else None) for x in
                         ("means_opacity", "quats", "scales", "flags", "nbr_pos", "nbr_cov")])
        self._check(lib().tsp_regularize(self._h, C.byref(g), C.byref(r), _dptr(view_moments), int(num_views),
                                         C.byref(o), C.byref(rr), _stream_handle(stream)), "tsp_regularize")
        if sync:
            self.sync(stream)
        return out

    def knn(self, means_opacity, mask, k=8, stream=None, sync=False):
        """The k nearest members of ``mask`` (uint8 [n]) of every point, by FP32
        squared distance then index; int32 [n, k], -1 padded."""
        import torch
        n = int(means_opacity.shape[0])
        dev = means_opacity.device
        _need(means_opacity, (n, 4), torch.float32, dev, "means_opacity")
        _need(mask, (n,), torch.uint8, dev, "mask")
        nbr = torch.empty((n, int(k)), dtype=torch.int32, device=dev)
        self._check(lib().tsp_knn(self._h, C.c_void_p(means_opacity.data_ptr()), C.c_void_p(mask.data_ptr()), n,
                                  int(k), C.c_void_p(nbr.data_ptr()), _stream_handle(stream)), "tsp_knn")
        if sync:
            self.sync(stream)
        return nbr

    def sync(self, stream=None, timeout_ms: int = -1):
        st = C.c_void_p(0) if stream is None and not _torch_cuda() else _stream_handle(stream)
        self._check(lib().tsp_sync(self._h, st, int(timeout_ms)), "tsp_sync")

    def inspect(self, which: int) -> np.ndarray:
        """Copy an intermediate of the last call to host memory (after sync)."""
        size = C.c_size_t()
        self._check(lib().tsp_inspect(self._h, which, None, 0, C.byref(size)), "tsp_inspect")
        dtype = {TSP.I_COUNTS: np.int64, TSP.I_RECT: np.int16, TSP.I_DEPTH: np.uint32,
                 TSP.I_TILES_TOUCHED: np.uint32, TSP.I_TILE_OFFSETS: np.uint32,
                 TSP.I_PAIRS: np.uint64, TSP.I_MOMENTS: np.float32, TSP.I_STATS: np.uint64,
                 TSP.I_VIEW_MEANS: np.float32, TSP.I_VIEW_COV: np.float32, TSP.I_KNN_PATH: np.uint32}[which]
        a = np.empty(size.value // np.dtype(dtype).itemsize, dtype)
        self._check(lib().tsp_inspect(self._h, which, _hptr(a), size.value, None), "tsp_inspect")
        return a

    def stage_times(self) -> dict:
        """Per-step device milliseconds of the last call (needs stage_timing=1)."""
        ms = (C.c_float * 7)()
        self._check(lib().tsp_stage_times(self._h, ms, 7, None), "tsp_stage_times")
        return dict(zip(TSP.STAGES, [float(x) for x in ms]))

    def workspace_bytes(self) -> int:
        b = C.c_size_t()
        self._check(lib().tsp_workspace_bytes(self._h, C.byref(b)), "tsp_workspace_bytes")
        return int(b.value)


def _torch_cuda() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False

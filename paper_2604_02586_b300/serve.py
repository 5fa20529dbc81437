"""Request loop for frame-pair motion solves (continuous batching on one GPU).

Requests arrive for scenes; a scene's consecutive frames chain (the Gaussians a
solve returns are the next frame's input, Sec. 5.1's per-frame pipeline).  The
server keeps each active scene resident on the device -- its Gaussians and a
library context whose workspace (sort buffers, moments) is reused frame after
frame -- and admits waiting requests as slots and device memory free up:

* a request is admitted when its scene has no frame in flight, fewer than
  ``max_inflight`` requests are on the device, and the estimated device bytes
  of everything resident plus its tracks stay within ``budget_bytes``; idle
  scenes are evicted (least recently used first, state copied to host memory)
  to make room;
* requests admitted while others run overlap on the device, each on a stream
  taken from a pool; a scene's frames are serialised by CUDA events.  With
  ``priority`` the pool's streams carry CUDA stream priorities and a request
  gets a lower one than every request already on the device, so that the block
  scheduler favours the oldest work (B300 offers four levels; on the serving
  benchmark it did not lower the p99, so it is off by default);
* completion is polled with CUDA events; latency = completion - arrival;
* each scene's library context is given the budget's headroom (the budget less
  what the other resident scenes and the in-flight tracks hold) before every
  solve, so the library itself refuses a workspace that would overrun it;
* a request fails alone -- bad arguments, a scene larger than the whole budget,
  a library refusal or error, a deadline that passed while it waited -- and is
  listed in ``failed`` with the reason; the others carry on.

``one_at_a_time`` replays the same arrivals through a single stream, one request
after the other, as the plain path to compare against.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import Context, TSP, TspError


def _to_device(a, dev):
    # host numpy arrays or (preferably pinned) CPU tensors; pinned sources copy
    # asynchronously on the current stream
    import torch
    t = a if isinstance(a, torch.Tensor) else torch.from_numpy(a)
    return t.to(dev, non_blocking=True)


@dataclasses.dataclass
class Request:
    """One frame pair of a scene: host (pinned) tracks for each of its views."""
    rid: int
    scene: str
    cams: object                 # camera set (width/height/fx/fy/cx/cy/R/t per view) or cameras() pair
    disp: list                   # host float32 [H, W, 2] per view (numpy or pinned tensor)
    vis: list                    # host uint8 [H, W] per view
    arrival: float = 0.0         # seconds, relative to the start of the run
    start: float = 0.0
    done: float = 0.0
    inputs: dict | None = None   # device Gaussians the solve started from (keep_inputs)
    result: dict | None = None   # device outputs
    deadline: float | None = None  # seconds after arrival by which it must start, or None
    error: str | None = None     # why the request failed (then result is None)
    late: bool = False           # finished after arrival + deadline

    @property
    def latency(self):
        return self.done - self.arrival

    def track_bytes(self):
        nb = lambda a: int(a.nbytes) if hasattr(a, "nbytes") else a.numel() * a.element_size()
        return sum(nb(d) + nb(v) for d, v in zip(self.disp, self.vis))


class _Scene:
    def __init__(self, sid, mo, q, s):
        self.sid = sid
        self.host = (mo, q, s)           # host copy while not resident
        self.dev = None                  # (means_opacity, quats, scales) on the device
        self.ctx = None
        self.stream = None               # the stream of the scene's latest frame
        self.last_ev = None              # recorded after the scene's latest device work
        self.busy = False
        self.last_used = 0.0
        self.ws_bytes = 0
        self.views = 1

    @property
    def n(self):
        return int((self.dev or self.host)[0].shape[0])

    def resident_bytes(self, views=0):
        # Gaussians (state + outputs) and the library workspace: ~190 B per
        # (view, Gaussian) record plus ~16 B per expected (tile, Gaussian) pair
        rec = self.n * max(views, self.views, 1)
        est = 2 * 48 * self.n + 190 * rec + 16 * 8 * rec
        return max(est, self.ws_bytes + 2 * 48 * self.n)


class MotionServer:
    def __init__(self, device=0, budget_bytes=120 << 30, max_inflight=8, keep_inputs=False, chain=True,
                 priority=False, **options):
        import torch
        self.torch = torch
        self.device = device
        self.dev = torch.device("cuda", device)
        self.budget = int(budget_bytes)
        self.max_inflight = int(max_inflight)
        self.keep_inputs = keep_inputs
        self.chain = chain                     # False: every frame starts from the resident first frame
        self.options = dict(async_pairs=1)
        self.options.update(options)
        self.scenes: dict[str, _Scene] = {}
        self.waiting: collections.deque[Request] = collections.deque()
        self.inflight: list[tuple[Request, _Scene, object, tuple]] = []
        self.retries = 0
        self.finished: list[Request] = []
        self.failed: list[Request] = []
        self.t0 = time.perf_counter()
        self.evictions = 0
        self.peak_bytes = 0
        # stream pool: level 0 is the highest priority; free streams per level
        self.priority = priority
        lo, hi = torch.cuda.Stream.priority_range() if priority else (0, 0)
        self.levels = list(range(hi, lo + 1)) if hi <= lo else list(range(lo, hi - 1, -1))
        self.free_streams = {k: [] for k in range(len(self.levels))}

    # ---------------------------------------------------------------- scenes
    def add_scene(self, sid, means_opacity, quats, scales):
        """Register a scene by its first frame's Gaussians (host float32 [n, 4])."""
        self.scenes[sid] = _Scene(sid, np.ascontiguousarray(means_opacity, np.float32),
                                  np.ascontiguousarray(quats, np.float32),
                                  np.ascontiguousarray(scales, np.float32))

    def scene_state(self, sid):
        """The scene's current Gaussians as host arrays."""
        sc = self.scenes[sid]
        if sc.dev is None:
            return sc.host
        if sc.last_ev is not None:
            sc.last_ev.synchronize()
        return tuple(t.cpu().numpy() for t in sc.dev)

    def _take_stream(self):
        """A free pool stream one level below every request on the device (the
        lowest level once they reach it).  Returns (level, stream)."""
        used = [item[4] for item in self.inflight]
        level = min(max(used) + 1, len(self.levels) - 1) if used else 0
        pool = self.free_streams[level]
        st = pool.pop() if pool else self.torch.cuda.Stream(device=self.dev, priority=self.levels[level])
        return level, st

    def _give_stream(self, level, st):
        self.free_streams[level].append(st)

    def _used_bytes(self, exclude=None):
        used = 0
        for sc in self.scenes.values():
            if sc.dev is not None and sc is not exclude:
                used += sc.resident_bytes()
        for item in self.inflight:
            used += item[0].track_bytes()
        return used

    def _fail(self, req, sc, why):
        req.error = why
        req.result = None
        req.done = self.now()
        if sc is not None:
            sc.busy = False
        self.failed.append(req)

    def _make_resident(self, sc, stream):
        torch = self.torch
        with torch.cuda.stream(stream):
            sc.dev = tuple(torch.from_numpy(a).pin_memory().to(self.dev, non_blocking=True) for a in sc.host)
        sc.stream = stream
        sc.host = None
        if sc.ctx is None:
            sc.ctx = Context(self.device, **self.options)

    def _evict(self, sc):
        if sc.last_ev is not None:
            sc.last_ev.synchronize()
        sc.host = tuple(t.cpu().numpy() for t in sc.dev)
        sc.dev = None
        sc.ws_bytes = sc.ctx.workspace_bytes()
        sc.ctx.close()
        sc.ctx = None
        self.evictions += 1

    # -------------------------------------------------------------- requests
    def now(self):
        return time.perf_counter() - self.t0

    def submit(self, req: Request):
        self.waiting.append(req)

    def _admit(self):
        """Launch every waiting request that fits (FIFO; a request whose scene is
        busy waits without blocking the ones behind it)."""
        keep = collections.deque()
        while self.waiting:
            req = self.waiting.popleft()
            sc = self.scenes.get(req.scene)
            if sc is None:
                self._fail(req, None, f"unknown scene {req.scene!r}")
                continue
            if req.deadline is not None and self.now() > req.arrival + req.deadline:
                self._fail(req, None, "deadline passed before the request could start")
                continue
            if sc.busy or len(self.inflight) >= self.max_inflight:
                keep.append(req)
                continue
            need = req.track_bytes() + (0 if sc.dev is not None else sc.resident_bytes(len(req.disp)))
            if req.track_bytes() + sc.resident_bytes(len(req.disp)) > self.budget:
                self._fail(req, None, "the scene and its tracks exceed the whole device budget")
                continue
            used = self._used_bytes()
            if used + need > self.budget:
                idle = sorted((s for s in self.scenes.values() if s.dev is not None and not s.busy and s is not sc),
                              key=lambda s: s.last_used)
                while idle and used + need > self.budget:
                    self._evict(idle.pop(0))
                    used = self._used_bytes()
                if used + need > self.budget:
                    keep.append(req)
                    continue
            r = self._launch(req, sc)
            if r == "wait":
                keep.append(req)
            elif r == "ok":
                self.peak_bytes = max(self.peak_bytes, self._used_bytes())
        self.waiting = keep

    def _launch(self, req, sc):
        """Start ``req`` on its scene's stream.  Returns "ok", "failed" (the
        request failed alone and is listed in ``failed``) or "wait" (the library
        refused a workspace that does not fit while other requests hold memory:
        the request waits for them)."""
        level, st = self._take_stream()
        if sc.dev is None:
            self._make_resident(sc, st)
        elif sc.stream is not st:
            # the frame follows the scene's previous one, which ran on another stream
            if sc.last_ev is not None:
                st.wait_event(sc.last_ev)
            for t in sc.dev:
                t.record_stream(st)
            sc.stream = st
        sc.busy = True
        sc.views = max(sc.views, len(req.disp))
        req.start = self.now()
        for attempt in range(2):
            try:
                self._fit(req, sc, level)
                return "ok"
            except TspError as e:
                if e.status != TSP.ERR_BUDGET:
                    self._fail(req, sc, f"TspError: {e}")
                    self._give_stream(level, st)
                    return "failed"
                idle = [x for x in self.scenes.values() if x.dev is not None and not x.busy and x is not sc]
                if attempt == 0 and idle:
                    for x in idle:                 # make room, then try once more
                        self._evict(x)
                    continue
                self._give_stream(level, st)
                if any(x.busy and x is not sc for x in self.scenes.values()):
                    sc.busy = False
                    return "wait"
                self._fail(req, sc, f"TspError: {e}")
                return "failed"
            except (ValueError, TypeError, IndexError) as e:
                # nothing of this request was enqueued (argument checks and workspace
                # refusals come first), and the scene keeps its state
                self._fail(req, sc, f"{type(e).__name__}: {e}")
                self._give_stream(level, st)
                return "failed"
        self._give_stream(level, st)
        return "failed"

    def _fit(self, req, sc, level):
        torch = self.torch
        # the library may grow this scene's workspace only into the headroom
        head = self.budget - self._used_bytes(exclude=sc) - req.track_bytes() - 2 * 48 * sc.n
        sc.ctx.set_budget(max(head, 1))
        with torch.cuda.stream(sc.stream):
            disp = [_to_device(d, self.dev) for d in req.disp]
            vis = [_to_device(v, self.dev) for v in req.vis]
            mo, q, s = sc.dev
            if self.keep_inputs:
                req.inputs = dict(means_opacity=mo.clone(), quats=q.clone(), scales=s.clone())
            out = sc.ctx.fit_motion(mo, q, s, req.cams, disp, vis, stream=sc.stream)
            if self.chain:                     # the solved Gaussians are the next frame's input
                sc.dev = (out["means"], out["quats"], out["scales"])
            ev = torch.cuda.Event()
            ev.record(sc.stream)
        sc.last_ev = ev
        req.result = out
        self.inflight.append((req, sc, ev, (disp, vis, (mo, q, s)), level, sc.stream))

    def poll(self):
        """Retire completed requests; admit waiting ones.  Returns the newly
        finished requests."""
        done = []
        still = []
        retry = []
        for item in self.inflight:
            req, sc, ev, (_, _, prev), level, st = item
            if ev.query():
                sc.busy = False
                self._give_stream(level, st)      # idle: nothing is enqueued before _admit
                try:
                    sc.ctx.sync(st)
                except TspError as e:
                    sc.dev = prev                      # the scene keeps its last good state
                    if e.status != TSP.ERR_OVERFLOW:
                        self._fail(req, sc, f"TspError: {e}")
                        continue
                    # the pair buffer was too small for this frame; the library has
                    # grown it, so the frame runs again from the previous state
                    self.retries += 1
                    retry.append(req)
                    continue
                req.done = self.now()
                req.late = req.deadline is not None and req.done > req.arrival + req.deadline
                sc.last_used = req.done
                done.append(req)
            else:
                still.append(item)
        self.waiting.extendleft(reversed(retry))
        self.inflight = still
        self._admit()
        self.finished.extend(done)
        return done

    def run(self, requests, rate_scale=1.0, poll_s=5e-5):
        """Serve ``requests`` (sorted by arrival, seconds) in real time: each is
        submitted when its arrival time comes.  Returns the finished requests."""
        self.t0 = time.perf_counter()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        while pending or self.waiting or self.inflight:
            t = self.now()
            while pending and pending[0].arrival * rate_scale <= t:
                r = pending.popleft()
                r.arrival *= rate_scale
                self.submit(r)
            self.poll()
            time.sleep(poll_s)
        return self.finished

    def close(self):
        for sc in self.scenes.values():
            if sc.ctx is not None:
                sc.ctx.close()
                sc.ctx = None


def one_at_a_time(requests, scenes, device=0, poll_s=5e-5, chain=True, **options):
    """The plain path: one context and one stream; each request starts when it
    has arrived and the previous one has finished."""
    import torch
    dev = torch.device("cuda", device)
    state = {sid: tuple(torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev) for a in g)
             for sid, g in scenes.items()}
    ctx = Context(device, **dict(dict(async_pairs=0), **options))
    t0 = time.perf_counter()
    out = []
    for req in sorted(requests, key=lambda r: r.arrival):
        while time.perf_counter() - t0 < req.arrival:
            time.sleep(poll_s)
        req.start = time.perf_counter() - t0
        disp = [_to_device(d, dev) for d in req.disp]
        vis = [_to_device(v, dev) for v in req.vis]
        mo, q, s = state[req.scene]
        r = ctx.fit_motion(mo, q, s, req.cams, disp, vis, sync=True)
        if chain:
            state[req.scene] = (r["means"], r["quats"], r["scales"])
        req.result = r
        req.done = time.perf_counter() - t0
        out.append(req)
    ctx.close()
    return out


def latency_stats(reqs, units_of):
    lat = np.array([r.latency for r in reqs]) * 1e3
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return dict(requests=len(reqs), p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                mean_ms=float(lat.mean()), fits_per_s=float(sum(units_of(r) for r in reqs) / span),
                req_per_s=len(reqs) / span)

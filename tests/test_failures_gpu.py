"""Failure handling made on the host, through the C ABI and the request loop
(needs a B300; nothing here faults, traps or hangs the GPU).

* Workspace allocation failure: an allocator hook (tsp_set_allocator) refuses
  the k-th request; the call reports TSP_ERR_OOM before enqueueing anything, the
  outputs keep their contents, and the context then fits as a fresh one does.
* Budget refusal: a workspace ceiling below what a call needs gives
  TSP_ERR_BUDGET before anything is enqueued; raising it lets the same context
  proceed.
* Request loop: a poisoned request (tracks of the wrong size), a scene larger
  than the whole device budget and a request whose deadline passes while it
  waits each fail alone, with the reason; every other request completes and
  equals the same solve run alone.
"""
import numpy as np
import pytest

import synth
from tests import parity as P
from tests.test_parity_gpu import POS_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu_ready():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02586_b300 import build as tbuild
    tbuild.build()
    return True


class HookAllocator:
    """Device blocks from torch's caching allocator; refuses call number
    ``fail_at`` (1-based) when set."""

    def __init__(self, fail_at=None):
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        self.freed = 0

    def alloc(self, nbytes, device):
        import torch
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return None
        t = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{device}")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def free(self, ptr, nbytes, device):
        t = self.live.pop(ptr)
        assert t.numel() == nbytes
        self.freed += 1


def fit(ctx, s, d, out=None, sync=True):
    return ctx.fit_motion(d["means_opacity"], d["quats"], d["scales"], s, d["disp"], d["vis"],
                          out=out, sync=sync)


def sentinel_outputs(n):
    import torch
    return dict(means=torch.full((n, 4), 7.0, device="cuda"), quats=torch.full((n, 4), 7.0, device="cuda"),
                scales=torch.full((n, 4), 7.0, device="cuda"),
                status=torch.full((n,), -1, dtype=torch.int32, device="cuda"))


def host(out):
    r = {k: v.cpu().numpy() for k, v in out.items()}
    r["status"] = r["status"].view(np.uint32)
    return r


def same_fit(a, b, extent):
    assert np.array_equal(a["status"] & 0xFF, b["status"] & 0xFF)
    both = (a["status"] & 1) > 0
    err = np.linalg.norm(a["means"][both, :3] - b["means"][both, :3], axis=1).max() / extent
    assert err < POS_TOL, err


def test_allocator_hook_owns_the_workspace(gpu_ready):
    import torch
    import paper_2604_02586_b300 as tsp
    s = synth.make_scene("tiny", 31, n=1500)
    d = P.to_device(s)
    with tsp.Context(0) as plain:
        ref = host(fit(plain, s, d))
    hook = HookAllocator()
    ctx = tsp.Context(0)
    ctx.set_allocator(hook.alloc, hook.free)
    got = host(fit(ctx, s, d))
    assert hook.calls > 10 and len(hook.live) == hook.calls
    assert ctx.workspace_bytes() == sum(t.numel() for t in hook.live.values())
    same_fit(got, ref, s.extent)
    ctx.close()
    torch.cuda.synchronize()
    assert not hook.live and hook.freed == hook.calls


@pytest.mark.parametrize("fail_at", [1, 6, "last"])
def test_injected_allocation_failure_reports_oom_and_recovers(gpu_ready, fail_at):
    import torch
    import paper_2604_02586_b300 as tsp
    s = synth.make_scene("tiny", 32, n=1200)
    d = P.to_device(s)
    with tsp.Context(0) as plain:
        ref = host(fit(plain, s, d))
    if fail_at == "last":                        # the number of buffers a first call allocates
        probe = HookAllocator()
        with tsp.Context(0, async_pairs=1, pair_capacity=1 << 20) as c:
            c.set_allocator(probe.alloc, probe.free)
            fit(c, s, d)
        fail_at = probe.calls
    hook = HookAllocator(fail_at=fail_at)
    with tsp.Context(0, async_pairs=1, pair_capacity=1 << 20) as ctx:
        ctx.set_allocator(hook.alloc, hook.free)
        out = sentinel_outputs(s.n)
        with pytest.raises(tsp.TspError) as e:
            fit(ctx, s, d, out=out, sync=False)
        assert e.value.status == tsp.TSP.ERR_OOM
        torch.cuda.synchronize()
        assert torch.all(out["means"] == 7.0) and torch.all(out["status"] == -1)   # nothing ran
        got = host(fit(ctx, s, d))               # the hook no longer refuses
    same_fit(got, ref, s.extent)
    assert not hook.live


def test_budget_refusal_before_enqueue_then_recovery(gpu_ready):
    import torch
    import paper_2604_02586_b300 as tsp
    s = synth.make_scene("tiny", 33, n=1500)
    d = P.to_device(s)
    with tsp.Context(0) as plain:
        ref = host(fit(plain, s, d))
        need = plain.workspace_bytes()
    with tsp.Context(0, async_pairs=1, budget_bytes=need // 4) as ctx:
        out = sentinel_outputs(s.n)
        with pytest.raises(tsp.TspError) as e:
            fit(ctx, s, d, out=out, sync=False)
        assert e.value.status == tsp.TSP.ERR_BUDGET
        torch.cuda.synchronize()
        assert torch.all(out["means"] == 7.0) and torch.all(out["status"] == -1)
        assert ctx.workspace_bytes() <= need // 4
        ctx.set_budget(0)                         # unlimited
        got = host(fit(ctx, s, d))
    same_fit(got, ref, s.extent)
    with pytest.raises(tsp.TspError):
        tsp.Context(0).set_budget(-1)


def requests_for_failures():
    from paper_2604_02586_b300.serve import Request
    scenes = {f"s{k}": synth.make_scene("tiny", 40 + k, n=n, views=v, width=w, height=h, focal=float(w))
              for k, (n, v, w, h) in enumerate([(900, 3, 128, 128), (1600, 4, 160, 120), (2500, 3, 128, 96)])}
    reqs, rid = [], 0
    for f in range(2):
        for sid, s in scenes.items():
            reqs.append(Request(rid, sid, s, list(s.disp), list(s.vis), arrival=0.001 * rid))
            rid += 1
    return scenes, reqs


def alone(req):
    import torch
    import paper_2604_02586_b300 as tsp
    with tsp.Context(0) as ctx:
        g = req.inputs
        return ctx.fit_motion(g["means_opacity"], g["quats"], g["scales"], req.cams,
                              [torch.from_numpy(d).cuda() for d in req.disp],
                              [torch.from_numpy(v).cuda() for v in req.vis], sync=True)


def test_poisoned_request_fails_alone(gpu_ready):
    from paper_2604_02586_b300.serve import MotionServer, Request
    scenes, reqs = requests_for_failures()
    s0 = scenes["s0"]
    bad_disp = [d[:-1] for d in s0.disp]                       # one row short per view
    reqs.insert(2, Request(100, "s0", s0, bad_disp, list(s0.vis), arrival=0.0015))
    reqs.append(Request(101, "nowhere", s0, list(s0.disp), list(s0.vis), arrival=0.002))
    srv = MotionServer(0, max_inflight=3, keep_inputs=True)
    for sid, s in scenes.items():
        srv.add_scene(sid, s.means_opacity, s.quats, s.scales)
    done = srv.run(reqs)
    srv.close()
    assert sorted(r.rid for r in srv.failed) == [100, 101]
    assert all(r.error for r in srv.failed)
    assert sorted(r.rid for r in done) == sorted(r.rid for r in reqs if r.rid < 100)
    for req in done:
        a = alone(req)
        same_fit(host(a), host(req.result), scenes[req.scene].extent)


def test_scene_over_budget_and_deadline_fail_alone(gpu_ready):
    from paper_2604_02586_b300.serve import MotionServer, Request
    scenes, reqs = requests_for_failures()
    big = synth.make_scene("tiny", 49, n=20000, views=3, width=256, height=256, focal=256.0)
    budget = 6 << 20                                 # fits the small scenes, not the big one
    reqs.append(Request(200, "big", big, list(big.disp), list(big.vis), arrival=0.0))
    # one request in flight at a time: a zero deadline queued behind others expires
    late = Request(201, "s1", scenes["s1"], list(scenes["s1"].disp), list(scenes["s1"].vis),
                   arrival=0.0, deadline=0.0)
    reqs.append(late)
    srv = MotionServer(0, budget_bytes=budget, max_inflight=1, keep_inputs=True)
    for sid, s in list(scenes.items()) + [("big", big)]:
        srv.add_scene(sid, s.means_opacity, s.quats, s.scales)
    done = srv.run(reqs)
    srv.close()
    failed = {r.rid: r.error for r in srv.failed}
    assert 200 in failed and "budget" in failed[200]
    assert 201 in failed and "deadline" in failed[201]
    assert sorted(r.rid for r in done) == sorted(r.rid for r in reqs if r.rid < 100)
    assert srv.peak_bytes <= budget
    for req in done:
        same_fit(host(alone(req)), host(req.result), scenes[req.scene].extent)


@pytest.mark.parametrize("variant", [0, 5])
def test_checked_mode_on_valid_inputs(gpu_ready, variant):
    """Checked mode (options.checked = 1) tests every index the kernels take
    from data; on valid inputs no test fails (tsp_sync is clean) and the
    results are the unchecked ones: tile lists and flags bit for bit, fitted
    values within the motion-fit tolerances (the float atomics' order varies)."""
    s = synth.make_scene("capture", 34, n=6000, views=4, width=320, height=240, focal=240.0)
    a = P.run_gpu(s, raster_variant=variant)
    b = P.run_gpu(s, raster_variant=variant, checked=1)
    for k in ("rect", "touched", "tile_off", "pairs", "view_flags", "counts"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["status"] & 0xFF, b["status"] & 0xFF)
    both = (a["status"] & 1) > 0
    err = np.linalg.norm(a["means"][both, :3] - b["means"][both, :3], axis=1).max() / s.extent
    assert err < POS_TOL, err
    np.testing.assert_allclose(a["view_moments"][..., 13:15], b["view_moments"][..., 13:15], rtol=0, atol=0)


def test_track_gate_that_nothing_opens_times_out_and_recovers(gpu_ready):
    """A device-side wait on a flag that nothing sets (the track gate) gives up
    after its limit: tsp_sync reports TSP_ERR_TIMEOUT, none of the fitted
    outputs is written, and the context then fits as a fresh one does."""
    import time
    import torch
    import paper_2604_02586_b300 as tsp
    s = synth.make_scene("tiny", 35, n=1500)
    d = P.to_device(s)
    with tsp.Context(0) as plain:
        ref = host(fit(plain, s, d))
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    with tsp.Context(0, async_pairs=1, pair_capacity=1 << 20) as ctx:
        ctx.set_track_gate(flag, 1, timeout_us=20_000)
        out = sentinel_outputs(s.n)
        t0 = time.perf_counter()
        fit(ctx, s, d, out=out, sync=False)
        with pytest.raises(tsp.TspError) as e:
            ctx.sync()
        waited = time.perf_counter() - t0
        assert e.value.status == tsp.TSP.ERR_TIMEOUT
        assert 0.01 < waited < 5.0
        assert torch.all(out["means"] == 7.0) and torch.all(out["status"] == -1)
        ctx.set_track_gate(None)
        got = host(fit(ctx, s, d))
    same_fit(got, ref, s.extent)


def test_track_gate_already_open_changes_nothing(gpu_ready):
    """A gate whose flag already holds a value at or above the one it waits for
    lets the call run as without a gate."""
    import torch
    import paper_2604_02586_b300 as tsp
    s = synth.make_scene("tiny", 36, n=1500)
    d = P.to_device(s)
    with tsp.Context(0) as plain:
        ref = host(fit(plain, s, d))
    flag = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    with tsp.Context(0) as ctx:
        ctx.set_track_gate(flag, 5, timeout_us=1_000_000)
        got = host(fit(ctx, s, d))
        with pytest.raises(tsp.TspError):
            ctx.set_track_gate(flag, 1, timeout_us=0)
    same_fit(got, ref, s.extent)

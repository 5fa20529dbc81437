"""The request loop (paper_2604_02586_b300.serve) on a B300.

Requests for several scenes arrive together, so they overlap on the device (one
stream per resident scene) and are admitted as slots and the memory budget
allow; each scene's frames chain (a solve's output Gaussians are the next
frame's input).  Every result must equal the same solve run alone on a fresh
context from the Gaussians it started from, within the motion-fit tolerances
(statuses equal but for blend decisions inside the FP32 window; positions
within 1e-4 of the scene extent) -- with and without evictions.
"""
import numpy as np
import pytest

import synth
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


def make_requests(frames_per_scene=3):
    from paper_2604_02586_b300.serve import Request
    scenes = {f"s{k}": synth.make_scene("tiny", 20 + k, n=n, views=v, width=w, height=h, focal=float(w))
              for k, (n, v, w, h) in enumerate([(800, 3, 128, 128), (1500, 4, 160, 120),
                                                (3000, 4, 128, 128), (5000, 3, 192, 144)])}
    reqs, rid = [], 0
    for f in range(frames_per_scene):
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


def check_same_as_alone(scenes, done):
    for req in done:
        a = alone(req)
        sa = a["status"].cpu().numpy().view(np.uint32)
        sb = req.result["status"].cpu().numpy().view(np.uint32)
        assert (sa == sb).mean() > 0.999, req.rid
        both = ((sa & 1) > 0) & ((sb & 1) > 0)
        d = np.linalg.norm(a["means"].cpu().numpy()[both, :3] - req.result["means"].cpu().numpy()[both, :3], axis=1)
        assert d.max() / scenes[req.scene].extent < POS_TOL, req.rid


@pytest.mark.parametrize("budget", [120 << 30, 8 << 20])
def test_overlapping_requests_equal_requests_alone(gpu_ready, budget):
    from paper_2604_02586_b300.serve import MotionServer
    scenes, reqs = make_requests()
    srv = MotionServer(0, budget_bytes=budget, max_inflight=4, keep_inputs=True)
    for sid, s in scenes.items():
        srv.add_scene(sid, s.means_opacity, s.quats, s.scales)
    done = srv.run(reqs)
    srv.close()
    assert sorted(r.rid for r in done) == [r.rid for r in reqs]
    for sid in scenes:                                   # a scene's frames finish in order
        ids = [r.rid for r in sorted(done, key=lambda r: r.done) if r.scene == sid]
        assert ids == sorted(ids)
    if budget < (1 << 30):
        assert srv.evictions > 0
    check_same_as_alone(scenes, done)


def test_chained_state_advances(gpu_ready):
    """The second frame of a scene starts from the first frame's solved Gaussians."""
    from paper_2604_02586_b300.serve import MotionServer
    scenes, reqs = make_requests(frames_per_scene=2)
    srv = MotionServer(0, keep_inputs=True)
    for sid, s in scenes.items():
        srv.add_scene(sid, s.means_opacity, s.quats, s.scales)
    done = {r.rid: r for r in srv.run(reqs)}
    srv.close()
    n_sc = len(scenes)
    for k in range(n_sc):
        first, second = done[k], done[k + n_sc]
        assert np.array_equal(second.inputs["means_opacity"].cpu().numpy(), first.result["means"].cpu().numpy())

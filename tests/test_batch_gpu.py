"""tsp_fit_motion_batch: frame pairs of uneven sizes in one launch of each step
(Sec. 4.6: frame pairs are independent units), through the C ABI (needs a B300).

Each frame of a batch must meet the single-frame bar against the FP64 oracle:
its tile lists bit-exactly (the batch numbers the tiles of all frames together),
its fitted Gaussians within the motion-fit tolerances; and it must agree with the
same frame solved alone (statuses equal, values within the tolerances: only the
order of the floating-point atomic additions differs).
"""
import numpy as np
import pytest

import oracle
import synth
from tests import parity as P
from tests.test_parity_gpu import caps_for, check_fitted, POS_TOL, SCALE_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu_ready():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02586_b300 import build as tbuild
    tbuild.build()
    return True


def scenes():
    return [synth.make_scene("tiny", 11, n=1500),
            synth.make_scene("capture", 12, n=6000, views=5, width=320, height=240, focal=240.0),
            synth.make_scene("tiny", 13, n=700, views=3, width=100, height=70, focal=80.0)]


def frame_args(s, **kw):
    d = P.to_device(s)
    return dict(means_opacity=d["means_opacity"], quats=d["quats"], scales=d["scales"], cams=s,
                disp=d["disp"], vis=d["vis"], **kw)


def host(out):
    r = {k: v.cpu().numpy() for k, v in out.items()}
    r["status"] = r["status"].view(np.uint32)
    if "view_flags" in r:
        r["view_flags"] = r["view_flags"].view(np.uint32)
    return r


@pytest.fixture(scope="module")
def batch(gpu_ready):
    import torch
    import paper_2604_02586_b300 as tsp
    ss = scenes()
    with tsp.Context(0) as ctx:
        outs = ctx.fit_motion_batch([frame_args(s, view_flags=True) for s in ss], sync=True)
        torch.cuda.synchronize()
        T = tsp.TSP
        inter = dict(tile_off=ctx.inspect(T.I_TILE_OFFSETS), pairs=ctx.inspect(T.I_PAIRS),
                     counts=ctx.inspect(T.I_COUNTS))
        alone = []
        for s in ss:
            alone.append(host(ctx.fit_motion(**frame_args(s, view_flags=True), sync=True)))
    return ss, [host(o) for o in outs], alone, inter


def test_batch_tile_lists_bit_exact_per_frame(batch):
    ss, _, _, inter = batch
    off_all = inter["tile_off"].astype(np.int64)
    pairs = inter["pairs"]
    t0, total = 0, 0
    for s in ss:
        off, ent = oracle.bin_lists(s)
        nt = len(off) - 1
        seg = off_all[t0:t0 + nt + 1]
        assert np.array_equal(seg - seg[0], off)
        assert np.array_equal(pairs[seg[0]:seg[-1]], ent)
        t0 += nt
        total += len(ent)
    assert int(inter["counts"][0]) == total and int(inter["counts"][3]) == 0


def test_batch_with_wide_tiles_meets_the_oracle(gpu_ready):
    """The batched launch with 32 x 8 tiles (the 100 x 70 frame is ragged in both
    directions): each frame's tile lists equal the oracle's for that tile shape
    bit for bit, and its fitted Gaussians meet the oracle bar."""
    import torch
    import paper_2604_02586_b300 as tsp
    ss = scenes()
    with tsp.Context(0, tile_w=32, tile_h=8) as ctx:
        outs = ctx.fit_motion_batch([frame_args(s) for s in ss], sync=True)
        torch.cuda.synchronize()
        off_all = ctx.inspect(tsp.TSP.I_TILE_OFFSETS).astype(np.int64)
        pairs = ctx.inspect(tsp.TSP.I_PAIRS)
    opt = oracle.default_options(tile=(32, 8))
    t0 = 0
    for s, out in zip(ss, outs):
        off, ent = oracle.bin_lists(s, tile=(32, 8))
        nt = len(off) - 1
        seg = off_all[t0:t0 + nt + 1]
        assert np.array_equal(seg - seg[0], off)
        assert np.array_equal(pairs[seg[0]:seg[-1]], ent)
        t0 += nt
        o = oracle.fit_motion(s, opt)
        check_fitted(s, host(out), o, P.sensitivity(s, o, options=opt), tag=f"batch32x8:{s.n}",
                     caps=caps_for(s))


def test_batch_frames_meet_the_oracle_bar(batch):
    ss, outs, _, _ = batch
    for s, g in zip(ss, outs):
        o = oracle.fit_motion(s)
        check_fitted(s, g, o, P.sensitivity(s, o), tag=f"batch:{s.n}",
                     caps=caps_for(s))


def test_batch_frames_equal_frames_alone(batch):
    ss, outs, alone, _ = batch
    for s, b, a in zip(ss, outs, alone):
        assert (b["status"] == a["status"]).mean() > 0.999
        both = ((b["status"] & 1) > 0) & ((a["status"] & 1) > 0)
        dp = np.linalg.norm(b["means"][both, :3] - a["means"][both, :3], axis=1) / s.extent
        assert dp.max() < POS_TOL
        assert (b["view_flags"] == a["view_flags"]).mean() > 0.999


def test_batch_with_empty_and_viewless_frames(gpu_ready):
    import torch
    import paper_2604_02586_b300 as tsp
    s = synth.make_scene("tiny", 14, n=400)
    viewless = frame_args(s.subset_views([]))
    empty = frame_args(s)
    for k in ("means_opacity", "quats", "scales"):
        empty[k] = empty[k][:0]
    with tsp.Context(0) as ctx:
        outs = ctx.fit_motion_batch([empty, frame_args(s), viewless], sync=True)
        ref = ctx.fit_motion(**frame_args(s), sync=True)
    assert outs[0]["means"].shape[0] == 0
    st = outs[2]["status"].cpu().numpy().view(np.uint32)
    assert np.all(st & oracle.OS_FEW_VIEWS) and not np.any(st & oracle.OS_POS_OK)
    assert torch.equal(outs[2]["means"], viewless["means_opacity"])
    assert (outs[1]["status"] == ref["status"]).float().mean().item() > 0.999


def test_batch_limits_are_enforced(gpu_ready):
    import paper_2604_02586_b300 as tsp
    s = synth.make_scene("tiny", 15, n=50, views=32, width=32, height=32, focal=32.0)
    with tsp.Context(0) as ctx:
        with pytest.raises(tsp.TspError):
            ctx.fit_motion_batch([frame_args(s)] * 7)        # 224 views > 192
        with pytest.raises(tsp.TspError):
            ctx.fit_motion_batch([frame_args(synth.make_scene("tiny", 16, n=20))] * 17)   # 17 frames


def test_batch_replays_from_a_cuda_graph(gpu_ready):
    """The batch call enqueues no host synchronisation and no allocation once its
    workspace is sized (asynchronous pair counting), so it can be captured in a
    CUDA graph; a replay after the tracks change in place gives what a direct
    call on the changed tracks gives."""
    import torch
    import paper_2604_02586_b300 as tsp
    ss = scenes()
    args = [frame_args(s) for s in ss]
    with tsp.Context(0) as probe:
        probe.fit_motion_batch(args, sync=True)
        K = int(probe.inspect(tsp.TSP.I_COUNTS)[0])
    for variant in (0, 5):
        with tsp.Context(0, async_pairs=1, pair_capacity=2 * K, raster_variant=variant) as ctx:
            outs = ctx.fit_motion_batch(args, sync=True)           # sizes the workspace
            for a, o in zip(args, outs):
                a["out"] = o
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                ctx.fit_motion_batch(args)                        # warm-up on the capture stream
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                ctx.fit_motion_batch(args)
            for a in args:                                        # new tracks, same buffers
                for d in a["disp"]:
                    d.mul_(0.5)
            graph.replay()
            torch.cuda.synchronize()
            got = [host(o) for o in outs]
            ctx.sync()
            direct = [host(o) for o in ctx.fit_motion_batch([{k: v for k, v in a.items() if k != "out"}
                                                             for a in args], sync=True)]
            for s, g, d in zip(ss, got, direct):
                assert (g["status"] == d["status"]).mean() > 0.999
                both = ((g["status"] & 1) > 0) & ((d["status"] & 1) > 0)
                dp = np.linalg.norm(g["means"][both, :3] - d["means"][both, :3], axis=1) / s.extent
                assert dp.max() < POS_TOL
        for a in args:                                            # restore for the next variant
            a.pop("out", None)
            for d in a["disp"]:
                d.mul_(2.0)


def test_single_fit_replays_from_a_cuda_graph(gpu_ready):
    """tsp_fit_motion on one frame, captured once in a CUDA graph (the bench times
    its steps this way) and replayed after the tracks change in place, gives what a
    direct call on the changed tracks gives; the tile lists are the same keys."""
    import torch
    import paper_2604_02586_b300 as tsp
    s = scenes()[1]
    a = frame_args(s)
    with tsp.Context(0) as probe:
        probe.fit_motion(a["means_opacity"], a["quats"], a["scales"], s, a["disp"], a["vis"], sync=True)
        K = int(probe.inspect(tsp.TSP.I_COUNTS)[0])
    with tsp.Context(0, async_pairs=1, pair_capacity=2 * K) as ctx:
        out = ctx.fit_motion(a["means_opacity"], a["quats"], a["scales"], s, a["disp"], a["vis"], sync=True)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            ctx.fit_motion(a["means_opacity"], a["quats"], a["scales"], s, a["disp"], a["vis"], out=out)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            ctx.fit_motion(a["means_opacity"], a["quats"], a["scales"], s, a["disp"], a["vis"], out=out)
        for d in a["disp"]:
            d.mul_(0.5)
        graph.replay()
        torch.cuda.synchronize()
        got = host(out)
        pairs_graph = ctx.inspect(tsp.TSP.I_PAIRS)
        ctx.sync()
    with tsp.Context(0) as ref:
        direct = host(ref.fit_motion(a["means_opacity"], a["quats"], a["scales"], s, a["disp"], a["vis"], sync=True))
        pairs_direct = ref.inspect(tsp.TSP.I_PAIRS)
    assert np.array_equal(pairs_graph, pairs_direct)
    assert (got["status"] == direct["status"]).mean() > 0.999
    both = ((got["status"] & 1) > 0) & ((direct["status"] & 1) > 0)
    assert both.mean() > 0.3
    dp = np.linalg.norm(got["means"][both, :3] - direct["means"][both, :3], axis=1) / s.extent
    assert dp.max() < POS_TOL


def test_autotune_cache_times_once_and_reuses_the_choice(gpu_ready, tmp_path):
    """The first call tunes and appends one line for the workload's key; the next
    call, and a fresh context, take that choice from the file without timing;
    lines of another form or another key do not match."""
    import paper_2604_02586_b300 as tsp
    ss = scenes()
    args = [frame_args(s) for s in ss]
    path = tmp_path / "tune.txt"
    path.write_text("not a tuning line\ntsp-autotune-v1 1 1 1 3 0.5\n")
    with tsp.Context(0) as ctx:
        chosen, times, hit = ctx.autotune_cached(args, str(path), repeats=1)
        assert not hit and chosen in tsp.Context.TUNE_CANDIDATES
        assert times[chosen] == min(times.values()) > 0
        lines = path.read_text().splitlines()
        assert len(lines) == 3 and lines[-1].startswith("tsp-autotune-v1 ")
        chosen2, times2, hit2 = ctx.autotune_cached(args, str(path), repeats=1)
        assert hit2 and chosen2 == chosen
        assert times2[chosen] == pytest.approx(times[chosen], rel=1e-3)
        assert all(v == -1.0 for c, v in times2.items() if c != chosen)
    with tsp.Context(0) as ctx:
        chosen3, _, hit3 = ctx.autotune_cached(args, str(path), repeats=1)
        assert hit3 and chosen3 == chosen
        o = ctx.opt
        assert (o.tile_w, o.tile_h, o.raster_variant) == chosen
    assert len(path.read_text().splitlines()) == 3


def test_autotune_picks_a_candidate_and_results_hold(gpu_ready):
    import paper_2604_02586_b300 as tsp
    ss = scenes()
    args = [frame_args(s) for s in ss]
    with tsp.Context(0) as ctx:
        ref = [host(o) for o in ctx.fit_motion_batch(args, sync=True)]
        chosen, times = ctx.autotune(args, repeats=2)
        assert chosen in tsp.Context.TUNE_CANDIDATES
        assert all(t > 0 for t in times.values()) and times[chosen] == min(times.values())
        got = [host(o) for o in ctx.fit_motion_batch(args, sync=True)]
    for g, r in zip(got, ref):
        assert (g["status"] == r["status"]).mean() > 0.999

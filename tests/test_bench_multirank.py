"""The multi-rank logic of bench.py on CPU: two gloo ranks on 127.0.0.1.

Frame pairs are independent, so each rank solves its own scene (its own seed)
with no collective on the data path; the only exchange is the max-reduce of
the timed region, and the job's throughput is every rank's units over the
slowest rank's time (weak scaling).  The reference arm runs on rank 0 only.
"""
import contextlib
import io
import os
import socket
import types

import numpy as np
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    local_ms = 10.0 + 5.0 * r                       # rank 1 is the slow one
    mx = bench.reduce_max(local_ms, w, "cpu")
    scene = bench.make_scene(types.SimpleNamespace(preset="capture", n=300, views=2), r)
    q.put((r, w, mx, bench.job_value(1000, w, 4, mx), bench.rank_seed(r),
           float(scene.means_opacity[:, :3].sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_solve_different_scenes():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=300) for _ in ps)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, w0, mx0, v0, s0, c0), (r1, w1, mx1, v1, s1, c1) = out
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert mx0 == mx1 == 15.0                       # both ranks see the slowest time
    assert v0 == v1 == 1000 * 2 * 4 / 0.015         # all units over that time
    assert s0 != s1 and c0 != c1                    # independent frame pairs


def test_single_rank_needs_no_process_group():
    assert bench.reduce_max(7.5, 1, "cpu") == 7.5
    assert bench.job_value(10, 1, 2, 20.0) == 1000.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(types.SimpleNamespace(preset="capture", n=300, views=2, steps=1, warmup=0, gpus=2))
    assert buf.getvalue() == ""


def test_reference_arm_line_on_rank_zero(monkeypatch):
    import json
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(types.SimpleNamespace(preset="capture", n=300, views=2, steps=1, warmup=0, gpus=1))
    line = json.loads(buf.getvalue())
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT,
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}

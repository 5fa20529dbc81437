"""Benchmark: Gaussian x view track fits per second on the capture-sized workload.

Workload (one step = one frame-pair motion solve, every hot-path step a1-a9):
200,000 Gaussians x 18 views at 1352x1014 (half the 2704x2028 frames of an
18-view capture), seeded synthetic scene and tracks.  Inputs (tracks 222 MB)
are larger than the 126 MB L2 and L2 is also flushed between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU: one process per GPU under torchrun;
each rank solves its own frame pair (frame pairs are independent), so scaling
is weak and there is no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gaussian·view track fits/s at 200k Gaussians×18 views; p50/p99 frame latency"
UNIT = "fits/s"
KERNELS_PER_STEP = 11         # project, scan (3), emit, tile sort (2), reference gather, raster, view solve, multi-view
RASTER_SRC = os.path.join(ROOT, "paper_2604_02586_b300", "csrc", "raster.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "raster_accumulate_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--preset", default="capture", choices=["capture", "tiny"],
                    help="capture: 200k Gaussians x 18 views at 1352x1014 (the metric's workload); "
                         "tiny: 2,000 Gaussians x 4 ring views at 128x128 (launch-bound)")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--views", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def config(a, scene=None):
    import synth
    p = synth.PRESETS[a.preset]
    n = a.n if a.n is not None else p["n"]
    views = a.views if a.views is not None else p["views"]
    w, h = (int(scene.width[0]), int(scene.height[0])) if scene is not None else (None, None)
    name = {"capture": "capture frame pair", "tiny": "tiny frame pair"}[a.preset]
    c = {"workload": f"{name}: {n} Gaussians x {views} views @ {w}x{h}, tracks + vis",
         "n_gaussians": n, "views": views, "width": w, "height": h, "tile": "16x16"}
    if a.preset == "capture":
        c["l2"] = "flushed between timed steps (256 MB write); inputs 222 MB > L2"
    else:
        c["l2"] = "flushed between timed steps (256 MB write); inputs fit in L2 (launch-bound case)"
    return c


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def raster_traffic():
    """Per-launch DRAM bytes of the raster kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as f:
        t = json.load(f)
    sha = hashlib.sha256(open(RASTER_SRC, "rb").read()).hexdigest()
    if t.get("raster_cu_sha256") != sha:
        return None
    return t.get("bytes_per_launch_full")


def rank_seed(rank):
    """Each rank solves its own frame pair: a scene drawn from its own seed."""
    return 2 + 1000 * rank


def make_scene(a, rank):
    import synth
    return synth.make_scene(a.preset, seed=rank_seed(rank), n=a.n, views=a.views)


def reduce_max(x, world, device):
    """The largest of the ranks' values (the job takes as long as its slowest rank)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, steps, total_ms):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world * steps / (total_ms / 1e3)


def cpu_baseline(scene, max_views=8):
    import oracle
    V = min(scene.num_views, max(1, os.cpu_count() or 1), max_views)
    sub = scene.subset_views(range(V))
    r = oracle.fit_motion(sub, per_view=False)
    return {"value": scene.n * V / r["seconds"], "unit": UNIT, "cores": int(r["threads"]),
            "kind": "oracle",
            "sample": f"all {scene.n} Gaussians over the first {V} of {scene.num_views} views "
                      f"(FP64 C oracle, OpenMP over views), {r['seconds']:.1f} s on {cpu_model()}"}


def run_reference(a):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    scene = make_scene(a, 0)
    V = min(scene.num_views, os.cpu_count() or 1, 8)
    sub = scene.subset_views(range(V))
    times = []
    threads = 1
    for i in range(a.warmup + a.steps):
        r = oracle.fit_motion(sub, per_view=False)
        threads = r["threads"]
        if i >= a.warmup:
            times.append(r["seconds"])
    tot = float(np.sum(times))
    value = scene.n * V * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(a, scene),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"each step: all {scene.n} Gaussians over {V} of "
                                       f"{scene.num_views} views, FP64 C oracle on {cpu_model()}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(a):
    import torch
    import paper_2604_02586_b300 as tsp
    from paper_2604_02586_b300 import build as tbuild
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tbuild.build()

    scene = make_scene(a, rank)
    units = scene.n * scene.num_views
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    mo, q, s = t(scene.means_opacity), t(scene.quats), t(scene.scales)
    disp = [t(d) for d in scene.disp]
    vis = [t(v) for v in scene.vis]

    # size the pair buffer once (synchronous call), then run asynchronously
    probe = tsp.Context(local)
    out = probe.fit_motion(mo, q, s, scene, disp, vis, sync=True)
    K = int(probe.inspect(tsp.TSP.I_COUNTS)[0])
    probe.close()
    # exact raster work for the ALU roofline (counting variant, untimed)
    cnt = tsp.Context(local, collect_stats=1, async_pairs=1, pair_capacity=int(K * 1.1) + 1024)
    cnt.fit_motion(mo, q, s, scene, disp, vis, out=out, sync=True)
    n_eval, n_blend, n_add, n_list = [int(x) for x in cnt.inspect(tsp.TSP.I_STATS)]
    cnt.close()

    ctx = tsp.Context(local, async_pairs=1, stage_timing=1, pair_capacity=int(K * 1.1) + 1024)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(a.warmup):
        ctx.fit_motion(mo, q, s, scene, disp, vis, out=out)
    ctx.sync()
    step_ms, raster_ms, stages = [], [], []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(a.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.fit_motion(mo, q, s, scene, disp, vis, out=out)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            st = ctx.stage_times()
            stages.append(st)
            raster_ms.append(st["raster"])
        torch.cuda.synchronize()
    ctx.sync()
    if world > 1:
        torch.distributed.barrier()
    total_ms = reduce_max(float(np.sum(step_ms)), world, dev)
    value = job_value(units, world, a.steps, total_ms)

    # end to end through the host-buffer entry point (pinned inputs and outputs)
    e2e = None
    if not a.no_e2e:
        pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()
        hmo, hq, hs = pin(scene.means_opacity), pin(scene.quats), pin(scene.scales)
        hd = [pin(d) for d in scene.disp]
        hv = [pin(v) for v in scene.vis]
        hout = {k: torch.empty(shp, dtype=dt).pin_memory().numpy() for k, shp, dt in
                (("means", (scene.n, 4), torch.float32), ("quats", (scene.n, 4), torch.float32),
                 ("scales", (scene.n, 4), torch.float32), ("status", (scene.n,), torch.int32))}
        hout["status"] = hout["status"].view(np.uint32)
        for _ in range(2):
            ctx.fit_motion_host(hmo, hq, hs, scene, hd, hv, out=hout)
        ts = []
        for _ in range(max(3, a.steps // 2)):
            t0 = time.perf_counter()
            ctx.fit_motion_host(hmo, hq, hs, scene, hd, hv, out=hout)
            ts.append(time.perf_counter() - t0)
        h2d = 3 * 16 * scene.n + sum(int(d.nbytes) + int(v.nbytes) for d, v in zip(hd, hv))
        d2h = 52 * scene.n
        e2e = {"value": units / float(np.mean(ts)), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * float(np.mean(ts))}
    ctx.close()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    peaks, kind = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # FP32 work the blend needs (FMA = 2 flops): 10 per evaluation (offsets,
    # whitening, quadratic form, opacity), 3 per blended contribution
    # (transmittance and weight), 27 per moment addition (12 products, 15 sums)
    flops = 10.0 * n_eval + 3.0 * n_blend + 27.0 * n_add
    t_r = float(np.mean(raster_ms)) / 1e3
    achieved = flops / t_r / 1e12
    peak = sms * 128 * 2 * sm_max * 1e6 / 1e12
    stage_mean = {k: float(np.mean([x[k] for x in stages])) for k in stages[0]}
    # whole step against HBM: the bytes the method must move per frame pair --
    # tracks and visibility, Gaussians in, results out, each pair written and read
    b_alg = (sum(int(d.nbytes) + int(v.nbytes) for d, v in zip(scene.disp, scene.vis))
             + 48 * scene.n + 52 * scene.n + 2 * 12 * K)
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    hbm_step = {"bytes": b_alg, "achieved_gbs": b_alg / (total_ms / a.steps / 1e3) / 1e9,
                "peak_gbs": hbm, "frac": b_alg / (total_ms / a.steps / 1e3) / 1e9 / hbm}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config(a, scene),
        "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": raster_traffic(),
                     "kernel": "k_raster_accumulate_2p",
                     "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (unit counts)",
                     "work": {"evaluations": n_eval, "blended": n_blend, "moment_adds": n_add,
                              "list_entries": n_list, "pairs_K": K},
                     "kernel_ms": t_r * 1e3},
        "hbm_step": hbm_step,
        "stage_ms": stage_mean,
        "gpu_launches": KERNELS_PER_STEP * a.steps,
        "clocks": clk.summary(),
        "e2e": e2e,
        "peaks_source": kind,
    }
    if not a.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline(scene)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()

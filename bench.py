#!/usr/bin/env python
"""Throughput of the Jacobi-PCA hot path on scene-shaped cubes (one JSON line).

Workload (one step): the two scene-shaped cubes of the paper's evaluation
(610x340 pixels x 103 bands and 512x217 pixels x 224 bands, FP32, 12-endmember
mixtures, k = 10, tol 1e-10, 30 sweeps max), each fitted end to end: band
means + covariance, Jacobi eigen-decomposition, sort/sign, projection.

Metric: Mpixel-bands/s = sum(N*B) / step time.  `value` is the mixed form
(tensor-core covariance + FP64 refinement) with inputs resident in HBM; the
plain FP32 form is measured beside it, each with its error against the FP64
oracle.  The L2 is flushed (256 MiB write) before every timed step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With torchrun (N > 1) every rank fits its own copy of the workload (weak
scaling, no data-path collective); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PCA Mpixel-bands/s end-to-end, mixed vs FP32 at stated error; % of roofline"
UNIT = "Mpixel-bands/s"
WORKLOAD = "paper-scene cubes 610x340x103 + 512x217x224, FP32, k=10"
SM_LANES_FP32 = 128          # FP32 lanes per SM (sm_103a)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", default="mix")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched form (256 tiles, 15.9 M pixels)")
    ap.add_argument("--no-paper-shapes", action="store_true",
                    help="skip the k=1 fits at the shapes of the paper's tables")
    ap.add_argument("--no-diff", action="store_true",
                    help="skip the differentiation form (forward + backward on 512 x 512 x 200)")
    ap.add_argument("--ncu-case", choices=["scenes", "big", "batched", "batched-small", "backward"],
                    default=None,
                    help="untimed fits for profiler captures: 'scenes' = the bench cubes, "
                         "'big' = one 1024x400x224 scene cube (367 MB, larger than L2), "
                         "'batched' = the 256-tile batch (10 GB), 'batched-small' = its first "
                         "48 tiles with N / 4 (about 0.5 GB), 'backward' = the adjoint on the "
                         "512x512x200 gradient cube; runs --warmup + --steps fits (or "
                         "backward passes) and prints no JSON line")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ distributed plumbing
def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(x: float, world: int) -> float:
    """Max of a host float over all ranks (the step time of the slowest rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate(units_per_rank_step: float, steps: int, max_seconds: float, world: int) -> float:
    """Whole-job throughput: units all ranks processed / the slowest rank's time."""
    return units_per_rank_step * steps * world / max_seconds / 1e6


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every interval_ms from one
    process started before the first timed region; `with sampler:` marks a timed
    region, and only samples whose timestamps fall inside a region are kept."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 20):
        self.regions = []
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(interval_ms)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        import atexit
        atexit.register(self._stop)          # never leave the sampler running
        time.sleep(0.5)                      # let the first samples arrive

    def _stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.proc = None

    def __enter__(self):
        self.regions.append([time.time(), None])
        return self

    def __exit__(self, *exc):
        self.regions[-1][1] = time.time()
        return False

    def summary(self):
        import datetime
        self._stop()
        if not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                t = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                clk, mx = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            if not any(r0 <= t <= r1 for r0, r1 in self.regions if r1 is not None):
                continue
            sm.append(clk)
            smax.append(mx)
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm),
                "regions": len(self.regions)}


# ------------------------------------------------------------------ helpers
def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def profiled_traffic(kernel: str):
    """dram bytes per launch recorded in profiles/<kernel>*.md ('traffic_bytes_per_launch: X')."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    for name in sorted(os.listdir(d)):
        if name.startswith(kernel) and name.endswith(".md"):
            m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", open(os.path.join(d, name)).read())
            if m:
                return float(m.group(1))
    return None


def jacobi_flops(B: int, sweeps: int) -> float:
    """Algorithmic FP32 flops of the Jacobi kernel: every parallel step rotates the
    B'(B'+1)/2 upper-triangle entries by their row pair and their column pair
    (3 flops each side: c*a + s*b), B' steps per sweep."""
    Bp = B + (B & 1)
    return float(sweeps) * Bp * 3.0 * Bp * (Bp + 1)


# ------------------------------------------------------------------ reference arm (oracle)
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    import synth
    threads = oracle.set_threads(0)
    cubes = synth.paper_scenes()
    units = sum(c.N * c.B for c in cubes)
    # bound the run: sample the pixels if one full step would take too long
    t0 = time.perf_counter()
    for c in cubes:
        oracle.pca_fit(c.Y, c.k, tol=c.tol, sweeps_max=c.sweeps_max)
    t_full = time.perf_counter() - t0
    frac = 1.0
    budget = 150.0 / max(1, args.steps + args.warmup)
    if t_full > budget:
        frac = max(0.05, budget / t_full)
    sample = [c.Y[: max(2, int(c.N * frac))] for c in cubes]
    units_s = sum(s.shape[0] * s.shape[1] for s in sample)
    for _ in range(args.warmup):
        for c, Y in zip(cubes, sample):
            oracle.pca_fit(Y, c.k, tol=c.tol, sweeps_max=c.sweeps_max)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for c, Y in zip(cubes, sample):
            oracle.pca_fit(Y, c.k, tol=c.tol, sweeps_max=c.sweeps_max)
    dt = time.perf_counter() - t0
    value = units_s * args.steps / dt / 1e6
    samp = ("full workload" if frac == 1.0 else
            f"first {frac:.3f} of each cube's pixels (all bands), Jacobi unchanged")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "units_per_step": units},
            "cpu_baseline": {"kind": "oracle", "cores": threads, "sample": samp, "value": value,
                             "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ profiler case
BATCH_WORKLOAD = ("256 tiles, N log-uniform in [4096, 262144], B uniform in "
                  "{64,96,128,160,200,224,256}, 3-15 endmember FP32 mixtures (seed 3), k=8, "
                  "tol 1e-8, 30 sweeps max")


def run_batched(args, dev, peaks, peak_src):
    """The batched form on the 256-tile workload: the batched MIX and P32 forms
    (plain launches and a replayed CUDA graph) against fitting the tiles one by
    one with the plain FP32 form, plus per-stage times and errors of sampled
    tiles against the oracle.  Inputs (10 GB) exceed the L2, so no flush."""
    import torch

    import paper_2403_18321_gb300 as g
    import synth
    specs = synth.tile_batch_specs(seed=3)
    cubes = [synth.tile_device(sp, dev) for sp in specs]
    Ys = [c.Y for c in cubes]
    units = sum(c.N * c.B for c in cubes)
    nbytes = sum(c.N * c.B * 4 for c in cubes)
    steps = max(3, min(args.steps, 10))
    out = {"workload": BATCH_WORKLOAD, "tiles": len(cubes),
           "pixels": sum(c.N for c in cubes), "values": units, "cube_GB": nbytes / 1e9,
           "l2": "inputs (10 GB) larger than L2; no flush", "forms": {}}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    keep = {}
    for prec in ("mix", "p32"):
        b = g.Batch(Ys, 8, tol=1e-8, sweeps_max=30, precision=prec)
        for _ in range(args.warmup):
            b.run()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(steps):
            e0.record()
            b.run()
            e1.record()
            e1.synchronize()
            tot += e0.elapsed_time(e1) / 1e3
        ms = tot / steps * 1e3
        g.profile(True)
        b.run()
        torch.cuda.synchronize()
        stage = g.profile_collect()[0]
        g.profile(False)
        # the same run captured once into a CUDA graph and replayed
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            b.run(stream=side)
        stream.wait_stream(side)
        for _ in range(2):
            graph.replay()
        torch.cuda.synchronize()
        tg = 0.0
        for _ in range(steps):
            e0.record()
            graph.replay()
            e1.record()
            e1.synchronize()
            tg += e0.elapsed_time(e1) / 1e3
        status, infos = b.info()
        sw = [i["sweeps"] for i in infos]
        cov_ms, proj_ms = stage["covariance"], stage["project"]
        proj_bytes = nbytes + sum(c.N * 8 * 4 for c in cubes)
        out["forms"][prec] = {
            "ms": ms, "value": units / (ms / 1e3) / 1e6, "unit": UNIT,
            "graph_ms": tg / steps * 1e3, "graph_value": units / (tg / steps) / 1e6,
            "kernel_launches": b.kernel_launches(), "status": status,
            "sweeps_min": min(sw), "sweeps_max": max(sw), "sweeps_mean": float(np.mean(sw)),
            "stage_ms": stage,
            "covariance_GB/s": nbytes / (cov_ms / 1e3) / 1e9 if cov_ms > 0 else None,
            "covariance_frac": (nbytes / (cov_ms / 1e3) / 1e9 / peaks["hbm_gbs"]) if cov_ms > 0 else None,
            "project_GB/s": proj_bytes / (proj_ms / 1e3) / 1e9 if proj_ms > 0 else None,
            "project_frac": (proj_bytes / (proj_ms / 1e3) / 1e9 / peaks["hbm_gbs"]) if proj_ms > 0 else None,
            "peak_basis": peak_src}
        keep[prec] = b
        del graph
    # the plain FP32 form, tile after tile on one stream
    wss = [g.make_workspace(c.N, c.B, 8, 0, "p32", dev) for c in cubes]
    outs = [(torch.empty(c.B, dtype=torch.float64, device=dev),
             torch.empty(c.B, dtype=torch.float64, device=dev),
             torch.empty(c.B, c.B, dtype=torch.float64, device=dev),
             torch.empty(c.N, 8, dtype=torch.float32, device=dev)) for c in cubes]

    def sequential():
        for c, w, o in zip(cubes, wss, outs):
            g.fit(c.Y, 8, tol=1e-8, sweeps_max=30, precision="p32", out=o, workspace=w, sync=False)
    sequential()
    torch.cuda.synchronize()
    reps = 2
    e0.record()
    for _ in range(reps):
        sequential()
    e1.record()
    e1.synchronize()
    ms_seq = e0.elapsed_time(e1) / reps
    out["sequential_p32"] = {"ms": ms_seq, "value": units / (ms_seq / 1e3) / 1e6, "unit": UNIT,
                             "how": "pca_fit (P32) per tile, one stream"}
    for prec in ("mix", "p32"):
        out["forms"][prec]["speedup_vs_sequential_p32"] = ms_seq / out["forms"][prec]["ms"]
    # errors of sampled tiles against the FP64 oracle (smallest, median, largest N)
    import oracle
    oracle.set_threads(0)
    order = np.argsort([c.N for c in cubes])
    sample = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    errs = {}
    for prec, b in keep.items():
        e_rel, e_l1 = [], []
        for t in sample:
            ref = oracle.pca_fit(cubes[t].Y.cpu().numpy(), 8, tol=1e-14)
            lam = b.results[t][1].cpu().numpy()
            err = np.abs(lam[:8] - ref["lam"][:8])
            e_rel.append(float((err / np.abs(ref["lam"][:8])).max()))
            e_l1.append(float(err.max() / abs(ref["lam"][0])))
        errs[prec] = {"eig_rel_err_topk_max": max(e_rel), "eig_err_topk_over_lam1": max(e_l1)}
        b.close()
    out["errors_sampled_tiles"] = {"tiles": [cubes[t].name for t in sample], **errs}
    return out


# the shapes of the paper's Tables 4 and 5 (k = 1) and its GTX 680 times (ms, FP32,
# PCIe copies included) -- context only, another machine's numbers
PAPER_SHAPES = [("Jasper-shaped 512x614x224", 512, 614, 224, 216.78, "Table 5"),
                ("Cuprite-large-shaped 350x350x188", 350, 350, 188, 166.48, "Table 5"),
                ("Cuprite-small-shaped 250x191x188", 250, 191, 188, 148.68, "Table 5"),
                ("synthetic 100x100x50", 100, 100, 50, 69.19, "Table 4"),
                ("synthetic 500x500x50", 500, 500, 50, 89.25, "Table 4"),
                ("synthetic 300x300x100", 300, 300, 100, 87.68, "Table 4"),
                ("synthetic 300x300x200", 300, 300, 200, 160.48, "Table 4")]


def run_paper_shapes(args, dev):
    """k = 1 fits (the paper's setting) on scene-like cubes of the paper's shapes,
    FP32: device-resident and end to end from pinned host memory (the paper's times
    include the host-device copies)."""
    import torch

    import paper_2403_18321_gb300 as g
    import synth
    rows = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = max(3, min(args.steps, 10))
    for i, (name, r, c, B, paper_ms, src) in enumerate(PAPER_SHAPES):
        cube = synth.paper_scene(60 + i, r, c, B, k=1, name=name)
        Yh = torch.from_numpy(cube.Y).pin_memory()
        Y = Yh.to(dev)
        row = {"workload": name, "N": cube.N, "B": B, "k": 1, "paper_ms": paper_ms,
               "paper_source": src, "paper_hardware": "GTX 680, FP32"}
        for prec in ("mix", "p32"):
            ws = g.make_workspace(cube.N, B, 1, 0, prec, dev)
            for _ in range(3):
                g.fit(Y, 1, precision=prec, workspace=ws, sync=False)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                g.fit(Y, 1, precision=prec, workspace=ws, sync=False)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            # end to end: copy in, fit, copy the results out, synchronise
            t0 = time.perf_counter()
            for _ in range(reps):
                g.fit_host(Yh, 1, precision=prec, workspace=ws, device=dev)
            ms_e2e = (time.perf_counter() - t0) / reps * 1e3
            row[prec] = {"ms": ms, "Mpixel-bands/s": cube.N * B / (ms / 1e3) / 1e6,
                         "ms_e2e": ms_e2e, "cubes_per_s_e2e": 1e3 / ms_e2e}
        rows.append(row)
    return rows


def run_ncu_case(args):
    """Fits without timing, for ncu captures of single kernels (-k/-s/-c select them)."""
    import torch

    import paper_2403_18321_gb300 as g
    import synth
    g.load()
    if args.ncu_case == "backward":
        gc = synth.gradient_cube()
        Y = torch.from_numpy(gc.Y).cuda()
        dQ = torch.from_numpy(gc.meta["dQ"]).cuda()
        mu, ev, V, _, _ = g.fit(Y, gc.k, precision=args.precision)
        for _ in range(args.warmup + args.steps):
            dY = g.backward(Y, mu, ev, V, dQ)
        torch.cuda.synchronize()
        print(f"backward {gc.N}x{gc.B} k={gc.k}: |dY| max {dY.abs().max().item():.3e}")
        return 0
    if args.ncu_case in ("batched", "batched-small"):
        specs = synth.tile_batch_specs(seed=3)
        if args.ncu_case == "batched-small":
            specs = [(max(4096, n // 4), b, e, sd) for n, b, e, sd in specs[:48]]
        dev = torch.device("cuda")
        Ys = [synth.tile_device(sp, dev).Y for sp in specs]
        b = g.Batch(Ys, 8, tol=1e-8, sweeps_max=30, precision=args.precision)
        for _ in range(args.warmup + args.steps):
            b.run()
        status, infos = b.info()
        print(f"{len(Ys)} tiles, {sum(y.numel() for y in Ys) * 4 / 1e9:.2f} GB: status {status}, "
              f"{b.kernel_launches()} launches per run")
        b.close()
        return 0
    if args.ncu_case == "big":
        cubes = [synth.paper_scene(2, 1024, 400, 224)]
    else:
        cubes = synth.paper_scenes()
    for c in cubes:
        Y = torch.from_numpy(c.Y).cuda()
        ws = g.make_workspace(c.N, c.B, c.k, 0, args.precision)
        for _ in range(args.warmup + args.steps):
            info = g.fit(Y, c.k, tol=c.tol, sweeps_max=c.sweeps_max, precision=args.precision,
                         workspace=ws)[4]
        torch.cuda.synchronize()
        print(f"{c.name} N={c.N} B={c.B}: {info}")
    return 0


# ------------------------------------------------------------------ our arm
def main(argv=None):
    args = parse_args(argv)
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.ncu_case is not None:
        return run_ncu_case(args)
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return rc

    import torch

    import paper_2403_18321_gb300 as g
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g.load()
    if args.warmup < 3:
        args.warmup = 3

    cubes = synth.paper_scenes()
    units = sum(c.N * c.B for c in cubes)
    Yd = [torch.from_numpy(c.Y).to(dev) for c in cubes]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def setup(prec):
        ws = [g.make_workspace(c.N, c.B, c.k, 0, prec, dev) for c in cubes]
        outs = [(torch.empty(c.B, dtype=torch.float64, device=dev),
                 torch.empty(c.B, dtype=torch.float64, device=dev),
                 torch.empty(c.B, c.B, dtype=torch.float64, device=dev),
                 torch.empty(c.N, c.k, dtype=torch.float32, device=dev)) for c in cubes]
        return ws, outs

    # the cubes are independent problems: each gets its own stream, joined per
    # step; the cube with the longest fit (most bands: the Jacobi steps grow
    # with B) gets the higher priority, so that its launches take the SMs first
    # when both cubes' kernels are pending
    longest = max(range(len(cubes)), key=lambda i: cubes[i].B)
    side = [torch.cuda.Stream(device=dev, priority=-1 if i == longest else 0)
            for i in range(len(cubes))]

    def step(prec, ws, outs, Ys=None):
        Ys = Yd if Ys is None else Ys
        main = torch.cuda.current_stream(dev)
        fork = torch.cuda.Event()
        fork.record(main)
        joins = []
        for c, Y, w, o, st in zip(cubes, Ys, ws, outs, side):
            st.wait_event(fork)
            g.fit(Y, c.k, tol=c.tol, sweeps_max=c.sweeps_max, precision=prec, out=o, workspace=w,
                  sync=False, stream=st)
            ev = torch.cuda.Event()
            ev.record(st)
            joins.append(ev)
        for ev in joins:
            main.wait_event(ev)

    def timed(prec, steps, warmup, with_profile=False, sampler=None):
        ws, outs = setup(prec)
        for _ in range(warmup):
            step(prec, ws, outs)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        if with_profile:
            g.profile(True)
        total = 0.0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ctx = sampler if sampler is not None else _Null()
        with ctx:
            for _ in range(steps):
                flush.fill_(1)
                e0.record()
                step(prec, ws, outs)
                e1.record()
                e1.synchronize()
                total += e0.elapsed_time(e1) / 1e3
        stages = g.profile_collect() if with_profile else []
        if with_profile:
            g.profile(False)
        torch.cuda.synchronize()
        barrier(world)
        infos = []
        for c, Y, w, o in zip(cubes, Yd, ws, outs):
            infos.append(g.fit(Y, c.k, tol=c.tol, sweeps_max=c.sweeps_max, precision=prec, out=o,
                               workspace=w, sync=True)[4])
        torch.cuda.synchronize()
        res = [tuple(t.cpu().numpy() for t in o) for o in outs]
        return total, stages, infos, res

    peaks, peak_src = load_peaks()
    sampler = ClockSampler(local)
    t_mix, stages, infos_mix, res_mix = timed(args.precision, args.steps, args.warmup, True, sampler)
    t_mix = max_over_ranks(t_mix, world)
    value = aggregate(units, args.steps, t_mix, world)
    t_p32, _, infos_p32, res_p32 = timed("p32", args.steps, args.warmup, False, sampler)
    t_p32 = max_over_ranks(t_p32, world)
    value_p32 = aggregate(units, args.steps, t_p32, world)

    # ---- per-stage times over the timed region (events on the launching stream)
    nfit = len(cubes)
    per_cube = [[r for i, r in enumerate(stages) if i % nfit == j] for j in range(nfit)]
    stage_ms = {s: float(sum(np.mean([r[s] for r in pc]) for pc in per_cube if pc))
                for s in g.STAGES}
    dom = max(stage_ms, key=stage_ms.get)
    roof = None
    if dom == "jacobi":
        # one launch per cube; report the larger-B cube's launch (the dominant one)
        j = int(np.argmax([c.B for c in cubes]))
        c = cubes[j]
        ms = float(np.mean([r["jacobi"] for r in per_cube[j]]))
        flops = jacobi_flops(c.B, infos_mix[j]["sweeps"])
        mhz = float(peaks.get("sm_max_mhz", 2070.0))
        nsm = g.jacobi_sms(c.B)
        peak = SM_LANES_FP32 * 2 * mhz * 1e6 * nsm / 1e9     # GFLOP/s of the SMs the kernel holds
        ach = flops / (ms / 1e3) / 1e9
        roof = {"kernel": "k_jacobi_cluster", "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "GFLOP/s", "frac": ach / peak,
                "peak_basis": f"FP32 SIMT peak of the {nsm} SMs of the kernel's one cluster "
                              f"({SM_LANES_FP32} lanes x 2 x {mhz:.0f} MHz each, {peak_src} "
                              f"clock); the Jacobi steps are sequential, so the kernel is "
                              f"latency-bound by design",
                "frac_of_gpu": ach / (SM_LANES_FP32 * 2 * mhz * 1e6 * 152 / 1e9),
                "traffic": profiled_traffic("k_jacobi_cluster"),
                "launch_ms": ms, "cube": c.name, "sweeps": infos_mix[j]["sweeps"],
                "sweeps_per_s": infos_mix[j]["sweeps"] / (ms / 1e3),
                "us_per_step": ms * 1e3 / max(1, infos_mix[j]["steps"])}
    else:
        key = {"covariance": "k_syrk_tc", "project": "k_project"}.get(dom, dom)
        byts = sum(c.N * c.B * 4 for c in cubes) / nfit
        ms = stage_ms[dom] / nfit
        ach = byts / (ms / 1e3) / 1e9
        roof = {"kernel": key, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "peak_basis": peak_src,
                "traffic": profiled_traffic(key), "launch_ms": ms}
    # covariance and projection kernels against the HBM roofline (cube bytes per
    # launch).  Inside the step the two cubes' launches share the SMs (a launch
    # whose CTAs need a whole SM waits for the SMs the other cube's kernels
    # hold), so each kernel is also timed with its cube fitted alone.
    def alone_stage_ms(prec, reps=5):
        ws, outs = setup(prec)
        res = []
        for c, Y, w, o in zip(cubes, Yd, ws, outs):
            g.fit(Y, c.k, tol=c.tol, sweeps_max=c.sweeps_max, precision=prec, out=o, workspace=w,
                  sync=True)
            torch.cuda.synchronize()
            g.profile(True)
            for _ in range(reps):
                flush.fill_(1)
                g.fit(Y, c.k, tol=c.tol, sweeps_max=c.sweeps_max, precision=prec, out=o,
                      workspace=w, sync=False)
            torch.cuda.synchronize()
            recs = g.profile_collect()
            g.profile(False)
            res.append({s: float(np.mean([r[s] for r in recs])) for s in g.STAGES})
        return res

    alone = alone_stage_ms(args.precision)
    hbm = {}
    for s, key in (("covariance", "k_syrk_tc"), ("project", "k_project")):
        per = []
        for j, c in enumerate(cubes):
            ms = alone[j][s]
            byts = c.N * c.B * 4 + (c.N * c.k * 4 if s == "project" else 0)
            per.append({"cube": c.name, "ms": ms, "GB/s": byts / (ms / 1e3) / 1e9,
                        "frac": byts / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                        "ms_in_step": float(np.mean([r[s] for r in per_cube[j]]))})
        hbm[key] = per
    hbm["how"] = ("each cube fitted alone on one stream, L2 flushed before each fit, CUDA "
                  "events around the launch; ms_in_step: the same launch inside the two-stream "
                  "step, where it shares the SMs with the other cube's kernels")

    # ---- errors against the oracle, and the CPU baseline (rank 0, N = 1 only)
    errors = {}
    cpu = None
    if rank == 0:
        import oracle
        threads = oracle.set_threads(0)
        t0 = time.perf_counter()
        refs = [oracle.pca_fit(c.Y, c.k, tol=1e-14) for c in cubes]
        t_ref_first = time.perf_counter() - t0
        for name, res in (("mix", res_mix), ("p32", res_p32)):
            e, en = [], []
            for c, r, ref in zip(cubes, res, refs):
                lam = r[1]
                err = np.abs(lam[:c.k] - ref["lam"][:c.k])
                e.append(float((err / np.abs(ref["lam"][:c.k])).max()))
                en.append(float(err.max() / abs(ref["lam"][0])))
            # per eigenvalue, and normwise (relative to the largest eigenvalue)
            errors[name] = {"eig_rel_err_topk_max": max(e), "eig_err_topk_over_lam1": max(en)}
        if world == 1 and not args.no_cpu_baseline:
            reps, t_cpu = 0, 0.0
            while reps < 1 or (t_cpu < 10.0 and reps < 5):
                t0 = time.perf_counter()
                for c in cubes:
                    oracle.pca_fit(c.Y, c.k, tol=c.tol, sweeps_max=c.sweeps_max)
                t_cpu += time.perf_counter() - t0
                reps += 1
            cpu = {"value": units * reps / t_cpu / 1e6, "unit": UNIT, "cores": threads,
                   "kind": "oracle",
                   "sample": f"full workload (both cubes, all four stages) x {reps}, "
                             f"FP64, OpenMP on the pixel loops, serial Jacobi"}

    # ---- end to end from pinned host buffers through the public API
    e2e = None
    if not args.no_e2e:
        Yh = [torch.from_numpy(c.Y).pin_memory() for c in cubes]
        ws, outs = setup(args.precision)
        host_out = [tuple(torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in o) for o in outs]
        h2d = sum(y.numel() * 4 for y in Yh)
        d2h = sum(sum(t.numel() * t.element_size() for t in o) for o in outs)

        Yin = [torch.empty(y.shape, dtype=y.dtype, device=dev) for y in Yh]

        # the cube with the longest fit (most bands: Jacobi steps grow with B)
        # is copied in first, with the link to itself; the next cube's copy
        # starts when it is done and overlaps the first cube's kernels
        order = sorted(range(len(cubes)), key=lambda i: -cubes[i].B)

        def e2e_step():
            # each cube on its own stream: copy in, fit, copy the results out
            main = torch.cuda.current_stream(dev)
            prev = torch.cuda.Event()
            prev.record(main)
            joins = []
            for i in order:
                c, yh, yd, w, o, h, st = cubes[i], Yh[i], Yin[i], ws[i], outs[i], host_out[i], side[i]
                st.wait_event(prev)
                with torch.cuda.stream(st):
                    yd.copy_(yh, non_blocking=True)
                    prev = torch.cuda.Event()
                    prev.record(st)
                    g.fit(yd, c.k, tol=c.tol, sweeps_max=c.sweeps_max, precision=args.precision,
                          out=o, workspace=w, sync=False, stream=st)
                    for t, th in zip(o, h):
                        th.copy_(t, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(st)
                joins.append(ev)
            for ev in joins:
                main.wait_event(ev)
            main.synchronize()

        for _ in range(args.warmup):
            e2e_step()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        total = 0.0
        with sampler:
            for _ in range(args.steps):
                flush.fill_(1)
                e0.record()
                e2e_step()
                e1.record()
                e1.synchronize()
                total += e0.elapsed_time(e1) / 1e3
        total = max_over_ranks(total, world)
        e2e = {"value": aggregate(units, args.steps, total, world), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": total / args.steps * 1e3}

    # ---- differentiation form: forward + adjoint of the projection layer on the
    #      512 x 512 x 200 planted cube, k = 10, dQ ~ N(0, 1) (rank 0 only)
    diff = None
    if not args.no_diff and rank == 0:
        gc = synth.gradient_cube()
        Yg = torch.from_numpy(gc.Y).to(dev)
        dQg = torch.from_numpy(gc.meta["dQ"]).to(dev)
        wsg = g.make_workspace(gc.N, gc.B, gc.k, 0, args.precision, dev)
        outg = g.fit(Yg, gc.k, precision=args.precision, workspace=wsg)
        mu_g, ev_g, V_g = outg[0], outg[1], outg[2]
        for _ in range(args.warmup):
            g.fit(Yg, gc.k, precision=args.precision, workspace=wsg, sync=False)
            g.backward(Yg, mu_g, ev_g, V_g, dQg, sync=False)
        torch.cuda.synchronize()
        f0, f1, b1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        tf = tb = 0.0
        reps = max(3, min(args.steps, 10))
        for _ in range(reps):
            flush.fill_(1)
            f0.record()
            g.fit(Yg, gc.k, precision=args.precision, workspace=wsg, sync=False)
            f1.record()
            g.backward(Yg, mu_g, ev_g, V_g, dQg, sync=False)
            b1.record()
            b1.synchronize()
            tf += f0.elapsed_time(f1) / 1e3
            tb += f1.elapsed_time(b1) / 1e3
        tf, tb = tf / reps, tb / reps
        units_g = gc.N * gc.B
        diff = {"workload": "planted 512x512x200 FP32, k=10, dQ ~ N(0,1) (seed 40)",
                "forward_ms": tf * 1e3, "backward_ms": tb * 1e3,
                "value": units_g / (tf + tb) / 1e6, "unit": UNIT,
                "backward_value": units_g / tb / 1e6,
                "backward_bytes": 2 * gc.N * gc.B * 4 + 2 * gc.N * gc.k * 4 + gc.N * gc.B * 4,
                "backward_GB/s": (2 * gc.N * gc.B * 4 + 2 * gc.N * gc.k * 4 + gc.N * gc.B * 4) / tb / 1e9}

    shapes = None
    if not args.no_paper_shapes and rank == 0:
        shapes = run_paper_shapes(args, dev)

    # band-sequential input (the paper's GPU layout): the conversion to the
    # pixel-major layout, one read and one write of each scene cube
    bsq = None
    if rank == 0:
        Bq = [y.t().contiguous() for y in Yd]
        for _ in range(3):
            for y in Bq:
                g.bsq_to_bip(y)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps, tot = 10, 0.0
        for _ in range(reps):
            flush.fill_(1)        # the cubes (53 MB) would otherwise stay in L2
            e0.record()
            for y in Bq:
                g.bsq_to_bip(y)
            e1.record()
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        ms = tot / reps
        moved = sum(2 * y.numel() * 4 for y in Bq)
        bsq = {"what": "pca_bsq_to_bip of both scene cubes (read + write), L2 flushed before "
                       "each repetition", "ms": ms,
               "GB/s": moved / (ms / 1e3) / 1e9, "frac": moved / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
               "peak_basis": peak_src}
        del Bq

    batched = None
    if not args.no_batched and rank == 0:
        batched = run_batched(args, dev, peaks, peak_src)

    launches = g.kernel_launches(args.precision, True) * len(cubes) * args.steps
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_mix / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16x3-f32acc+f32+f64" if args.precision == "mix" else args.precision,
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": args.precision,
                       "cubes": [f"{c.name} N={c.N} B={c.B}" for c in cubes],
                       "units_per_step": units, "l2": "flushed by a 256 MiB write before each step",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "streams": "one CUDA stream per cube, joined every step"},
            "forms": {"mix": {"value": value, "ms_per_step": t_mix / args.steps * 1e3,
                              "sweeps": [i["sweeps"] for i in infos_mix], **errors.get("mix", {})},
                      "p32": {"value": value_p32, "ms_per_step": t_p32 / args.steps * 1e3,
                              "sweeps": [i["sweeps"] for i in infos_p32], **errors.get("p32", {})}},
            "stage_ms_per_step": stage_ms, "roofline": roof, "hbm_kernels": hbm,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": sampler.summary(),
            "differentiation": diff, "batched": batched, "paper_shapes_k1": shapes,
            "bsq_input": bsq}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


if __name__ == "__main__":
    sys.exit(main())

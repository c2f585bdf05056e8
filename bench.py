#!/usr/bin/env python
"""Throughput of the Jacobi-PCA hot path (one JSON line).

Headline workload (one step): the precision-form cube of the evaluation --
2048 x 2048 pixels x 224 bands, BF16 values in [0, 1], planted spectrum
(s_i = 0.7^(i-1) over 20 components above a 1e-3 floor), k = 20 -- fitted
end to end: band means + covariance, Jacobi eigen-decomposition, sort/sign,
projection.  The cube (1.88 GB) is larger than the L2, so no flush is needed.

Metric: Mpixel-bands/s = N*B / step time.  `value` is the mixed form
(tensor-core covariance + FP64 refinement) with the input resident in HBM;
the plain FP32 and the FP64-step forms are measured beside it on the same
cube, and the FP16 variant of the cube, each with its error against the FP64
oracle.  The same line carries the scene-shaped cubes (610x340x103 and
512x217x224, FP32, k = 10), the 100x100x128 mixing cube, the batched form
(256 tiles), the differentiation form and the paper's k = 1 table shapes.
`value` fits one cube at a time (the K steps back to back between two
synchronisations); `two_in_flight` gives the same fits two at a time on two
streams, and `e2e` the fits of a stream of host-resident cubes through
pca_fit_host with two calls in flight (with the one-at-a-time figure beside
it), every step copying its cube in and its results out.

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
WORKLOAD = ("precision form: planted 2048x2048x224 BF16 in [0,1], s_i=0.7^(i-1) over 20 "
            "components + 1e-3 floor, k=20, tol 1e-10")
SCENES = "paper-scene cubes 610x340x103 + 512x217x224, FP32, k=10"
SM_LANES_FP32 = 128          # FP32 lanes per SM (sm_103a)
NUM_SMS = 152
C2_SIDE, C2_BANDS, C2_K = 2048, 224, 20
ORACLE_SAMPLE_PIXELS = 1 << 18   # the oracle's bounded sample of the 2048^2 cube


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
    ap.add_argument("--no-scenes", action="store_true",
                    help="skip the scene-shaped cubes and the 100x100x128 cube")
    ap.add_argument("--ncu-case", choices=["scenes", "big", "c2", "c2-small", "batched",
                                           "batched-small", "backward"],
                    default=None,
                    help="untimed fits for profiler captures: 'scenes' = the scene cubes, "
                         "'big' = one 1024x400x224 scene cube (367 MB, larger than L2), "
                         "'c2' = the 2048x2048x224 BF16 cube, 'c2-small' = a 1024x1024x224 "
                         "BF16 cube of the same recipe (470 MB), "
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


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload`, from the ncu summary
    profiles/<kernel>_<workload>*.md ('traffic_bytes_per_launch: X'); None when
    there is no capture of the current kernel on that workload."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    for name in sorted(os.listdir(d)):
        if name.startswith(f"{kernel}_{workload}") and name.endswith(".md"):
            m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)",
                          open(os.path.join(d, name)).read())
            if m:
                return float(m.group(1))
    return None


def jacobi_flops(B: int, sweeps: int) -> float:
    """Algorithmic FP32 flops of the cyclic Jacobi on a symmetric B x B matrix:
    6 B^3 per sweep (every rotation of a pair updates two
    rows and two columns of the symmetric matrix, 6 flops per entry pair, and a
    sweep rotates B(B-1)/2 pairs)."""
    return 6.0 * float(sweeps) * float(B) ** 3


def fp32_peak_gflops(mhz: float, sms: int = NUM_SMS) -> float:
    """FP32 SIMT peak (FFMA = 2 flops per lane per clock) of `sms` SMs."""
    return SM_LANES_FP32 * 2 * mhz * 1e6 * sms / 1e9


# ------------------------------------------------------------------ reference arm (oracle)
def c2_oracle_sample(dtype: str = "bf16", pixels: int = ORACLE_SAMPLE_PIXELS):
    """The first `pixels` pixels of the 2048 x 2048 x 224 planted cube as the host
    generator draws it (same recipe as the device-drawn benchmark cube)."""
    import synth
    return synth.planted_spectrum(side=C2_SIDE, bands=C2_BANDS, dtype=dtype, pixels=pixels)


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores, on a bounded sample of the headline
    workload (the first 2^18 pixels of the 2048 x 2048 x 224 BF16 cube, all four
    stages), sized so that warm-up + timed fits end within a few minutes."""
    if rank != 0:
        return 0
    import oracle
    threads = oracle.set_threads(0)
    cube = c2_oracle_sample()
    Y = oracle.as_f64(cube.Y)
    t0 = time.perf_counter()
    oracle.pca_fit(Y, C2_K, tol=1e-10, sweeps_max=30)
    t_one = time.perf_counter() - t0
    budget = 150.0 / max(1, args.steps + args.warmup)
    rows = Y.shape[0]
    if t_one > budget:
        rows = max(4096, int(rows * budget / t_one))
    Ys = np.ascontiguousarray(Y[:rows])
    units_s = Ys.shape[0] * Ys.shape[1]
    for _ in range(args.warmup):
        oracle.pca_fit(Ys, C2_K, tol=1e-10, sweeps_max=30)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.pca_fit(Ys, C2_K, tol=1e-10, sweeps_max=30)
    dt = time.perf_counter() - t0
    value = units_s * args.steps / dt / 1e6
    samp = (f"first {rows} pixels (of 4,194,304) of the 2048x2048x224 BF16 planted cube, "
            f"all bands, all four stages, FP64, OpenMP on the pixel loops, serial Jacobi")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "units_per_step": units_s, "sample_pixels": rows},
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
    # the autotuner on this batch (MIX): its fastest parameters against the defaults
    from paper_2403_18321_gb300 import tune
    cache = os.path.join(tempfile.mkdtemp(prefix="gbpca_tune_"), "tuning.json")
    res = tune.tune_batch(Ys, 8, precision="mix", tol=1e-8, warmup=2, reps=5, path=cache)
    bt = g.Batch(Ys, 8, tol=1e-8, sweeps_max=30, precision="mix", tuning=tune.lookup(res["key"], cache))
    for _ in range(args.warmup):
        bt.run()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        e0.record()
        bt.run()
        e1.record()
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    status, _ = bt.info()
    bt.close()
    ms_t = tot / steps
    out["autotuned_mix"] = {"ms": ms_t, "value": units / (ms_t / 1e3) / 1e6, "unit": UNIT,
                            "untuned_ms": out["forms"]["mix"]["ms"], "status": status,
                            "params": res["params"], "candidates_timed": len(res["trials"]),
                            "tuning_seconds": res["seconds"],
                            "speedup_vs_untuned": out["forms"]["mix"]["ms"] / ms_t}
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
            # end to end through pca_fit_host: pinned host cube in, results out
            hb = g.HostFit(cube.N, B, 1, Yh.dtype, prec, dev)
            hout = (torch.empty(B, dtype=torch.float64).pin_memory(),
                    torch.empty(B, dtype=torch.float64).pin_memory(),
                    torch.empty(B, B, dtype=torch.float64).pin_memory(),
                    torch.empty(cube.N, 1, dtype=torch.float32).pin_memory())
            for _ in range(2):
                g.fit_host(Yh, 1, precision=prec, buffers=hb, out=hout, sync=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                g.fit_host(Yh, 1, precision=prec, buffers=hb, out=hout, sync=False)
                torch.cuda.current_stream(dev).synchronize()
            ms_e2e = (time.perf_counter() - t0) / reps * 1e3
            del hb
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
    if args.ncu_case in ("c2", "c2-small"):
        side = C2_SIDE if args.ncu_case == "c2" else C2_SIDE // 2
        c = synth.planted_spectrum_device(torch.device("cuda"), side=side, bands=C2_BANDS)
        ws = g.make_workspace(c.N, c.B, c.k, 1, args.precision)
        for _ in range(args.warmup + args.steps):
            info = g.fit(c.Y, c.k, tol=c.tol, sweeps_max=c.sweeps_max, precision=args.precision,
                         workspace=ws)[4]
        torch.cuda.synchronize()
        print(f"planted {side}x{side}x{C2_BANDS} bf16: {info}")
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


# ------------------------------------------------------------------ error reports
# the comparison rules of the parity tests, restated for the report: a leading
# component is compared individually when its relative gap to both neighbours
# is at least 1e3 eps of the form (P64: 1e-5, the gap below which its
# refinement treats a pair as part of a cluster)
EPS_FORM = {"p64": 1e-8, "mix": 1e-7, "p32": 1e-6}
LAM_TARGET = {"p64": 1e-10, "mix": 2e-5, "p32": 2e-3}
Q_TARGET = 1e-4


def fit_errors(gpu, ref, k, form):
    """Errors of one fit against the oracle's: eigenvalues per eigenvalue
    (separated components i <= k) and relative to lam_1, projection per
    component against that component's own scale; which components miss the
    targets (MIX 2e-5, P64 1e-10 per eigenvalue; 1e-4 projection)."""
    mu, lam, V, Q = gpu
    lam_ref = ref["lam"]
    l1 = abs(lam_ref[0])
    d = np.abs(np.diff(lam_ref)) / l1
    gaps = np.minimum(np.r_[np.inf, d], np.r_[d, np.inf])
    kk = min(k, lam_ref.shape[0])
    sep = gaps[:kk] >= 1e3 * EPS_FORM[form]
    rel = np.abs(lam[:kk] - lam_ref[:kk]) / np.abs(lam_ref[:kk])
    out = {"eig_rel_err_topk_max": float(rel[sep].max()) if sep.any() else None,
           "eig_err_topk_over_lam1": float(np.abs(lam[:kk] - lam_ref[:kk]).max() / l1),
           "eig_target": LAM_TARGET[form], "separated_components": int(sep.sum()),
           "mu_err": float(np.abs(mu - ref["mu"]).max() / np.abs(ref["mu"]).max())}
    miss = [[int(i + 1), float(lam_ref[i] / l1), float(rel[i])] for i in range(kk)
            if sep[i] and rel[i] > LAM_TARGET[form]]
    out["eig_target_met"] = not miss
    out["eig_components_over_target"] = miss       # [component, lam/lam_1, relative error]
    if Q is not None and ref.get("Q") is not None:
        qe = []
        for j in range(kk):
            if not sep[j]:
                continue
            sgn = 1.0 if np.dot(V[:, j], ref["V"][:, j]) >= 0 else -1.0
            scale = max(np.abs(ref["Q"][:, j]).max(), 1e-300)
            qe.append((j, float(np.abs(sgn * Q[:, j] - ref["Q"][:, j]).max() / scale)))
        out["q_err_max"] = max(e for _, e in qe) if qe else None
        out["q_err_per_component"] = [e for _, e in qe]
        out["q_target_met"] = all(e <= Q_TARGET for _, e in qe)
    return out


def exact_residuals(Y16, lam, V, k, chunk=1 << 18):
    """Full-size properties of a fit of a 16-bit cube, in FP64 on the host from
    the same values: band means against the exact means, and for j < k the
    eigen-residual |C v_j - lam_j v_j| / lam_1 and the Rayleigh quotient
    |v_j^T C v_j - lam_j| / lam_1 with the exact covariance C."""
    Yh = Y16.cpu()
    N, B = Yh.shape
    s = np.zeros(B)
    for n0 in range(0, N, chunk):
        s += Yh[n0:n0 + chunk].double().numpy().sum(axis=0)
    mu = s / N
    Vk = V[:, :k]
    CV = np.zeros((B, k))
    for n0 in range(0, N, chunk):
        X = Yh[n0:n0 + chunk].double().numpy() - mu[None, :]
        CV += X.T @ (X @ Vk)
    CV /= (N - 1)
    l1 = abs(lam[0])
    res = np.linalg.norm(CV - Vk * lam[None, :k], axis=0) / l1
    rq = np.abs(np.einsum("bj,bj->j", Vk, CV) - lam[:k]) / l1
    return mu, {"residual_max_over_lam1": float(res.max()),
                "rayleigh_max_over_lam1": float(rq.max()),
                "residuals_over_lam1": [float(x) for x in res]}


# ------------------------------------------------------------------ timing helpers
class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


def timed_fits(g, Y, k, prec, steps, warmup, world=1, sampler=None, profile=False, flush=None,
               tol=1e-10, sweeps_max=30):
    """steps fits of one device cube on the current stream, CUDA events around
    each; returns (seconds, per-fit stage dicts, info, host outputs)."""
    import torch
    N, B = Y.shape
    dev = Y.device
    dt = g._dtype_code(Y)
    ws = g.make_workspace(N, B, k, dt, prec, dev)
    out = (torch.empty(B, dtype=torch.float64, device=dev),
           torch.empty(B, dtype=torch.float64, device=dev),
           torch.empty(B, B, dtype=torch.float64, device=dev),
           torch.empty(N, k, dtype=torch.float32, device=dev))
    for _ in range(warmup):
        g.fit(Y, k, tol=tol, sweeps_max=sweeps_max, precision=prec, out=out, workspace=ws,
              sync=False)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    if profile:
        g.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    total = 0.0
    with (sampler if sampler is not None else _Null()):
        if flush is None:
            # the K steps back to back between two synchronisations (inputs
            # larger than L2)
            e0.record()
            for _ in range(steps):
                g.fit(Y, k, tol=tol, sweeps_max=sweeps_max, precision=prec, out=out, workspace=ws,
                      sync=False)
            e1.record()
            e1.synchronize()
            total = e0.elapsed_time(e1) / 1e3
        else:
            # an L2 flush before each step, outside the timed interval
            for _ in range(steps):
                flush.fill_(1)
                e0.record()
                g.fit(Y, k, tol=tol, sweeps_max=sweeps_max, precision=prec, out=out,
                      workspace=ws, sync=False)
                e1.record()
                e1.synchronize()
                total += e0.elapsed_time(e1) / 1e3
    stages = g.profile_collect() if profile else []
    if profile:
        g.profile(False)
    torch.cuda.synchronize()
    barrier(world)
    info = g.fit(Y, k, tol=tol, sweeps_max=sweeps_max, precision=prec, out=out, workspace=ws,
                 sync=True)[4]
    host = tuple(t.cpu().numpy().astype(np.float64) for t in out)
    del ws
    return total, stages, info, host


def two_in_flight(g, Y, k, prec, steps, warmup, tol=1e-10, sweeps_max=30):
    """A stream of fits of resident cubes with two in flight: fits alternate
    between two CUDA streams, each with its own workspace and outputs, and
    nothing waits between them, so one fit's Jacobi (one thread-block cluster)
    runs beside the other's streaming kernels.  Returns seconds for `steps`
    fits (CUDA events: the start on the current stream, the later of the two
    streams' ends)."""
    import torch
    N, B = Y.shape
    dev = Y.device
    dt = g._dtype_code(Y)
    sets = []
    for _ in range(2):
        ws = g.make_workspace(N, B, k, dt, prec, dev)
        out = (torch.empty(B, dtype=torch.float64, device=dev),
               torch.empty(B, dtype=torch.float64, device=dev),
               torch.empty(B, B, dtype=torch.float64, device=dev),
               torch.empty(N, k, dtype=torch.float32, device=dev))
        sets.append((ws, out))
    streams = (torch.cuda.Stream(dev), torch.cuda.Stream(dev))

    def run(n):
        cur = torch.cuda.current_stream(dev)
        p0 = torch.cuda.Event(enable_timing=True)
        p0.record(cur)
        for s_ in streams:
            s_.wait_event(p0)
        for i in range(n):
            ws, out = sets[i % 2]
            g.fit(Y, k, tol=tol, sweeps_max=sweeps_max, precision=prec, out=out, workspace=ws,
                  sync=False, stream=streams[i % 2])
        ends = []
        for s_ in streams:
            pe = torch.cuda.Event(enable_timing=True)
            pe.record(s_)
            ends.append(pe)
        for pe in ends:
            pe.synchronize()
        return max(p0.elapsed_time(pe) for pe in ends) / 1e3

    run(warmup)
    torch.cuda.synchronize()
    t = run(steps)
    del sets
    return t


def mean_stages(g, stages):
    if not stages:
        return {}
    return {s: float(np.mean([r[s] for r in stages])) for s in g.STAGES}


# ------------------------------------------------------------------ the headline workload
def run_c2(args, g, dev, peaks, peak_src, sampler, world, rank):
    """The 2048 x 2048 x 224 planted cube: headline form (timed, profiled,
    end to end), the other forms, the FP16 variant, errors."""
    import torch

    import oracle
    import synth
    c = synth.planted_spectrum_device(dev, dtype="bf16")
    Y, k = c.Y, C2_K
    N, B = Y.shape
    units = N * B
    s_in = 2
    res = {}
    # stage times from a profiled pass (CUDA events between the stages), the
    # step time from a pass without them
    _, stages, _, _ = timed_fits(g, Y, k, args.precision, args.steps, args.warmup, world,
                                 None, profile=True)
    t, _, info, host = timed_fits(g, Y, k, args.precision, args.steps, args.warmup, world,
                                  sampler, profile=False)
    t = max_over_ranks(t, world)
    res["headline"] = {"seconds": t, "stages": stages, "info": info, "host": host}
    forms = {args.precision: {"ms": t / args.steps * 1e3,
                              "value": aggregate(units, args.steps, t, world),
                              "sweeps": info["sweeps"], "stage_ms": mean_stages(g, stages)}}
    for prec in ("p32", "p64", "mix"):
        if prec in forms:
            continue
        steps = args.steps if prec != "p64" else max(3, min(args.steps, 5))
        tp, st, inf, _ = timed_fits(g, Y, k, prec, steps, 2, world,
                                    sampler if prec == "p32" else None, profile=True)
        tp = max_over_ranks(tp, world)
        forms[prec] = {"ms": tp / steps * 1e3, "value": aggregate(units, steps, tp, world),
                       "sweeps": inf["sweeps"], "steps_timed": steps,
                       "stage_ms": mean_stages(g, st)}
    # a stream of resident cubes, two fits in flight, without and with the SMs
    # that the streaming kernels leave to the other fit's Jacobi cluster
    tif = {}
    for reserve in (0, g.jacobi_sms(B)):
        prev = g.set_tuning({**g.tuning(), "stream_sms_reserve": int(reserve)})
        try:
            t2 = two_in_flight(g, Y, k, args.precision, args.steps, args.warmup)
        finally:
            g.set_tuning(prev)
        t2 = max_over_ranks(t2, world)
        tif[f"sms_reserved_{reserve}"] = {"ms_per_fit": t2 / args.steps * 1e3,
                                          "value": aggregate(units, args.steps, t2, world)}
    res["two_in_flight"] = {"unit": UNIT, **tif,
                            "how": "fits of the resident cube alternate between two CUDA streams, "
                                   "each with its own workspace and outputs, nothing waits "
                                   "between them; the tensor-core covariance and projection "
                                   "optionally leave the Jacobi cluster's SMs free "
                                   "(stream_sms_reserve)"}
    # the FP16 variant of the cube (mixed form)
    c16 = synth.planted_spectrum_device(dev, dtype="fp16")
    tf, st, inf, host16 = timed_fits(g, c16.Y, k, "mix", args.steps, 2, world, profile=True)
    tf = max_over_ranks(tf, world)
    forms["mix_fp16"] = {"ms": tf / args.steps * 1e3, "value": aggregate(units, args.steps, tf, world),
                         "sweeps": inf["sweeps"], "stage_ms": mean_stages(g, st)}
    # per-kernel HBM roofline of the two streaming kernels (headline form)
    hs = forms[args.precision]["stage_ms"]
    hbm = {}
    for stage, key, byts in (("covariance", "k_syrk_tc" if args.precision == "mix" else "k_syrk_simt",
                              N * B * s_in),
                             ("project", "k_project", N * B * s_in + 4 * N * k)):
        ms = hs.get(stage, 0.0)
        if ms > 0:
            gbs = byts / (ms / 1e3) / 1e9
            hbm[key] = {"ms": ms, "bytes": byts, "GB/s": gbs, "frac": gbs / peaks["hbm_gbs"],
                        "peak_basis": f"{peak_src} copy bandwidth"}
    errors = {}
    if rank == 0:
        # reduced cube (256 x 256 pixels, host generator) against the oracle, every form
        oracle.set_threads(0)
        for dtype in ("bf16", "fp16"):
            r = synth.planted_spectrum(side=256, dtype=dtype)
            ref = oracle.pca_fit(r.Y, k, tol=1e-14)
            for prec in (("mix", "p32", "p64") if dtype == "bf16" else ("mix",)):
                mu, ev, V, Q, _ = g.fit(r.Y.to(dev), k, tol=1e-10, sweeps_max=30, precision=prec)
                gpu = tuple(x.cpu().numpy().astype(np.float64) for x in (mu, ev, V, Q))
                errors[f"reduced_256x256_{dtype}_{prec}"] = fit_errors(gpu, ref, k, prec)
        # full size: exact-covariance residuals of the headline fit
        mu_ex, props = exact_residuals(Y, host[1], host[2], k)
        props["mu_err"] = float(np.abs(host[0] - mu_ex).max() / np.abs(mu_ex).max())
        errors[f"full_size_bf16_{args.precision}"] = props
        mu_ex, props = exact_residuals(c16.Y, host16[1], host16[2], k)
        props["mu_err"] = float(np.abs(host16[0] - mu_ex).max() / np.abs(mu_ex).max())
        errors["full_size_fp16_mix"] = props
    del c16
    # end to end through the C ABI with host buffers (pca_fit_host): the pinned
    # host cube goes in, the results come back to pinned host memory
    e2e = None
    if not args.no_e2e:
        Yh = Y.cpu().pin_memory()
        hb = g.HostFit(N, B, k, Yh.dtype, args.precision, dev)
        hout = (torch.empty(B, dtype=torch.float64).pin_memory(),
                torch.empty(B, dtype=torch.float64).pin_memory(),
                torch.empty(B, B, dtype=torch.float64).pin_memory(),
                torch.empty(N, k, dtype=torch.float32).pin_memory())
        h2d = Yh.numel() * Yh.element_size()
        d2h = sum(o.numel() * o.element_size() for o in hout)

        def e2e_step():
            g.fit_host(Yh, k, tol=1e-10, sweeps_max=30, precision=args.precision, buffers=hb,
                       out=hout, sync=False)
            torch.cuda.current_stream(dev).synchronize()

        # the same through the device-resident API with the copies around it, one
        # stream; timed step by step in alternation with the pca_fit_host steps, so
        # that both see the same state of the (shared) host memory path
        Yin = torch.empty_like(Y)
        ws = g.make_workspace(N, B, k, 1, args.precision, dev)
        outs = (torch.empty(B, dtype=torch.float64, device=dev),
                torch.empty(B, dtype=torch.float64, device=dev),
                torch.empty(B, B, dtype=torch.float64, device=dev),
                torch.empty(N, k, dtype=torch.float32, device=dev))

        def serial_step():
            Yin.copy_(Yh, non_blocking=True)
            g.fit(Yin, k, tol=1e-10, sweeps_max=30, precision=args.precision, out=outs,
                  workspace=ws, sync=False)
            for o, h in zip(outs, hout):
                h.copy_(o, non_blocking=True)
            torch.cuda.current_stream(dev).synchronize()

        for _ in range(args.warmup):
            e2e_step()
            serial_step()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        total, t_serial = 0.0, 0.0
        for _ in range(args.steps):
            with sampler:
                e0.record()
                e2e_step()
                e1.record()
                e1.synchronize()
            total += e0.elapsed_time(e1) / 1e3
            e0.record()
            serial_step()
            e1.record()
            e1.synchronize()
            t_serial += e0.elapsed_time(e1) / 1e3
        total = max_over_ranks(total, world)
        e2e = {"value": aggregate(units, args.steps, total, world), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": total / args.steps * 1e3,
               "how": "pca_fit_host: pinned host cube copied in 16 pixel ranges, each range's "
                      "covariance as its copy lands, the ranges' moments pooled, eigen stage, "
                      "each range's projection copied back while the next is projected; "
                      "synchronise"}
        t_serial = max_over_ranks(t_serial, world)
        # a stream of cubes, two in flight: the steps alternate between two CUDA
        # streams, each with its own device buffers and host outputs, and nothing
        # waits between steps, so the upload of one cube overlaps the eigen stage,
        # projection and download of the previous one (every step still copies its
        # cube in and its results out inside the timed region)
        hb2 = g.HostFit(N, B, k, Yh.dtype, args.precision, dev)
        hout2 = tuple(torch.empty(o.shape, dtype=o.dtype, pin_memory=True) for o in hout)
        pstreams = (torch.cuda.Stream(dev), torch.cuda.Stream(dev))
        pbufs = ((hb, hout), (hb2, hout2))

        def pipelined(nsteps):
            cur = torch.cuda.current_stream(dev)
            p0 = torch.cuda.Event(enable_timing=True)
            p0.record(cur)
            for ps in pstreams:
                ps.wait_event(p0)
            for i in range(nsteps):
                b, o = pbufs[i % 2]
                g.fit_host(Yh, k, tol=1e-10, sweeps_max=30, precision=args.precision, buffers=b,
                           out=o, sync=False, stream=pstreams[i % 2])
            ends = []
            for ps in pstreams:
                pe = torch.cuda.Event(enable_timing=True)
                pe.record(ps)
                ends.append(pe)
            for pe in ends:
                pe.synchronize()
            return max(p0.elapsed_time(pe) for pe in ends) / 1e3

        pipelined(args.warmup)
        barrier(world)
        with sampler:
            t_pipe = pipelined(args.steps)
        t_pipe = max_over_ranks(t_pipe, world)
        e2e.update({"value": aggregate(units, args.steps, t_pipe, world),
                    "ms_per_step": t_pipe / args.steps * 1e3,
                    "how": "pca_fit_host, a stream of cubes with two in flight: steps alternate "
                           "between two CUDA streams with their own device buffers and pinned host "
                           "outputs, nothing waits between steps; within a call the pinned host "
                           "cube is copied in 16 pixel ranges, each range's covariance runs as its "
                           "copy lands, the ranges' moments are pooled, eigen stage, each range's "
                           "projection is copied back while the next is projected",
                    "one_in_flight_ms_per_step": total / args.steps * 1e3,
                    "one_in_flight_value": aggregate(units, args.steps, total, world)})
        e2e["serial_copies_ms_per_step"] = t_serial / args.steps * 1e3
        del Yh, Yin, ws, hb, hb2, hout2
    res.update({"forms": forms, "hbm": hbm, "errors": errors, "e2e": e2e, "N": N, "B": B, "k": k,
                "units": units})
    return res


def roofline_of(g, c2, peaks, peak_src, prec):
    """The dominant kernel of the headline step against its roofline."""
    st = c2["forms"][prec]["stage_ms"]
    N, B, k = c2["N"], c2["B"], c2["k"]
    dom = max(st, key=st.get)
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    info = c2["headline"]["info"]
    if dom == "jacobi":
        ms = st["jacobi"]
        sweeps = info["sweeps"]
        flops = jacobi_flops(B, sweeps)
        peak = fp32_peak_gflops(mhz)
        ach = flops / (ms / 1e3) / 1e9
        nsm = g.jacobi_sms(B)
        Bp = B + (B & 1)
        steps = max(1, info["steps"])
        alu_us = flops / steps / (fp32_peak_gflops(mhz, nsm) * 1e3)   # per step, cluster SMs
        return {"kernel": "k_jacobi_cluster", "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "GFLOP/s", "frac": ach / peak,
                "peak_basis": f"FP32 SIMT peak of the whole GPU ({NUM_SMS} SMs x "
                              f"{SM_LANES_FP32} lanes x 2 flops x {mhz:.0f} MHz, clock from "
                              f"{peak_src} peaks); flops = 6 B^3 per sweep",
                "traffic": profiled_traffic("k_jacobi_cluster", "planted_2048x2048x224"),
                "launch_ms": ms, "sweeps": sweeps, "sweeps_per_s": sweeps / (ms / 1e3),
                "latency_model": {"steps": steps, "steps_per_sweep": Bp - 1 if Bp > 1 else 1,
                                  "us_per_step": ms * 1e3 / steps,
                                  "alu_us_per_step_on_cluster_sms": alu_us,
                                  "exchange_us_per_step": ms * 1e3 / steps - alu_us,
                                  "cluster_sms": nsm}}
    key = {"covariance": "k_syrk_tc" if prec == "mix" else "k_syrk_simt",
           "project": "k_project"}.get(dom, dom)
    byts = N * B * 2 + (4 * N * k if dom == "project" else 0)
    ms = st[dom]
    ach = byts / (ms / 1e3) / 1e9
    return {"kernel": key, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "peak_basis": f"{peak_src} copy",
            "traffic": profiled_traffic(key, "planted_2048x2048x224"), "launch_ms": ms}


# ------------------------------------------------------------------ scene cubes and the mixing cube
def run_scenes(args, g, dev, peaks, peak_src, world, rank):
    """The two scene-shaped FP32 cubes fitted side by side on two streams, every
    form, with errors and per-kernel HBM fractions; L2 flushed before each step."""
    import torch

    import oracle
    import synth
    cubes = synth.paper_scenes()
    units = sum(c.N * c.B for c in cubes)
    Yd = [torch.from_numpy(c.Y).to(dev) for c in cubes]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    longest = max(range(len(cubes)), key=lambda i: cubes[i].B)
    side = [torch.cuda.Stream(device=dev, priority=-1 if i == longest else 0)
            for i in range(len(cubes))]

    def setup(prec):
        ws = [g.make_workspace(c.N, c.B, c.k, 0, prec, dev) for c in cubes]
        outs = [(torch.empty(c.B, dtype=torch.float64, device=dev),
                 torch.empty(c.B, dtype=torch.float64, device=dev),
                 torch.empty(c.B, c.B, dtype=torch.float64, device=dev),
                 torch.empty(c.N, c.k, dtype=torch.float32, device=dev)) for c in cubes]
        return ws, outs

    def step(prec, ws, outs):
        main = torch.cuda.current_stream(dev)
        fork = torch.cuda.Event()
        fork.record(main)
        joins = []
        for c, Y, w, o, st in zip(cubes, Yd, ws, outs, side):
            st.wait_event(fork)
            g.fit(Y, c.k, tol=c.tol, sweeps_max=c.sweeps_max, precision=prec, out=o, workspace=w,
                  sync=False, stream=st)
            ev = torch.cuda.Event()
            ev.record(st)
            joins.append(ev)
        for ev in joins:
            main.wait_event(ev)

    out = {"workload": SCENES, "units_per_step": units,
           "l2": "flushed by a 256 MiB write before each step",
           "streams": "one CUDA stream per cube, joined every step", "forms": {}}
    results = {}
    for prec in ("mix", "p32", "p64"):
        ws, outs = setup(prec)
        steps = args.steps if prec != "p64" else max(3, min(args.steps, 10))
        for _ in range(args.warmup):
            step(prec, ws, outs)
        torch.cuda.synchronize()
        g.profile(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        total = 0.0
        for _ in range(steps):
            flush.fill_(1)
            e0.record()
            step(prec, ws, outs)
            e1.record()
            e1.synchronize()
            total += e0.elapsed_time(e1) / 1e3
        recs = g.profile_collect()
        g.profile(False)
        total = max_over_ranks(total, world)
        infos = [g.fit(Y, c.k, tol=c.tol, sweeps_max=c.sweeps_max, precision=prec, out=o,
                       workspace=w, sync=True)[4] for c, Y, w, o in zip(cubes, Yd, ws, outs)]
        results[prec] = [tuple(t.cpu().numpy().astype(np.float64) for t in o) for o in outs]
        nfit = len(cubes)
        per_cube = [[r for i, r in enumerate(recs) if i % nfit == j] for j in range(nfit)]
        out["forms"][prec] = {"ms_per_step": total / steps * 1e3,
                              "value": aggregate(units, steps, total, world),
                              "sweeps": [i["sweeps"] for i in infos],
                              "stage_ms": {c.name: mean_stages(g, pc)
                                           for c, pc in zip(cubes, per_cube)}}
    # per-kernel HBM fractions, each cube fitted alone (L2 flushed)
    hbm = {}
    for stage, key in (("covariance", "k_syrk_tc"), ("project", "k_project")):
        per = []
        ws, outs = setup("mix")
        for c, Y, w, o in zip(cubes, Yd, ws, outs):
            g.fit(Y, c.k, precision="mix", out=o, workspace=w, sync=True)
            g.profile(True)
            for _ in range(5):
                flush.fill_(1)
                g.fit(Y, c.k, tol=c.tol, sweeps_max=c.sweeps_max, precision="mix", out=o,
                      workspace=w, sync=False)
            torch.cuda.synchronize()
            recs = g.profile_collect()
            g.profile(False)
            ms = float(np.mean([r[stage] for r in recs]))
            byts = c.N * c.B * 4 + (c.N * c.k * 4 if stage == "project" else 0)
            per.append({"cube": c.name, "ms": ms, "GB/s": byts / (ms / 1e3) / 1e9,
                        "frac": byts / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]})
        hbm[key] = per
    out["hbm_kernels_alone"] = hbm
    if rank == 0:
        oracle.set_threads(0)
        refs = [oracle.pca_fit(c.Y, c.k, tol=1e-14) for c in cubes]
        out["errors"] = {prec: {c.name: fit_errors(r, ref, c.k, prec)
                                for c, r, ref in zip(cubes, results[prec], refs)}
                         for prec in results}
    del flush
    return out


def run_c0(args, g, dev, world, rank):
    """The 100 x 100 x 128 linear-mixing cube (k = 5): every form, errors."""
    import torch

    import oracle
    import synth
    c = synth.linear_mixing(seed=0)
    Y = torch.from_numpy(c.Y).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = {"workload": "linear mixing 100x100x128 FP32, 5 endmembers, k=5, tol 1e-10",
           "l2": "flushed by a 256 MiB write before each fit", "forms": {}}
    ref = oracle.pca_fit(c.Y, c.k, tol=1e-14) if rank == 0 else None
    for prec in ("mix", "p32", "p64"):
        t, _, info, host = timed_fits(g, Y, c.k, prec, args.steps, 3, world, flush=flush)
        out["forms"][prec] = {"ms": t / args.steps * 1e3,
                              "value": aggregate(c.N * c.B, args.steps, t, world),
                              "sweeps": info["sweeps"]}
        if ref is not None:
            out["forms"][prec]["errors"] = fit_errors(host, ref, c.k, prec)
    del flush
    return out


def oracle_timings(args):
    """The FP64 oracle as it stands on the host cores: all cores (OpenMP on the
    pixel loops) and one core, on the headline cube's bounded sample, the scene
    cubes and the mixing cube (Mpixel-bands/s of each)."""
    import oracle
    import synth
    out = {}
    ncores = oracle.set_threads(0)

    def rate(Y, k, min_s, max_reps):
        reps, t = 0, 0.0
        while reps < 1 or (t < min_s and reps < max_reps):
            t0 = time.perf_counter()
            oracle.pca_fit(Y, k, tol=1e-10, sweeps_max=30)
            t += time.perf_counter() - t0
            reps += 1
        return Y.shape[0] * Y.shape[1] * reps / t / 1e6, reps, t

    samp = c2_oracle_sample()
    Yc2 = oracle.as_f64(samp.Y)
    v, reps, t = rate(Yc2, C2_K, 10.0, 20)
    out["headline_sample"] = {"value": v, "unit": UNIT, "cores": ncores, "reps": reps,
                              "seconds": t, "pixels": int(Yc2.shape[0])}
    oracle.set_threads(1)
    Y1 = np.ascontiguousarray(Yc2[:1 << 16])
    v1, reps1, t1 = rate(Y1, C2_K, 0.0, 1)
    out["headline_sample_single_thread"] = {"value": v1, "unit": UNIT, "cores": 1,
                                            "seconds": t1, "pixels": int(Y1.shape[0])}
    c0 = synth.linear_mixing(seed=0)
    for threads, tag in ((0, "all_cores"), (1, "single_thread")):
        n = oracle.set_threads(threads)
        v, reps, t = rate(c0.Y, c0.k, 2.0, 20)
        out[f"mixing_100x100x128_{tag}"] = {"value": v, "unit": UNIT, "cores": n, "reps": reps}
    if not args.no_scenes:
        cubes = synth.paper_scenes()
        for threads, tag in ((0, "all_cores"), (1, "single_thread")):
            n = oracle.set_threads(threads)
            t0 = time.perf_counter()
            for c in cubes:
                oracle.pca_fit(c.Y, c.k, tol=1e-10, sweeps_max=30)
            t = time.perf_counter() - t0
            out[f"scenes_{tag}"] = {"value": sum(c.N * c.B for c in cubes) / t / 1e6,
                                    "unit": UNIT, "cores": n, "seconds": t}
    oracle.set_threads(0)
    return out


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
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g.load()
    if args.warmup < 3:
        args.warmup = 3
    peaks, peak_src = load_peaks()
    sampler = ClockSampler(local)

    c2 = run_c2(args, g, dev, peaks, peak_src, sampler, world, rank)
    t_head = c2["headline"]["seconds"]
    value = aggregate(c2["units"], args.steps, t_head, world)
    roof = roofline_of(g, c2, peaks, peak_src, args.precision)

    scenes = c0 = None
    if not args.no_scenes:
        scenes = run_scenes(args, g, dev, peaks, peak_src, world, rank)
        c0 = run_c0(args, g, dev, world, rank)

    cpu = timings = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        timings = oracle_timings(args)
        hs = timings["headline_sample"]
        cpu = {"value": hs["value"], "unit": UNIT, "cores": hs["cores"], "kind": "oracle",
               "sample": f"first {hs['pixels']} pixels of the 2048x2048x224 BF16 planted cube "
                         f"(host generator, same recipe), all four stages, FP64, OpenMP on the "
                         f"pixel loops, serial Jacobi, x{hs['reps']}",
               "single_thread": timings["headline_sample_single_thread"]}

    diff = None
    if not args.no_diff and rank == 0:
        import synth
        gc = synth.gradient_cube()
        Yg = torch.from_numpy(gc.Y).to(dev)
        dQg = torch.from_numpy(gc.meta["dQ"]).to(dev)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
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
        bwd_bytes = 2 * gc.N * gc.B * 4 + 2 * gc.N * gc.k * 4 + gc.N * gc.B * 4
        diff = {"workload": "planted 512x512x200 FP32, k=10, dQ ~ N(0,1) (seed 40)",
                "forward_ms": tf * 1e3, "backward_ms": tb * 1e3,
                "value": units_g / (tf + tb) / 1e6, "unit": UNIT,
                "backward_value": units_g / tb / 1e6, "backward_bytes": bwd_bytes,
                "backward_GB/s": bwd_bytes / tb / 1e9}
        del flush

    shapes = None
    if not args.no_paper_shapes and rank == 0:
        shapes = run_paper_shapes(args, dev)

    batched = None
    if not args.no_batched and rank == 0:
        batched = run_batched(args, dev, peaks, peak_src)

    launches = g.kernel_launches(args.precision, c2["k"]) * args.steps
    forms = c2["forms"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_head / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("bf16 in; f16 tensor products (x1, x3 when a lo part is non-zero), f32 "
                      "accumulation; f32 Jacobi; f64/double-float refinement"
                      if args.precision == "mix" else args.precision),
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": args.precision,
                       "cube": f"N={c2['N']} B={c2['B']} bf16 (drawn on the device)",
                       "k": c2["k"], "units_per_step": c2["units"],
                       "l2": "input (1.88 GB) larger than L2; no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "forms": forms, "stage_ms_per_step": forms[args.precision]["stage_ms"],
            "hbm_kernels": c2["hbm"], "errors": c2["errors"], "roofline": roof,
            "step_hbm_frac": (2 * c2["N"] * c2["B"] * 2 + 4 * c2["N"] * c2["k"])
            / (t_head / args.steps) / 1e9 / peaks["hbm_gbs"],
            "cpu_baseline": cpu, "oracle_timings": timings, "e2e": c2["e2e"],
            "two_in_flight": c2.get("two_in_flight"),
            "gpu_launches": launches, "clocks": sampler.summary(),
            "scenes": scenes, "mixing_100x100x128": c0, "differentiation": diff,
            "batched": batched, "paper_shapes_k1": shapes}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

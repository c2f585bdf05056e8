"""Autotuner of the batched form (many tiles in one go).

The batched plan splits the tiles' pixels over the CTAs of its persistent
launches by a cost model (a fixed cost per chunk plus a cost per band) and
gives every tile's Jacobi a thread-block cluster of some number of CTAs.  The
library ships measured defaults for both (pca_tuning in include/gbpca.h);
this module measures, on the GPU at hand and for a given batch, which values
of those parameters run fastest, and keeps the result in a JSON cache keyed
by the device, the input type and the precision form.  ``Batch(...)`` reads
the cache (``tuning="auto"``) and installs the cached values while it plans.

What is tuned (coordinate descent, one parameter at a time, each candidate
timed over whole batched runs with CUDA events; the best so far is kept):
  * the CTAs of the Jacobi cluster for every band bucket (32 bands wide) that
    occurs in the batch: every cluster size from the fewest CTAs that hold
    the matrix (fewer SMs per matrix, more matrices side by side) to 8 (the
    latency-oriented shape of the single-cube form for wide matrices);
  * the fixed per-chunk cost of the covariance and of the projection in the
    work split (half, the default, twice the default);
  * for the SIMT covariance forms, the work items per SM.
The accumulation-run length of the tensor-core covariance is an accuracy
parameter, not a speed one, and is never changed here.

Cache file: $GBPCA_TUNING_CACHE, else ~/.cache/gbpca/tuning.json.
"""
from __future__ import annotations

import json
import os
import time

CACHE_ENV = "GBPCA_TUNING_CACHE"
SPEED_KEYS = ("batch_jacobi_ctas", "batch_cov_tc_fixed", "batch_proj_fixed",
              "batch_cov_simt_fixed", "batch_simt_items_per_sm")
PREC_NAMES = {0: "p64", 1: "p32", 2: "mix"}
DTYPE_NAMES = {0: "f32", 1: "bf16", 2: "f16"}


def cache_path(path: str | None = None) -> str:
    if path:
        return path
    env = os.environ.get(CACHE_ENV)
    if env:
        return env
    return os.path.join(os.path.expanduser("~"), ".cache", "gbpca", "tuning.json")


def cache_key(device_name: str, sms: int, dtype_code: int, precision: int) -> str:
    return (f"{device_name}|sm{int(sms)}|{DTYPE_NAMES.get(int(dtype_code), dtype_code)}|"
            f"{PREC_NAMES.get(int(precision), precision)}")


def device_key(device, dtype_code: int, precision: int) -> str:
    import torch
    p = torch.cuda.get_device_properties(device)
    return cache_key(p.name, p.multi_processor_count, dtype_code, precision)


def load_cache(path: str | None = None) -> dict:
    p = cache_path(path)
    if not os.path.exists(p):
        return {}
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return {}
    return d if isinstance(d, dict) else {}


def lookup(key: str, path: str | None = None) -> dict | None:
    """The cached speed parameters for `key`, or None."""
    e = load_cache(path).get(key)
    if not isinstance(e, dict) or not isinstance(e.get("params"), dict):
        return None
    return {k: v for k, v in e["params"].items() if k in SPEED_KEYS}


def store(key: str, params: dict, meta: dict | None = None, path: str | None = None) -> str:
    p = cache_path(path)
    d = load_cache(p)
    d[key] = {"params": {k: v for k, v in params.items() if k in SPEED_KEYS}, **(meta or {})}
    os.makedirs(os.path.dirname(os.path.abspath(p)), exist_ok=True)
    tmp = f"{p}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)
    return p


class applied:
    """Context manager: installs speed parameters on top of the library's current
    tuning and restores the previous tuning on exit."""

    def __init__(self, params: dict | None):
        self.params = params

    def __enter__(self):
        from . import set_tuning, tuning
        self.prev = tuning()
        if self.params:
            set_tuning({**self.prev, **self.params})
        return self

    def __exit__(self, *exc):
        from . import set_tuning
        set_tuning(self.prev)
        return False


def _bucket(B: int) -> int:
    Bp = B + (B & 1)
    return min(7, max(0, (Bp - 1) // 32))


def _time_batch(cubes, k, tol, sweeps_max, precision, params, warmup, reps):
    import torch

    from . import Batch
    b = Batch(cubes, k, tol=tol, sweeps_max=sweeps_max, precision=precision, tuning=params)
    try:
        for _ in range(warmup):
            b.run()
        torch.cuda.synchronize()
        times = []
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for _ in range(reps):
            e0.record()
            b.run()
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        status, _ = b.info()
    finally:
        b.close()
    times.sort()
    return times[len(times) // 2], status


def tune_batch(cubes, k, precision="mix", tol: float = 1e-8, sweeps_max: int = 30,
               warmup: int = 2, reps: int = 5, path: str | None = None, write: bool = True):
    """Times candidate speed parameters of the batched form on these device
    cubes and returns {"key", "params", "ms", "default_ms", "trials"}; with
    write=True the best parameters go to the cache under the device key."""
    from . import _dtype_code, _prec_code, tuning_defaults
    prec = _prec_code(precision)
    dt = _dtype_code(cubes[0])
    key = device_key(cubes[0].device, dt, prec)
    base = {k_: v for k_, v in tuning_defaults().items() if k_ in SPEED_KEYS}
    trials = []
    t0 = time.perf_counter()

    def measure(params):
        ms, status = _time_batch(cubes, k, tol, sweeps_max, prec, params, warmup, reps)
        trials.append({"params": json.loads(json.dumps(params)), "ms": ms, "status": status})
        return ms if status in (0, 2) else float("inf")

    best = dict(base)
    best_ms = default_ms = measure(best)
    # Jacobi cluster CTAs, bucket by bucket (the largest bands first: they run longest)
    buckets = sorted({_bucket(int(c.shape[1])) for c in cubes}, reverse=True)
    from . import batch_jacobi_ctas
    for bk in buckets:
        Bs = [int(c.shape[1]) for c in cubes if _bucket(int(c.shape[1])) == bk]
        seen = {tuple(batch_jacobi_ctas(B, best["batch_jacobi_ctas"][bk]) for B in Bs)}
        for n in (1, 2, 3, 4, 5, 6, 7, 8):
            eff = tuple(batch_jacobi_ctas(B, n) for B in Bs)
            if eff in seen:          # the same clusters as a shape already timed
                continue
            seen.add(eff)
            cand = dict(best)
            ctas = list(best["batch_jacobi_ctas"])
            ctas[bk] = n
            cand["batch_jacobi_ctas"] = ctas
            ms = measure(cand)
            if ms < best_ms * 0.99:
                best, best_ms = cand, ms
    # work-split cost model
    knobs = [("batch_proj_fixed", (0.5, 2.0))]
    if prec == 2:
        knobs.insert(0, ("batch_cov_tc_fixed", (0.5, 2.0)))
    else:
        knobs.insert(0, ("batch_cov_simt_fixed", (0.5, 2.0)))
        knobs.append(("batch_simt_items_per_sm", (0.5, 2.0)))
    for name, factors in knobs:
        for f in factors:
            cand = dict(best)
            v = best[name] * f
            cand[name] = int(round(v)) if name == "batch_simt_items_per_sm" else v
            ms = measure(cand)
            if ms < best_ms * 0.99:
                best, best_ms = cand, ms
    out = {"key": key, "params": best, "ms": best_ms, "default_ms": default_ms,
           "trials": trials, "seconds": time.perf_counter() - t0}
    if write:
        out["cache"] = store(key, best, {"ms": best_ms, "default_ms": default_ms,
                                         "tiles": len(cubes)}, path)
    return out

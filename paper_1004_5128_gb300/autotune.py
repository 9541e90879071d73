"""Launch-geometry autotuner for the engine.

The engine's launch geometry (temporal block and its kind of update unit, threads per CTA,
memory terms per work unit, rows per TMA stage, ring stages, resident CTAs per SM) trades
parallelism against
per-unit overhead, and the best point depends on the grid size, the step count, the
history dtype and the memory mode.  `tune` times candidates on the GPU (CUDA events
around whole runs, so every step's work is included) by coordinate descent from the
library's defaults and caches the winner in a JSON file keyed by
(dtypes, memory mode, dimension, N bucket, K bucket).  `lookup` returns a cached
geometry (or {} when none is known); `FRD(..., **lookup(p, ...))` applies it.

Cache path: $FD_TUNE_CACHE, else ~/.cache/fd_tune.json.  When the cache has no entry for a
problem, `lookup` falls back to the table shipped with the package (tuned.json, measured on a
GB300 with this tuner), first by exact key, then by the nearest step-count bucket.

    python -m paper_1004_5128_gb300.autotune c2 c4 [--modes adaptive] [--budget 60] [--out tuned.json]
"""
from __future__ import annotations

import json
import math
import os
import time

import torch

from . import _lib as L
from .frd import FRD, FRDBatch

PARAMS = {
    "time_block": [0, 8, 16, 32, 64],
    "step_updates": [0, 1],
    "tile_threads": [128, 256, 512],
    "chunk_terms": [32, 64, 128, 256, 512, 1024, 2048],
    "stage_rows": [4, 8, 16],
    "stages": [2, 3, 4, 6],
    "ctas_per_sm": [1, 2, 3],
}


def cache_path() -> str:
    return os.environ.get("FD_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                                        "fd_tune.json"))


def _bucket(x: int) -> int:
    return 1 << max(0, int(math.ceil(math.log2(max(1, x)))))


def key(p: dict, state: str = "f32", hist: str | None = None, kahan: bool = False) -> str:
    N = p["nx"] * p["ny"] * p.get("nz", 1)
    return (f"{state}/{hist or state}/{'kahan' if kahan else 'plain'}/mode{p['mem_mode']}"
            f"/d{p['ndim']}/N{_bucket(N)}/K{_bucket(p['K'])}")


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(k: str, geo: dict, rate: float):
    d = _load()
    d[k] = {"geometry": geo, "terms_per_s": rate}
    os.makedirs(os.path.dirname(cache_path()), exist_ok=True)
    tmp = cache_path() + f".{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path())


SHIPPED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def _shipped() -> dict:
    try:
        with open(SHIPPED) as f:
            return json.load(f)
    except Exception:
        return {}


def lookup(p: dict, state: str = "f32", hist: str | None = None, kahan: bool = False) -> dict:
    """Tuned geometry for p: user cache, then the shipped table (nearest K bucket)."""
    k = key(p, state, hist, kahan)
    for table in (_load(), _shipped()):
        if k in table:
            return dict(table[k]["geometry"])
    prefix, kb = k.rsplit("/K", 1)
    best = None
    for table in (_load(), _shipped()):
        for kk, e in table.items():
            pre, b = kk.rsplit("/K", 1)
            if pre == prefix:
                d = abs(math.log2(int(b)) - math.log2(int(kb)))
                if best is None or d < best[0]:
                    best = (d, e)
        if best:
            return dict(best[1]["geometry"])
    return {}


def batch_key(probs: list, state: str = "f32") -> str:
    n = sum(p["nx"] * p["ny"] * p.get("nz", 1) for p in probs)
    k = max(p["K"] for p in probs)
    return f"batch/{state}/mode{probs[0]['mem_mode']}/n{len(probs)}/N{_bucket(n)}/K{_bucket(k)}"


def lookup_batch(probs: list, state: str = "f32") -> dict:
    k = batch_key(probs, state)
    for table in (_load(), _shipped()):
        if k in table:
            return dict(table[k]["geometry"])
    return {}


def _time_single(p, geo, reps, **kw) -> float:
    s = FRD(p, tuned=False, **kw, **geo)
    terms = s.geometry()["terms_total"]
    u0 = torch.from_numpy(p["u0"]).to(s.device, s.dtype)
    st = s.stream
    best = float("inf")
    for i in range(reps + 1):
        s.set_state(u0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        s.step(p["K"])
        b.record(st)
        if s.status() != 0:
            raise RuntimeError("engine error while tuning")
        if i:  # first run is a warm-up
            best = min(best, a.elapsed_time(b))
    s.close()
    return terms / (best / 1e3)


def _time_batch(probs, geo, reps, **kw) -> float:
    b = FRDBatch(probs, tuned=False, **kw, **geo)
    best = float("inf")
    u0 = [torch.from_numpy(p["u0"]).to(b.device, b.dtype) for p in probs]
    for i in range(reps + 1):
        for j, u in enumerate(u0):
            b.set_state(j, u)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        b.run()
        e1.record(b.stream)
        if b.status() != 0:
            raise RuntimeError("engine error while tuning")
        if i:
            best = min(best, e0.elapsed_time(e1))
    b.close()
    return 1e3 / best  # runs per second


def tune(p, state: str = "f32", hist: str | None = None, kahan: bool = False, reps: int = 2,
         budget_s: float = 60.0, batch: list | None = None, verbose: bool = False, **fixed) -> dict:
    """Coordinate descent over PARAMS from the defaults; returns and caches the best geometry.

    With `batch` (a list of problems) the whole batch launch is timed instead of `p` alone.
    Geometry options passed in `fixed` (e.g. time_block) are held at their value and kept in
    the result.
    """
    kw = dict(state=state, hist=hist, kahan=kahan)
    cur: dict = dict(fixed)
    timer = (lambda g: _time_batch(batch, g, reps, **kw)) if batch else \
        (lambda g: _time_single(p, g, reps, **kw))
    best = timer(cur)
    t_end = time.time() + budget_s
    improved = True
    while improved and time.time() < t_end:
        improved = False
        for name, values in PARAMS.items():
            if name in fixed:
                continue
            for v in values:
                if time.time() > t_end:
                    break
                cand = dict(cur)
                cand[name] = v
                if cand == cur:
                    continue
                try:
                    r = timer(cand)
                except (L.FdError, RuntimeError):
                    continue  # geometry not launchable (e.g. shared memory)
                if verbose:
                    print(f"  {cand} -> {r:.4g}")
                if r > best * 1.01:
                    best, cur, improved = r, cand, True
    _store(batch_key(batch, state) if batch else key(p, state, hist, kahan), cur, best)
    return cur


def _main():
    import argparse

    from . import synth
    ap = argparse.ArgumentParser(description="tune launch geometry for named workloads")
    ap.add_argument("workloads", nargs="+")
    ap.add_argument("--budget", type=float, default=60.0, help="seconds per run")
    ap.add_argument("--K", type=int, default=0)
    ap.add_argument("--modes", default="", help="comma-separated runs of each workload to tune")
    ap.add_argument("--out", default="", help="cache file (default: $FD_TUNE_CACHE or ~/.cache)")
    args = ap.parse_args()
    if args.out:
        os.environ["FD_TUNE_CACHE"] = os.path.abspath(args.out)
    for w in args.workloads:
        for name, p, kw in synth.workload_runs(w, args.K, args.modes):
            t0 = time.time()
            if isinstance(p, list):
                g = tune(None, batch=p, budget_s=args.budget, **kw)
            else:
                g = tune(p, budget_s=args.budget, **kw)
            print(f"{w}:{name} -> {g} ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    _main()

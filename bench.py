"""Benchmark: GL history terms/s of the GB300 engine (one JSON line on rank 0).

Default workload (c3, the largest configuration): 2-D 512x512 Dirichlet fractional
reaction-diffusion (gamma=0.6, f=u(1-u)-0.05u, S=0.1, seeded U[0,0.1] noise), 20000 steps of
full memory with BF16, FP16 and FP32 history.  One benchmark step = the three 20000-step runs
from u0.  Also reported, measured outside the timed region: each run's error against the FP64
oracle at 128x128 x 2000 steps and against the FP32-history run at full size, and the c5
forward + adjoint rate against a plain FP32 forward.  Other workloads:
  c1  1-D N=256, 1000 steps, full memory, FP64
  c2  2-D 256x256 no-flux, 5000 steps, full / short L=500 / adaptive a=10 memory, FP32
  c4  64 uneven instances in one persistent launch (full and adaptive memory)
  c5  128x128, 4000 steps: forward + checkpointed adjoint, against a plain FP32 forward
  c2cl config 2's adaptive schedule (a=10) in closed loop, tau 0.1 and 0.01, and open loop,
       on the per-step kernel, FP32

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
                  [--workload c2|c1|c3|c4|c5|c2cl] [--K k] [--modes a,b] [--geom k=v,...]

`--impl reference` times the FP64 CPU oracle on bounded samples of the same workload (the
oracle is the only reference this method has).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GL history terms/s and % of HBM roofline; fwd+adjoint steps/s vs plain FP32"
L2_BYTES = 129 * 1024 * 1024
HBYTES = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}

CONFIG_NAMES = {
    "c2": "2-D 256x256 no-flux, gamma=0.8, alpha=0.5, f=-0.1u, S=0.1, 8 Gaussians, 5000 steps x "
          "{full, short L=500, adaptive a=10}, FP32",
    "c1": "1-D N=256 Dirichlet, gamma=0.5, S=0.2, 1000 steps, full memory, FP64",
    "c3": "2-D 512x512 Dirichlet, gamma=0.6, alpha=1, f=u(1-u)-0.05u, S=0.1, U[0,0.1] noise, 20000 "
          "steps, full memory; history BF16, FP16 (row-tile scaled) and FP32 (row-tile scaled FP16 hi "
          "+ lo planes), blocks of 64 steps with the far rows on tcgen05 tensor cores; FP32 state and "
          "accumulation, FP64-generated weights",
    "c4": "64 instances (32 1-D N 64-4096, 32 2-D side 64-384), gamma~U[0.3,0.95], steps "
          "U{1000..8000}, one persistent launch (CUDA graph), {full, adaptive a=10}, FP32",
    "c5": "2-D 128x128 Dirichlet, gamma=0.7, alpha=0.8, f=-0.1u, 4000 steps, FP32: forward with "
          "checkpoints every 200 + reverse-time adjoint (grad gamma, alpha, react, u0) vs plain "
          "FP32 forward",
    "c2cl": "2-D 256x256 no-flux, gamma=0.8, alpha=0.5, f=-0.1u, S=0.1, 8 Gaussians, 5000 steps, "
            "adaptive a=10: closed loop (tau 0.1, 0.01; medians kept while the history's relative "
            "variation across their increment stays below tau) and open loop, per-step kernel, FP32",
}


def peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- workloads

def problems(name: str, K: int = 0, modes: str = ""):
    """[(run name, problem or list of problems, solver kwargs)] for a workload."""
    from paper_1004_5128_gb300 import synth
    return synth.workload_runs(name, K, modes)


def alg_bytes(geo: dict, p: dict, kw: dict) -> int:
    """History rows the launch's kernel must read plus, per step, the u read/write and the delta
    write.  Per-step kernel: every lag >= 1 of every step.  Temporally blocked kernel: the far rows
    once per block in the history's precision, plus each step's newest rows; with 16-bit history
    (and FP32 history kept as two FP16 planes for the tensor cores) those come from the FP32 ring,
    which every step also writes."""
    N = p["nx"] * p["ny"] * p.get("nz", 1)
    sh = HBYTES[kw.get("hist", kw.get("state", "f32"))]
    ss = 8 if kw.get("state") == "f64" else 4
    rows = geo.get("stream_rows_total", geo["hist_rows_total"])
    ring = sh != ss or bool(geo.get("far_tensor_cores"))
    if not geo.get("time_block") or not ring:
        return rows * N * sh + p["K"] * N * (2 * ss + sh)
    head = geo["head_rows_total"]
    return (rows - head) * N * sh + head * N * 4 + p["K"] * N * (2 * ss + sh + 4)


def code_hash(path: str) -> str:
    """SHA-256 of a C/C++/CUDA source with its comments and blank space removed: the code that
    the compiler sees, so that a comment edit does not count as a kernel change."""
    import hashlib
    import re
    text = open(path, encoding="utf-8").read()
    # string literals are kept whole (inline PTX holds no comment markers); comments go
    pattern = re.compile(r'"(?:\\.|[^"\\])*"|//[^\n]*|/\*.*?\*/', re.S)
    code = pattern.sub(lambda m: m.group(0) if m.group(0).startswith('"') else " ", text)
    return hashlib.sha256(" ".join(code.split()).encode()).hexdigest()


def measured_traffic(key: str, geometry: dict):
    """DRAM bytes (read + write) of one launch from an ncu capture stored in profiles/traffic.json,
    or None when there is none for this run, or when the kernel code (comments aside) or the
    launch geometry have changed since the counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            entries = json.load(f)["entries"]
        for e in entries:
            if e["key"] != key:
                continue
            if any(geometry.get(k) != v for k, v in e["geometry"].items()):
                continue
            if all(code_hash(os.path.join(ROOT, src)) == h for src, h in e["sources"].items()):
                return e["bytes"]
    except (OSError, KeyError, ValueError):
        return None
    return None


def _sample_terms(p, K):
    import oracle
    return sum(len(oracle.schedule(p["mem_mode"], p["mem_L"], p["mem_a"], p.get("adaptive_rule", 0),
                                   k)[0]) for k in range(K)) * p["nx"] * p["ny"] * p.get("nz", 1)


class SingleRun:
    def __init__(self, name, p, kw, geo, dev):
        import torch
        from paper_1004_5128_gb300 import FRD
        self.name, self.p, self.kw = name, p, kw
        self.s = FRD(p, device=dev, **kw, **geo)
        self.geo = self.s.geometry()
        self.terms = self.geo["terms_total"]
        self.alg = alg_bytes(self.geo, p, kw)
        self.u0 = torch.from_numpy(p["u0"]).to(dev, self.s.dtype)
        self.launches = 1
        if kw.get("closed_tau") is not None:
            # closed loop: the terms follow the decisions, counted on the device by one run
            self.launch()
            n, N = self.s.memory_terms(), p["nx"] * p["ny"] * p.get("nz", 1)
            self.terms = n * N
            rows = n - p["K"]  # lags >= 1
            self.geo = dict(self.geo, terms_total=self.terms, hist_rows_total=rows, stream_rows_total=rows)
            self.alg = alg_bytes(self.geo, p, kw)

    def launch(self):
        self.s.set_state(self.u0)
        self.s.step(self.p["K"])

    def status(self):
        return self.s.status()

    def e2e_prepare(self):
        import torch
        self.hin = torch.from_numpy(self.p["u0"]).to(self.s.dtype).pin_memory()
        self.hout = torch.empty_like(self.hin).pin_memory()
        return self.hin.numel() * self.hin.element_size(), self.hout.numel() * self.hout.element_size()

    def e2e_run(self):
        from paper_1004_5128_gb300 import _lib as L
        L.fd_set_state(self.s.h, self.hin.data_ptr())
        L.fd_run(self.s.h, self.p["K"], self.hout.data_ptr())


class BatchRun:
    def __init__(self, name, probs, kw, geo, dev):
        import torch
        from paper_1004_5128_gb300 import FRDBatch
        self.name, self.probs, self.kw = name, probs, kw
        self.b = FRDBatch(probs, device=dev, **kw, **geo)
        geos = [self.b.geometry(i) for i in range(len(probs))]
        self.geo = dict(geos[0])
        self.terms = sum(g["terms_total"] for g in geos)
        self.alg = sum(alg_bytes(g, p, kw) for g, p in zip(geos, probs))
        self.u0 = [torch.from_numpy(p["u0"]).to(dev, self.b.dtype) for p in probs]
        self.launches = 1

    def launch(self):
        for i, u in enumerate(self.u0):
            self.b.set_state(i, u)
        self.b.run()

    def status(self):
        return self.b.status()

    def e2e_prepare(self):
        import torch
        self.hin = [torch.from_numpy(p["u0"]).to(self.b.dtype).pin_memory() for p in self.probs]
        self.hout = [torch.empty_like(h).pin_memory() for h in self.hin]
        nb = sum(h.numel() * h.element_size() for h in self.hin)
        return nb, nb

    def e2e_run(self):
        from paper_1004_5128_gb300 import _lib as L
        for i, h in enumerate(self.hin):
            L.fd_batch_set_state(self.b.b, i, h.data_ptr())
        L.fd_batch_run(self.b.b)
        for i, h in enumerate(self.hout):
            L.fd_batch_get_state(self.b.b, i, h.data_ptr())
        if L.fd_batch_get_status(self.b.b) != 0:
            raise SystemExit("batch status error")


class AdjointRun:
    """Forward with checkpoints + fd_adjoint; also times a plain FP32 forward of the same problem."""

    def __init__(self, name, p, kw, geo, dev):
        import torch
        from paper_1004_5128_gb300 import FRD, synth
        self.name, self.p, self.kw = name, p, kw
        self.C = 200
        self.s = FRD(p, device=dev, keep_tape=True, ckpt_every=self.C, **kw, **geo)
        self.plain = FRD(p, device=dev, **kw, **geo)
        tgt = FRD(synth.config5(K=p["K"], target=True), device=dev, **kw)
        tgt.set_state(p["u0"])
        self.target = tgt.run(p["K"])
        tgt.close()
        self.geo = self.s.geometry()
        K, N = p["K"], p["nx"] * p["ny"] * p.get("nz", 1)
        fwd = self.geo["terms_total"]
        recompute = fwd - sum((k + 1) * N for k in range(self.C - 1, K, self.C))
        self.terms = fwd + recompute + fwd  # forward, segment recompute, adjoint (lags 0..q)
        self.alg = alg_bytes(self.geo, p, kw)
        self.u0 = torch.from_numpy(p["u0"]).to(dev, self.s.dtype)
        self.launches = 1 + 2 * ((K + self.C - 1) // self.C)

    def launch(self):
        self.s.set_state(self.u0)
        self.s.step(self.p["K"])
        dJ = self.s.state() - self.target
        self.grads = self.s.adjoint(dJ)

    def status(self):
        return self.s.status()

    def time_plain(self, reps=3):
        import torch
        best = float("inf")
        for _ in range(reps + 1):
            self.plain.set_state(self.u0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(self.plain.stream)
            self.plain.step(self.p["K"])
            b.record(self.plain.stream)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    def e2e_prepare(self):
        import torch
        self.hin = torch.from_numpy(self.p["u0"]).to(self.s.dtype).pin_memory()
        self.htgt = self.target.cpu().pin_memory()
        self.hout = torch.empty_like(self.hin).pin_memory()
        self.hdj = torch.empty_like(self.hin).pin_memory()
        nb = self.hin.numel() * self.hin.element_size()
        return 2 * nb, 2 * nb

    def e2e_run(self):
        from paper_1004_5128_gb300 import _lib as L
        L.fd_set_state(self.s.h, self.hin.data_ptr())
        L.fd_run(self.s.h, self.p["K"], self.hout.data_ptr())
        self.hdj.copy_(self.hout - self.htgt)
        L.fd_adjoint(self.s.h, self.hdj.data_ptr(), self.hout.data_ptr())


def _rel_inf(a, ref) -> float:
    a, ref = np.asarray(a, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(a - ref)) / max(np.max(np.abs(ref)), 1e-300))


def closed_loop_checks(runs, dev) -> dict:
    """Measured outside the timed region: each closed-loop run's kernel options on config 2's
    schedule at 64x64, 2000 steps, against the FP64 oracle's closed loop (field error, terms used
    and the oracle's closest decision to tau, relative), and the open-loop run against or_run."""
    import oracle
    from paper_1004_5128_gb300 import FRD, synth
    q = synth.config2(synth.MEM_ADAPTIVE, K=2000, n=64)
    out = {"tolerance": 1e-5, "errors": {}}
    for r in runs:
        s = FRD(q, device=dev, max_steps=q["K"], **r.kw)
        s.set_state(q["u0"])
        got = s.run(q["K"]).cpu().double().numpy()
        tau = r.kw.get("closed_tau")
        if tau is None:
            e = {"vs_oracle_64x64_K2000": _rel_inf(got, oracle.run(q, threads=0))}
        else:
            ref, n, mg = oracle.run_closed(q, tau, threads=0, margin=True)
            e = {"vs_oracle_64x64_K2000": _rel_inf(got, ref), "terms": s.memory_terms(),
                 "oracle_terms": n, "oracle_decision_margin": mg}
        s.close()
        out["errors"][r.name] = e
    return out


def side_measurements(runs, dev) -> dict:
    """Measured outside the timed region: each config-3 run's error against the FP64 oracle at
    the size it finishes in seconds (128x128, 2000 steps, same kernel options) and, at full size,
    against the FP32-history run; and the config-5 forward + checkpointed adjoint rate against a
    plain FP32 forward, with the gradients' error against the oracle's adjoint at 600 steps."""
    import torch

    import oracle
    from paper_1004_5128_gb300 import FRD, synth
    out = {"tolerance": {"bf16": 2e-3, "f16": 2e-3, "f32": 1e-5}}
    finals = {r.name: r.s.state().cpu().double().numpy() for r in runs if hasattr(r, "s")}
    q = synth.config3(n=128, K=2000)
    ref = oracle.run(q, threads=0)
    errs = {}
    for r in runs:
        s = FRD(q, device=dev, **r.kw)
        s.set_state(q["u0"])
        e = {"vs_oracle_128x128_K2000": _rel_inf(s.run(q["K"]).cpu().double().numpy(), ref)}
        s.close()
        if r.name != "f32" and "f32" in finals:
            e["vs_fp32_history_512x512_K20000"] = _rel_inf(finals[r.name], finals["f32"])
        errs[r.name] = e
    out["errors"] = errs

    a = AdjointRun("adjoint", synth.config5(), {}, {}, dev)
    a.launch()
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(a.s.stream)
        a.launch()
        e1.record(a.s.stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    plain = a.time_plain()
    K = a.p["K"]
    q5 = synth.config5(K=600)
    tgt = oracle.run(synth.config5(K=600, target=True), threads=0)
    s = FRD(q5, device=dev, keep_tape=True, ckpt_every=200)
    s.set_state(q5["u0"])
    uK = s.run(q5["K"])
    g = s.adjoint(uK - torch.as_tensor(tgt, device=uK.device, dtype=uK.dtype))
    s.close()
    go = oracle.adjoint(q5, tgt, threads=0)
    gerr = max(abs(g["dgamma"] - go["dgamma"]) / abs(go["dgamma"]), abs(g["dalpha"] - go["dalpha"]) / abs(go["dalpha"]),
               _rel_inf(g["du0"].cpu().numpy(), go["du0"]), _rel_inf(g["dreact"], go["dreact"]))
    out["adjoint"] = {"workload": CONFIG_NAMES["c5"], "fwd_adjoint_steps_per_s": K / (best / 1e3),
                      "plain_fp32_fwd_steps_per_s": K / (plain / 1e3), "fwd_adjoint_over_plain_fwd_time": best / plain,
                      "grad_error_vs_oracle_adjoint_K600": gerr, "tolerance": 1e-5}
    return out


def shard_runs(runs: list, ws: int, rank: int) -> tuple:
    """This rank's share of the workload: a batch's instances split over the ranks by
    parallel.shard (strong scaling: the ranks together run the one batch), single-instance runs
    as replicas (weak scaling: every rank runs the whole step)."""
    from paper_1004_5128_gb300 import parallel
    out, sharded = [], False
    for name, p, kw in runs:
        if isinstance(p, list) and ws > 1:
            p = [p[i] for i in parallel.shard(p, ws)[rank]]
            sharded = True
        out.append((name, p, kw))
    return out, sharded


def make_runs(args, dev, ws: int = 1, rank: int = 0):
    geo = {}
    for item in filter(None, args.geom.split(",")):
        k_, v_ = item.split("=")
        geo[k_] = int(v_)
    cls = {"c4": BatchRun, "c5": AdjointRun}.get(args.workload, SingleRun)
    runs, sharded = shard_runs(problems(args.workload, args.K, args.modes), ws, rank)
    return [cls(name, p, kw, geo, dev) for name, p, kw in runs], sharded


# ------------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1004_5128_gb300 import parallel

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    runs, sharded = make_runs(args, dev, ws, rank)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)

    def one_step(events=None):
        for r in runs:
            flush.fill_(1)
            if events is not None:
                events[r.name][0].record(stream)
            r.launch()
            if events is not None:
                events[r.name][1].record(stream)

    for _ in range(args.warmup):
        one_step()
    for r in runs:
        if r.status() != 0:
            raise SystemExit(f"engine status error in warm-up ({r.name})")
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    ev = {r.name: [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
          for r in runs}
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for i in range(args.steps):
        one_step({k: v[i] for k, v in ev.items()})
    t1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = parallel.max_over_ranks(t0.elapsed_time(t1))
    for r in runs:
        if r.status() != 0:
            raise SystemExit(f"engine status error in timed region ({r.name})")
    # every rank's terms (replicas: the same step on each; a sharded batch: its own instances)
    terms_step = parallel.sum_over_ranks(sum(r.terms for r in runs))
    value = terms_step * args.steps / (ms / 1e3)

    modes = {}
    for r in runs:
        per = float(np.mean([a.elapsed_time(b) for a, b in ev[r.name]]))
        g = r.geo
        modes[r.name] = dict(ms=per, terms=r.terms, terms_per_s=r.terms / (per / 1e3),
                             alg_bytes=r.alg, gbs=r.alg / (per / 1e3) / 1e9,
                             geometry={k: g.get(k) for k in ("tile_threads", "tiles", "chunk_terms",
                                                             "stage_rows", "stages", "ctas_per_sm",
                                                             "grid", "head_lags", "time_block", "block_updates",
                                                             "far_tensor_cores")})
        modes[r.name]["frac_of_measured_hbm"] = round(modes[r.name]["gbs"] / peaks()[0], 4)
    extra = {}
    if args.workload == "c5":
        r = runs[0]
        plain_ms = r.time_plain()
        K = r.p["K"]
        fa_ms = modes[r.name]["ms"]
        extra = {"fwd_adjoint_steps_per_s": K / (fa_ms / 1e3),
                 "plain_fp32_fwd_steps_per_s": K / (plain_ms / 1e3),
                 "fwd_adjoint_over_plain_fwd_time": fa_ms / plain_ms,
                 "grads": {k: v for k, v in r.grads.items() if k != "du0"}}
        # the roofline line is for the plain forward launch (one engine launch, timed alone)
        modes[r.name]["gbs"] = r.alg / (plain_ms / 1e3) / 1e9
        modes[r.name]["roofline_launch"] = "plain FP32 forward"
    if args.workload == "c3" and not args.no_extra and rank == 0:
        extra = side_measurements(runs, dev)
    if args.workload == "c2cl" and not args.no_extra and rank == 0:
        extra = closed_loop_checks(runs, dev)
    dom = max(modes, key=lambda k: modes[k]["ms"])
    peak, which = peaks()
    ach = modes[dom]["gbs"]
    gd = modes[dom]["geometry"]
    hist = next(r.kw.get("hist", r.kw.get("state", "f32")) for r in runs if r.name == dom)
    kname = (f"engine_tb_kernel<{gd['time_block']}, {hist} history"
             f"{', tensor-core far units' if gd.get('far_tensor_cores') else ''}>") \
        if gd.get("time_block") else "engine_kernel"
    traffic = None if (args.geom or args.K) else measured_traffic(f"{args.workload}:{dom}",
                                                                  modes[dom]["geometry"])
    roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(ach / peak, 4), "traffic": traffic,
            "kernel": f"{kname} ({dom}, one persistent launch per run)",
            "peak_source": f"{which} hbm_gbs (burst copy)"}

    e2e = None
    if not args.no_e2e:
        h2d = d2h = 0
        for r in runs:
            a, b = r.e2e_prepare()
            h2d += a
            d2h += b
        torch.cuda.synchronize()
        # the config-3 step is seconds long: its end-to-end leg times at most two steps
        k = max(1, min(args.steps, 2) if args.workload == "c3" else args.steps)
        w0 = time.perf_counter()
        for _ in range(k):
            for r in runs:
                r.e2e_run()
        torch.cuda.synchronize()
        we = parallel.max_over_ranks(time.perf_counter() - w0)
        e2e = {"value": terms_step * k / we, "unit": "terms/s",
               "h2d_bytes_per_step": int(parallel.sum_over_ranks(h2d)),
               "d2h_bytes_per_step": int(parallel.sum_over_ranks(d2h))}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(args)
    if rank == 0:
        kw0 = runs[0].kw
        dtype = "f64" if kw0.get("state") == "f64" else "f32"
        if args.workload == "c3":
            dtype = "f32 state and accumulation; bf16, f16 and f32 history"
        line = {
            "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic (seeded SplitMix64 inputs)",
            "config": {"workload": CONFIG_NAMES[args.workload] +
                       (f" [K={args.K}]" if args.K else "") + (f" [{args.modes}]" if args.modes else ""),
                       "l2": "a 258 MB L2 flush before every run; every run's history exceeds L2 "
                             "(config 3: 10.5 GB BF16/FP16, 21 GB FP32)",
                       "parallelism": (f"instances sharded over {ws} GPUs (parallel.shard)" if sharded
                                       else f"replicas x{ws}" if ws > 1 else "single GPU")},
            "modes": modes, "roofline": roof, "e2e": e2e,
            "gpu_launches": sum(r.launches for r in runs) * args.steps,
            "clocks": ck, "cpu_baseline": cpu,
        }
        line.update(extra)
        print(json.dumps(line))
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------------------- CPU oracle

def _oracle_sample(args, kp, threads):
    """(terms, seconds) of the oracle on the first kp steps of every run of the workload."""
    import oracle
    from paper_1004_5128_gb300 import synth
    terms, t = 0, 0.0
    for name, p, kw in problems(args.workload, args.K, args.modes):
        if args.workload == "c5":
            K = min(kp, p["K"])
            N = p["nx"] * p["ny"] * p.get("nz", 1)
            tgt = oracle.run(synth.config5(K=K, target=True), threads=threads)
            w = time.perf_counter()
            oracle.adjoint(p, tgt, K=K, threads=threads)
            t += time.perf_counter() - w
            terms += 2 * sum((k + 1) * N for k in range(K))
            continue
        for q in (p[:: max(1, len(p) // 8)] if isinstance(p, list) else [p]):
            K = min(kp, q["K"])
            if kw.get("closed_tau") is not None:
                w = time.perf_counter()
                n = oracle.run_closed(q, kw["closed_tau"], K=K, threads=threads)[1]
                t += time.perf_counter() - w
                terms += n * q["nx"] * q["ny"] * q.get("nz", 1)
                continue
            n = _sample_terms(q, K)
            w = time.perf_counter()
            oracle.run(q, K=K, threads=threads)
            t += time.perf_counter() - w
            terms += n
    return terms, t


def _oracle_budget(args, seconds):
    """Grow the sampled prefix until the oracle sample takes about `seconds`."""
    threads = os.cpu_count() or 1
    kmax = max(q["K"] for _, p, _ in problems(args.workload, args.K, args.modes)
               for q in (p if isinstance(p, list) else [p]))
    kp = 8
    while True:
        terms, t = _oracle_sample(args, kp, threads)
        if t > seconds / 4 or kp >= kmax:
            break
        kp = int(kp * max(1.5, min(4.0, math.sqrt(seconds / 4 / max(t, 1e-3)))))
    what = "every 8th instance" if args.workload == "c4" else "each run"
    return terms, t, threads, f"first {min(kp, kmax)} steps of {what}"


def cpu_baseline(args):
    terms, t, threads, desc = _oracle_budget(args, args.cpu_seconds)
    return {"value": terms / t, "unit": "terms/s", "cores": threads, "kind": "oracle",
            "sample": desc + f"; {terms:.3e} terms in {t:.1f} s, OpenMP over grid points"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    total_terms, total_t, desc, threads = 0, 0.0, "", 1
    for i in range(args.warmup + args.steps):
        terms, t, threads, desc = _oracle_budget(args, args.cpu_seconds)
        if i >= args.warmup:
            total_terms += terms
            total_t += t
    value = total_terms / total_t
    line = {
        "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_t / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded SplitMix64 inputs)", "impl": "reference",
        "config": {"workload": CONFIG_NAMES[args.workload], "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": "terms/s", "cores": threads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c3", "c1", "c2", "c4", "c5", "c2cl"])
    ap.add_argument("--no-extra", action="store_true", help="skip the error and adjoint side measurements")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--K", type=int, default=0, help="override the step count (profiling cases)")
    ap.add_argument("--modes", default="", help="comma list of runs to keep, e.g. full")
    ap.add_argument("--geom", default="", help="launch geometry overrides, e.g. chunk_terms=256")
    args = ap.parse_args()
    if args.impl == "reference":
        args.cpu_seconds = min(args.cpu_seconds, 8.0)
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

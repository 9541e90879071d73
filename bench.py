"""Benchmark: GL history terms/s of the GB300 engine (one JSON line on rank 0).

Default workload: 2-D 256x256 no-flux fractional reaction-diffusion (gamma=0.8,
alpha=0.5, f=-0.1u, S=0.1, eight seeded Gaussians), 5000 steps in each of the
three memory modes (full, short window 500, adaptive a=10), FP32 state and
history.  One benchmark step = the three 5000-step runs from u0.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
                  [--workload c2|c1|c3|c4|c5]

`--impl reference` times the FP64 CPU oracle on bounded samples of the same
workload (the oracle is the only reference this method has).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GL history terms/s and % of HBM roofline; fwd+adjoint steps/s vs plain FP32"
L2_BYTES = 129 * 1024 * 1024


def peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
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
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- workloads

def workload(name: str, K: int = 0, modes: str = ""):
    runs = _workload(name)
    if modes:
        keep = modes.split(",")
        runs = [r for r in runs if r[0] in keep]
    if K:
        for _, p, _ in runs:
            p["K"] = K
    return runs


def _workload(name: str):
    from paper_1004_5128_gb300 import synth
    if name == "c2":
        return [("full", synth.config2(synth.MEM_FULL), {}),
                ("short", synth.config2(synth.MEM_SHORT), {}),
                ("adaptive", synth.config2(synth.MEM_ADAPTIVE), {})]
    if name == "c1":
        return [("full", synth.config1(), {"state": "f64"})]
    if name == "c3":
        return [("bf16", synth.config3(), {"hist": "bf16", "kahan": True}),
                ("f16", synth.config3(), {"hist": "f16", "kahan": True}),
                ("f32", synth.config3(), {})]
    raise SystemExit(f"unknown workload {name}")


CONFIG_NAMES = {
    "c2": "2-D 256x256 no-flux, gamma=0.8, alpha=0.5, f=-0.1u, S=0.1, 8 Gaussians, 5000 steps x "
          "{full, short L=500, adaptive a=10}, FP32",
    "c1": "1-D N=256 Dirichlet, gamma=0.5, S=0.2, 1000 steps, full memory, FP64",
    "c3": "2-D 512x512 Dirichlet, gamma=0.6, f=u(1-u)-0.05u, 20000 steps, full memory, "
          "{BF16, FP16, FP32} history, FP32 (Kahan) accumulation",
}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1004_5128_gb300 import FRD

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    runs = []
    geo_over = {}
    for item in filter(None, args.geom.split(",")):
        k_, v_ = item.split("=")
        geo_over[k_] = int(v_)
    for name, p, kw in workload(args.workload, args.K, args.modes):
        s = FRD(p, device=dev, **kw, **geo_over)
        geo = s.geometry()
        runs.append(dict(name=name, p=p, kw=kw, solver=s, geo=geo,
                         u0=torch.from_numpy(p["u0"]).to(dev, s.dtype)))
    hist_bytes = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)

    def one_step(events=None):
        for r in runs:
            flush.fill_(1)
            s = r["solver"]
            s.set_state(r["u0"])
            if events is not None:
                events[r["name"]][0].record(stream)
            s.step(r["p"]["K"])
            if events is not None:
                events[r["name"]][1].record(stream)

    for _ in range(args.warmup):
        one_step()
    for r in runs:
        st = r["solver"].status()
        if st != 0:
            raise SystemExit(f"engine status {st} in warm-up ({r['name']})")
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    ev = {r["name"]: [[torch.cuda.Event(enable_timing=True) for _ in range(2)]
                      for _ in range(args.steps)] for r in runs}
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for i in range(args.steps):
        one_step({k: v[i] for k, v in ev.items()})
    t1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1)
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    for r in runs:
        if r["solver"].status() != 0:
            raise SystemExit(f"engine status error in timed region ({r['name']})")
    terms_step = sum(r["geo"]["terms_total"] for r in runs)
    value = ws * terms_step * args.steps / (ms / 1e3)

    # per-mode breakdown and the roofline of the dominant launch
    modes = {}
    for r in runs:
        per = [a.elapsed_time(b) for a, b in ev[r["name"]]]
        g = r["geo"]
        p = r["p"]
        N = p["nx"] * p["ny"]
        sh = hist_bytes[r["kw"].get("hist", r["kw"].get("state", "f32"))]
        ss = 8 if r["kw"].get("state") == "f64" else 4
        alg = g["hist_rows_total"] * N * sh + p["K"] * N * (2 * ss + sh)
        modes[r["name"]] = dict(ms=float(np.mean(per)), terms=g["terms_total"],
                                terms_per_s=g["terms_total"] / (np.mean(per) / 1e3),
                                alg_bytes=alg, gbs=alg / (np.mean(per) / 1e3) / 1e9,
                                geometry={k: g[k] for k in ("tile_threads", "tiles", "chunk_terms",
                                                            "stage_rows", "stages", "ctas_per_sm",
                                                            "grid")})
    dom = max(modes, key=lambda k: modes[k]["ms"])
    peak, which = peaks()
    ach = modes[dom]["gbs"]
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            traffic = json.load(open(tfile)).get(f"{args.workload}:{dom}")
        except Exception:
            traffic = None
    roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(ach / peak, 4), "traffic": traffic,
            "kernel": f"engine_kernel ({dom} mode, one persistent launch per run)",
            "peak_source": f"{which} hbm_gbs"}

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        import ctypes  # noqa: F401
        from paper_1004_5128_gb300 import _lib as L
        host_in = [torch.from_numpy(r["p"]["u0"]).to(r["solver"].dtype).pin_memory() for r in runs]
        host_out = [torch.empty_like(h).pin_memory() for h in host_in]
        torch.cuda.synchronize()
        k = max(1, args.steps)
        w0 = time.perf_counter()
        for _ in range(k):
            for r, hi, ho in zip(runs, host_in, host_out):
                L.fd_set_state(r["solver"].h, hi.data_ptr())
                L.fd_run(r["solver"].h, r["p"]["K"], ho.data_ptr())
        torch.cuda.synchronize()
        we = time.perf_counter() - w0
        if ws > 1:
            t = torch.tensor([we], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            we = float(t.item())
        e2e = {"value": ws * terms_step * k / we, "unit": "terms/s",
               "h2d_bytes_per_step": int(sum(h.numel() * h.element_size() for h in host_in)),
               "d2h_bytes_per_step": int(sum(h.numel() * h.element_size() for h in host_out))}

    launches = len(runs) * args.steps  # one persistent engine launch per run
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(args.workload, args.cpu_seconds, args.K, args.modes)
    if rank == 0:
        dtype = runs[0]["kw"].get("state", "f32")
        line = {
            "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"f32": "f32", "f64": "f64"}[dtype] if args.workload != "c3" else "f32 (bf16/f16 history)",
            "data": "synthetic (seeded SplitMix64 inputs)",
            "config": {"workload": CONFIG_NAMES[args.workload],
                       "l2": "inputs larger than L2 (1.3 GB history per full/adaptive run) and a "
                             "258 MB L2 flush before every run",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "modes": modes, "roofline": roof, "e2e": e2e, "gpu_launches": launches,
            "clocks": ck, "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------------------- CPU oracle

def _oracle_sample(name, seconds, K=0, modes=""):
    """Run the oracle on the first K' steps of each run of the workload, K' grown until the
    whole sample takes about `seconds`.  Returns (terms, wall seconds, description)."""
    import oracle
    runs = workload(name, K, modes)
    threads = os.cpu_count() or 1
    kp = 8
    while True:
        terms, t = 0, 0.0
        for rname, p, kw in runs:
            K = min(kp, p["K"])
            N = p["nx"] * p["ny"]
            n = sum(len(oracle.schedule(p["mem_mode"], p["mem_L"], p["mem_a"],
                                        p.get("adaptive_rule", 0), k)[0]) for k in range(K))
            w = time.perf_counter()
            oracle.run(p, K=K, threads=threads)
            t += time.perf_counter() - w
            terms += n * N
        if t > seconds / 4 or kp >= max(p["K"] for _, p, _ in runs):
            break
        kp = int(kp * max(1.5, min(4.0, math.sqrt(seconds / 4 / max(t, 1e-3)))))
    return terms, t, threads, f"first {kp} steps of each run ({', '.join(r[0] for r in runs)})"


def cpu_baseline(name, seconds, K=0, modes=""):
    terms, t, threads, desc = _oracle_sample(name, seconds, K, modes)
    return {"value": terms / t, "unit": "terms/s", "cores": threads, "kind": "oracle",
            "sample": desc + f"; {terms:.3e} terms in {t:.1f} s, OpenMP over grid points"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    vals = []
    desc = ""
    total_t = 0.0
    for i in range(args.warmup + args.steps):
        terms, t, threads, desc = _oracle_sample(args.workload, args.cpu_seconds, args.K, args.modes)
        if i >= args.warmup:
            vals.append((terms, t))
            total_t += t
    terms = sum(v[0] for v in vals)
    value = terms / total_t
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
    ap.add_argument("--workload", default="c2", choices=["c2", "c1", "c3"])
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

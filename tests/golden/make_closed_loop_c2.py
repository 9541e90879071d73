"""Writes closed_loop_c2.json: the FP64 oracle's closed-loop adaptive memory (the reading of the
Discussion, Section 4) on the config-2 problem at full size (256 x 256 no-flux, 5000 steps,
adaptive a = 10) for tau = 0.1 and 0.01.  For each tau it stores the memory terms used, the
decisions' closest relative distance to tau, max |u^K| and u^K at 64 seeded sample points.

Calls only the oracle; takes several minutes per tau on a few cores:
    python tests/golden/make_closed_loop_c2.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1004_5128_gb300 import synth  # noqa: E402


def main():
    p = synth.config2(synth.MEM_ADAPTIVE)
    N = p["nx"] * p["ny"]
    idx = sorted(set(int(i) for i in np.floor(synth.SplitMix64(77).uniform(64, 0, N))))
    out = {"problem": "config 2, adaptive a=10, PAPER rule, 256x256, 5000 steps", "samples": idx, "runs": {}}
    for tau in (0.1, 0.01):
        u, n, margin = oracle.run_closed(p, tau, margin=True)
        out["runs"][str(tau)] = {"terms": n, "margin": margin, "max_abs": float(np.max(np.abs(u))),
                                 "values": [float(u[i]) for i in idx]}
        print(tau, n, margin, flush=True)
    with open(os.path.join(HERE, "closed_loop_c2.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

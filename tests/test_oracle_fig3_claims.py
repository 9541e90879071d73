"""The qualitative claims of Section 3.2 about the Fig. 3 experiment, checked on the FP64
oracle (20x20 grid, U_{10,10} = 10, alpha = 1, beta = 0, dt = 1, dx = 10, 1500 steps):

* adaptive memory has a lower error than short memory at the same cost (memory terms stand in
  for run time, which the oracle does not model);
* increasing L or a lowers the error (end points of each sweep);
* the short-memory error is larger for gamma nearer 1 when the window approaches t.
"""
import numpy as np
import pytest

import oracle
from paper_1004_5128_gb300 import experiments as E
from paper_1004_5128_gb300 import synth


def terms(mode, L, a, K=1500):
    return sum(len(oracle.schedule(mode, L, a, 0, k)[0]) for k in range(K))


@pytest.fixture(scope="module")
def runs():
    out = {}
    for g in (0.5, 0.9):
        ref = oracle.run(E.fig3_problem(g))
        for L in (50, 100, 1200):
            u = oracle.run(E.fig3_problem(g, synth.MEM_SHORT, L=L))
            out[(g, "short", L)] = (terms(synth.MEM_SHORT, L, 0), E.percent_errors(u, ref))
        for a in (2, 3, 50):
            u = oracle.run(E.fig3_problem(g, synth.MEM_ADAPTIVE, a=a))
            out[(g, "adaptive", a)] = (terms(synth.MEM_ADAPTIVE, 0, a), E.percent_errors(u, ref))
    return out


@pytest.mark.parametrize("g", [0.5, 0.9])
def test_adaptive_beats_short_at_equal_cost(runs, g):
    # each adaptive run against the cheapest short run that costs at least as much
    for a in (2, 3, 50):
        ca, ea = runs[(g, "adaptive", a)]
        costlier = sorted(runs[(g, "short", L)] for L in (50, 100, 1200) if runs[(g, "short", L)][0] >= ca)
        assert costlier, a
        cs, es = costlier[0]
        assert ea["max_point_pct"] < es["max_point_pct"] and ea["l2_pct"] < es["l2_pct"]


@pytest.mark.parametrize("g", [0.5, 0.9])
def test_longer_memory_lowers_error(runs, g):
    assert runs[(g, "short", 1200)][1]["l2_pct"] < runs[(g, "short", 50)][1]["l2_pct"]
    assert runs[(g, "adaptive", 50)][1]["l2_pct"] < runs[(g, "adaptive", 2)][1]["l2_pct"]


def test_short_memory_error_grows_toward_gamma_one_for_long_windows(runs):
    assert runs[(0.9, "short", 1200)][1]["max_point_pct"] > runs[(0.5, "short", 1200)][1]["max_point_pct"]


def test_fig1_problem_layout():
    p = E.fig1_problem(0.75)
    u = p["u0"].reshape(100, 100)
    assert u[50, 50] == 0.1 and u[50, 51] == u[49, 50] == 0.05 and u.sum() == pytest.approx(0.3)
    assert p["K"] * p["dt"] == 100.0

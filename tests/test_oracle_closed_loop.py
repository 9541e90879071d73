"""Pins of the oracle's closed-loop adaptive memory (a reading of the Discussion: the backward
sum's spacing follows the derivative of the past history).  A median keeps standing for its
increment only while the history's relative variation across the increment is below tau."""
import math

import numpy as np
import pytest

import oracle
from paper_1004_5128_gb300 import synth


def base(a=3, rule=synth.ADAPT_PAPER, K=160, gamma=0.75):
    p = synth.problem(2, 13, 11, gamma, 0.7, synth.dt_for_courant(0.12, 0.7, 1.0, gamma), 1.0,
                      synth.BC_NOFLUX, react=(0.01, -0.2, 0.3, -0.4), mem_mode=synth.MEM_ADAPTIVE,
                      mem_a=a, adaptive_rule=rule, K=K, u0=synth.SplitMix64(19).uniform(13 * 11, 0, 1))
    return p


def schedule_terms(p):
    return sum(len(oracle.schedule(p["mem_mode"], p["mem_L"], p["mem_a"], p["adaptive_rule"], k)[0])
               for k in range(p["K"]))


@pytest.mark.parametrize("a,rule", [(2, synth.ADAPT_PAPER), (3, synth.ADAPT_PAPER), (3, synth.ADAPT_PARTITION)])
def test_infinite_threshold_is_the_papers_rule(a, rule):
    """No feedback: every median stands for its increment, as in Proposition 3.1."""
    p = base(a, rule)
    u, n = oracle.run_closed(p, math.inf)
    assert np.array_equal(u, oracle.run(p))
    assert n == schedule_terms(p)


@pytest.mark.parametrize("a", [2, 3, 5])
def test_zero_threshold_with_partition_is_full_memory(a):
    """Every increment is summed lag by lag; the partition rule's increments tile the lags once,
    so the sum is full memory's, in the same ascending order."""
    p = base(a, synth.ADAPT_PARTITION)
    u, n = oracle.run_closed(p, 0.0)
    assert np.array_equal(u, oracle.run(synth.with_mode(p, synth.MEM_FULL)))
    assert n == p["K"] * (p["K"] + 1) // 2


def test_terms_grow_as_the_threshold_falls():
    p = base(3, synth.ADAPT_PARTITION, K=200)
    counts = [oracle.run_closed(p, tau)[1] for tau in (math.inf, 1.0, 0.3, 0.1, 0.03, 0.0)]
    assert all(x <= y for x, y in zip(counts, counts[1:]))
    assert counts[0] < counts[-1]


def test_feedback_rescues_oscillating_superdiffusion():
    """Superdiffusion (gamma = 1.3) of a single high mode oscillates in time, the fast-evolving
    history the Discussion warns about.  The open-loop medians alias the oscillation and the run
    blows up; the feedback expands the increments across it and stays within 1e-2 of full memory
    (5e-3 at the smaller threshold), at the cost of more terms."""
    p = synth.problem(1, 31, 1, 1.3, 1.0, synth.dt_for_courant(0.6 * synth.stability_bound(1.3, 1), 1.0, 1.0, 1.3),
                      1.0, synth.BC_DIRICHLET0, mem_mode=synth.MEM_ADAPTIVE, mem_a=3,
                      adaptive_rule=synth.ADAPT_PARTITION, K=400)
    p["u0"] = synth.eigenmode(p, 25)
    ref = oracle.run(synth.with_mode(p, synth.MEM_FULL))
    scale = np.max(np.abs(ref))

    def err(tau):
        u, n = oracle.run_closed(p, tau)
        return np.max(np.abs(u - ref)) / scale, n

    e_open, n_open = err(math.inf)
    e1, n1 = err(0.03)
    e2, n2 = err(0.01)
    assert e_open > 1.0
    assert e1 < 1e-2 and e2 < 5e-3
    assert n_open < n1 <= n2 <= p["K"] * (p["K"] + 1) // 2


def test_decision_margin():
    """The margin is the distance of the closest decision to the threshold, relative to it: no
    decision at tau = inf, and a threshold placed on a decision's own ratio has margin 0 there."""
    p = base(3, synth.ADAPT_PARTITION, K=120)
    assert oracle.run_closed(p, math.inf, margin=True)[2] == math.inf
    u, n, mg = oracle.run_closed(p, 0.2, margin=True)
    assert 0.0 < mg < math.inf
    # moving the threshold by less than the margin keeps every decision (same terms, same field)
    u2, n2, _ = oracle.run_closed(p, 0.2 * (1 + 0.5 * mg), margin=True)
    assert n2 == n and np.array_equal(u2, u)
    # moving it by more than the margin flips at least the closest decision
    u3, n3, _ = oracle.run_closed(p, 0.2 * (1 + 1.5 * mg), margin=True)
    u4, n4, _ = oracle.run_closed(p, 0.2 * (1 - 1.5 * mg), margin=True)
    assert n3 != n or n4 != n


@pytest.mark.parametrize("a", [2, 3, 5, 10])
@pytest.mark.parametrize("rule", [synth.ADAPT_PAPER, synth.ADAPT_PARTITION])
def test_increments_start_above_the_base_interval(a, rule):
    """Every increment a median stands for lies at lags >= a + 1 (both rules), so the decisions of
    step k read rows up to k - a - 1 only: the GPU decides step k once row k - a - 1 is complete
    everywhere.  Increment lengths stay far below 256 (the GPU keeps them in one byte)."""
    for k in (a + 3, 50, 400, 3000):
        lags, mult = oracle.schedule(synth.MEM_ADAPTIVE, 0, a, rule, k)
        los = [m - (d - 1) // 2 for m, d in zip(lags, mult) if d > 1]
        assert los and min(los) == a + 1
        assert max(mult) < 64

"""Pins of the oracle's memory schedules (Section 3.2).

Hand-derived cases from Definitions 3.1/3.2 and Proposition 3.1 live in
tests/golden/adaptive_schedule.txt; the remaining checks are structural
properties that follow from the definitions.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "adaptive_schedule.txt")
RULES = {"paper": oracle.ADAPT_PAPER, "partition": oracle.ADAPT_PARTITION}


def load_golden():
    cases, cur = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("case"):
            kv = dict(t.split("=") for t in line.split()[1:])
            cur = dict(a=int(kv["a"]), k=int(kv["k"]), rule=RULES[kv["rule"]], terms=[])
            cases.append(cur)
        else:
            m, d = line.split()
            cur["terms"].append((int(m), int(d)))
    return cases


@pytest.mark.parametrize("case", load_golden(), ids=lambda c: f"a{c['a']}k{c['k']}r{c['rule']}")
def test_golden_adaptive_schedules(case):
    lag, mult = oracle.schedule(oracle.MEM_ADAPTIVE, 0, case["a"], case["rule"], case["k"])
    assert list(zip(lag.tolist(), mult.tolist())) == case["terms"]


@pytest.mark.parametrize("k", [0, 1, 7, 100])
def test_full_and_short(k):
    lag, mult = oracle.schedule(oracle.MEM_FULL, 0, 0, 0, k)
    assert lag.tolist() == list(range(k + 1)) and np.all(mult == 1)
    for L in (0, 3, 50, 1000):
        lag, mult = oracle.schedule(oracle.MEM_SHORT, L, 0, 0, k)
        assert lag.tolist() == list(range(min(L, k) + 1)) and np.all(mult == 1)


def expand(lag, mult):
    """Lags each term stands for: a median m of weight d=2i-1 covers m-(i-1)..m+(i-1)."""
    cover = np.zeros(int(lag.max() + mult.max()) + 2, dtype=np.int64)
    for m, d in zip(lag, mult):
        h = (d - 1) // 2
        cover[m - h:m + h + 1] += 1
    return cover


@pytest.mark.parametrize("a", [2, 3, 5, 10, 20])
def test_partition_counts_every_lag_once(a):
    for k in list(range(0, 400)) + [999, 1234, 5000]:
        lag, mult = oracle.schedule(oracle.MEM_ADAPTIVE, 0, a, oracle.ADAPT_PARTITION, k)
        assert mult.sum() == k + 1
        cov = expand(lag, mult)
        assert np.all(cov[:k + 1] == 1) and np.all(cov[k + 1:] == 0)


@pytest.mark.parametrize("a", [2, 3, 5, 10, 20, 50])
def test_paper_rule_structure(a):
    for k in list(range(0, 300)) + [777, 2000, 5000]:
        lag, mult = oracle.schedule(oracle.MEM_ADAPTIVE, 0, a, oracle.ADAPT_PAPER, k)
        assert np.all(np.diff(lag) > 0) and lag[0] == 0 and lag[-1] <= k
        if k <= a:
            assert lag.tolist() == list(range(k + 1))
            continue
        assert lag[:a + 1].tolist() == list(range(a + 1)) and np.all(mult[:a + 1] == 1)
        cov = expand(lag, mult)
        assert cov[k] >= 1 and np.all(cov[k + 1:] == 0)      # nothing past k, k itself used
        for m, d in zip(lag[a + 1:], mult[a + 1:]):
            if d == 1:
                continue
            i = (d + 1) // 2
            assert a ** (i - 1) + i <= m <= a ** i           # medians inside I_i (Def. 3.1)
            assert (m - (a ** (i - 1) + i)) % d == 0         # on the eta grid (Prop. 3.1)


def test_paper_and_partition_coincide_for_a10():
    # For a = 10 every interval's increments end exactly on a^i up to i = 3, so both
    # readings give the same terms while k stays below the first i=5 increment.
    for k in range(0, 10001, 37):
        a1 = oracle.schedule(oracle.MEM_ADAPTIVE, 0, 10, oracle.ADAPT_PAPER, k)
        a2 = oracle.schedule(oracle.MEM_ADAPTIVE, 0, 10, oracle.ADAPT_PARTITION, k)
        assert a1[0].tolist() == a2[0].tolist() and a1[1].tolist() == a2[1].tolist()


def test_prefix_property():
    # Sampled medians used at step k are a prefix (ordered by increment end) of those at k+1,
    # and the tail always runs to k: the device form (prefix pointer + tail range) relies on it.
    for a in (2, 3, 10):
        for rule in (oracle.ADAPT_PAPER, oracle.ADAPT_PARTITION):
            prev = []
            for k in range(0, 3000):
                lag, mult = oracle.schedule(oracle.MEM_ADAPTIVE, 0, a, rule, k)
                med = [(int(m), int(d)) for m, d in zip(lag, mult) if d > 1]
                assert med[:len(prev)] == prev
                prev = med
                tail = lag[a + 1 + len(med):] if k > a else []
                if len(tail):
                    assert tail[-1] == k and np.all(np.diff(tail) == 1)

"""Adaptive memory (Definitions 3.1/3.2, Proposition 3.1): once a median's increment is in the
schedule, every lag it stands for keeps its weight at all later steps.  So at every step k the
schedule's multiplicities equal the settled ones g(m) (1 on the base interval [0, a], the
increment length d at a median, 0 between medians) up to a lag e(k), and are 1 on the tail
e(k)+1 .. k.  e(k) never decreases and the tail is shorter than a few increments.

The temporally blocked path rests on this decomposition: it streams rows older than a block's
longest tail with the settled weights and adds the tail rows with each step's own weights.
These checks use only the oracle's schedule."""
import numpy as np
import pytest

import oracle

MEM_ADAPTIVE = 2


def multiplicities(a, rule, k):
    lags, mult = oracle.schedule(MEM_ADAPTIVE, 0, a, rule, k)
    w = np.zeros(k + 1, dtype=np.int64)
    np.add.at(w, lags, mult)
    return w


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("a", [2, 3, 5, 10])
def test_adaptive_weights_settle_below_a_short_tail(a, rule):
    K = 2500
    g = multiplicities(a, rule, K)
    # settled part of step K: up to the last lag above a whose multiplicity is not 1
    above = np.nonzero(g[a + 1:] != 1)[0]
    eK = a + 1 + int(above[-1]) if above.size else a
    g = g[: eK + 1]
    assert np.all(g[: a + 1] == 1) and set(np.unique(g[a + 1:]).tolist()) <= {0} | set(range(3, 200, 2))
    prev = -1
    for k in range(K + 1):
        w = multiplicities(a, rule, k)
        top = min(k, eK)
        diff = np.nonzero(w[: top + 1] != g[: top + 1])[0]
        e = top if diff.size == 0 else int(diff[0]) - 1
        assert np.all(w[e + 1:] == 1), (k, e)  # the tail: weight psi_m, multiplicity 1
        assert e >= prev, (k, e, prev)          # settled lags stay settled
        prev = e
        i_max = 1
        while a ** i_max <= k:
            i_max += 1
        assert k - e <= 4 * i_max, (k, e)       # fewer than two increments of the widest interval
    # the schedule's terms are the settled weights plus the tail, at every step
    assert prev == eK
    w = multiplicities(a, rule, K)
    assert w.sum() == g.sum() + (K - eK)


def test_settled_weights_of_a_worked_case():
    """a = 3, paper rule, written out from Def. 3.1/3.2 and Prop. 3.1: base lags 0..3; interval
    2 = [5, 9]: medians 5, 8 (d = 3) standing for 4..6 and 7..9; interval 3 = [12, 27]:
    medians 12, 17, 22, 27 (d = 5) standing for 10..14, 15..19, 20..24, 25..29."""
    g = multiplicities(3, 0, 40)
    want = {m: 1 for m in range(4)}
    want.update({5: 3, 8: 3, 12: 5, 17: 5, 22: 5, 27: 5})
    assert all(g[m] == want.get(m, 0) for m in range(30))
    # at k = 26 the increment 25..29 is not yet in: lags 25, 26 are the tail
    w = multiplicities(3, 0, 26)
    assert list(w[25:27]) == [1, 1] and w[22] == 5 and w[23] == 0

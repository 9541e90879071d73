"""The paper's experiments (Figs. 1 and 3) on the engine, in FP64, against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1004_5128_gb300 import FRD, experiments as E, synth
from tests.helpers import rel_inf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode,L,a", [(synth.MEM_FULL, 0, 0), (synth.MEM_SHORT, 100, 0),
                                      (synth.MEM_ADAPTIVE, 0, 3), (synth.MEM_ADAPTIVE, 0, 10)])
def test_fig3_runs_match_oracle(mode, L, a):
    p = E.fig3_problem(0.9, mode, L=L, a=a)
    s = FRD(p, state="f64")
    s.set_state(p["u0"])
    assert rel_inf(s.run(p["K"]).cpu().numpy(), oracle.run(p)) < 1e-12


def test_fig1_trace_and_profile():
    res = E.fig1()
    for g in E.FIG1_GAMMAS:
        ref, tape = oracle.run(E.fig1_problem(g), tape=True)
        assert rel_inf(res[g]["profile"], ref.reshape(100, 100)[50]) < 1e-12
        assert rel_inf(res[g]["centre_trace"], tape[:, 50 * 100 + 50]) < 1e-12


def test_fig3_table_rows():
    rows = E.fig3(gammas=(0.9,), Ls=(50, 400), As=(3, 20))
    assert [r["method"] for r in rows] == ["full", "short", "short", "adaptive", "adaptive"]
    assert all(r["ms"] > 0 and np.isfinite(r["l2_pct"]) for r in rows)
    assert "| 0.9 | adaptive | 3 |" in E.fig3_table(rows)

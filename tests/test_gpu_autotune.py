"""The autotuner on the GPU: a short coordinate descent on a small problem returns a geometry
from its parameter table, and a run with that geometry matches the oracle."""
import pytest

import oracle
from paper_1004_5128_gb300 import FRD, autotune, synth
from tests.helpers import rel_inf

pytestmark = pytest.mark.gpu


def test_tune_small_problem(tmp_path, monkeypatch):
    monkeypatch.setenv("FD_TUNE_CACHE", str(tmp_path / "tune.json"))
    p = synth.with_mode(synth.config2(K=200, n=48), synth.MEM_ADAPTIVE, a=3)
    geo = autotune.tune(p, budget_s=15.0, reps=1)
    assert set(geo) <= set(autotune.PARAMS) and all(geo[k] in autotune.PARAMS[k] for k in geo)
    assert autotune.lookup(p) == geo          # cached under the problem's key
    s = FRD(p, **geo)
    s.set_state(p["u0"])
    assert rel_inf(s.run(p["K"]).cpu().double().numpy(), oracle.run(p)) < 1e-5

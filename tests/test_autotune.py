"""The autotuner's cache lookup and the geometry a handle takes from it (CPU: no kernel runs)."""
import json

import pytest

from paper_1004_5128_gb300 import autotune, synth
from paper_1004_5128_gb300.frd import tuned_geometry


@pytest.fixture
def cache(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("FD_TUNE_CACHE", str(path))
    return path


def test_key_buckets_grid_and_steps():
    p = synth.config2(K=5000)
    assert autotune.key(p) == "f32/f32/plain/mode0/d2/N65536/K8192"
    assert autotune.key(synth.config3(K=20000), hist="bf16") == "f32/bf16/plain/mode0/d2/N262144/K32768"
    q = synth.config2(K=4097)
    assert autotune.key(q).endswith("/K8192") and autotune.key(synth.config2(K=4096)).endswith("/K4096")


def test_exact_key_then_nearest_step_bucket(cache):
    p = synth.config2(K=700)  # K bucket 1024
    k = autotune.key(p)
    cache.write_text(json.dumps({
        k.replace("/K1024", "/K256"): {"geometry": {"chunk_terms": 64}, "terms_per_s": 1.0},
        k.replace("/K1024", "/K8192"): {"geometry": {"chunk_terms": 256}, "terms_per_s": 1.0}}))
    assert autotune.lookup(p) == {"chunk_terms": 64}          # 1024 is 2 octaves from 256, 3 from 8192
    cache.write_text(json.dumps({k: {"geometry": {"stages": 4}, "terms_per_s": 1.0}}))
    assert autotune.lookup(p) == {"stages": 4}                # exact key wins


def test_falls_back_to_the_shipped_table(cache):
    cache.write_text("{}")
    shipped = json.load(open(autotune.SHIPPED))
    p = synth.config2(K=5000)
    assert autotune.lookup(p) == shipped[autotune.key(p)]["geometry"]
    # an unknown problem class (here: 3-D) has no geometry
    q = synth.problem(3, 8, 8, 0.5, 1.0, 0.01, 1.0, synth.BC_NOFLUX, K=100, nz=8)
    assert autotune.lookup(q) == {}


def test_handles_take_the_tuned_geometry_unless_given_one(cache):
    cache.write_text("{}")
    p = synth.config2(K=5000)
    assert tuned_geometry(p, {}) == {"time_block": 64}
    assert tuned_geometry(p, {"chunk_terms": 64}) == {}      # explicit geometry: no lookup
    # a taped handle caps the block at 8 steps (the blocked adjoint's limit)
    assert tuned_geometry(p, {"keep_tape": True})["time_block"] == 8


def test_tuner_holds_fixed_options(cache, monkeypatch):
    """tune() explores PARAMS but never the options it was given (no GPU: only the candidate
    generation is exercised, through a stub timer)."""
    seen = []
    monkeypatch.setattr(autotune, "_time_single",
                        lambda p, g, reps, **kw: (seen.append(dict(g)), 1.0 + len(g) * 0.1)[1])
    g = autotune.tune(synth.config2(K=100), budget_s=5.0, time_block=16)
    assert g["time_block"] == 16 and all(s.get("time_block") == 16 for s in seen)
    assert set(g) <= set(autotune.PARAMS) and all(g[k] in autotune.PARAMS[k] for k in g if k != "time_block")

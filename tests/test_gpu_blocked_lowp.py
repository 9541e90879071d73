"""Temporally blocked engine with BF16 and FP16 (row-tile scaled) history: the far rows stream
in 16-bit precision, the newest 2T rows come from an FP32 ring.  Against the FP64 oracle at
the stated low-precision tolerance (2e-3, infinity norm relative to max |u_ref|), and, at the
full 512^2 x 20000-step size, element by element against the FP32-history run."""
import numpy as np
import pytest

import oracle
from paper_1004_5128_gb300 import FRD, synth
from tests.helpers import rel_inf

pytestmark = pytest.mark.gpu

TOL = 2e-3


def ragged(bc, mode, L=0, a=0, K=300, scale=1.0):
    return synth.problem(2, 45, 37, 0.75, 0.7, synth.dt_for_courant(0.15, 0.7, 1.0, 0.75), 1.0, bc,
                         react=(0.01, -0.2, 0.3, -0.4), mem_mode=mode, mem_L=L, mem_a=a, K=K,
                         u0=scale * synth.SplitMix64(21).uniform(45 * 37, 0, 1))


def run(p, **kw):
    s = FRD(p, **kw)
    s.set_state(p["u0"])
    out = s.run(p["K"]).cpu().double().numpy()
    assert s.status() == 0
    return out, s


MODES = [("full", synth.MEM_FULL, 0, 0), ("short7", synth.MEM_SHORT, 7, 0),
         ("short50", synth.MEM_SHORT, 50, 0), ("adapt3", synth.MEM_ADAPTIVE, 0, 3)]


@pytest.mark.parametrize("step_updates", [False, True])
@pytest.mark.parametrize("tb", [4, 8, 16])
@pytest.mark.parametrize("name,mode,L,a", MODES, ids=[m[0] for m in MODES])
@pytest.mark.parametrize("hist", ["bf16", "f16"])
def test_blocked_lowp_matches_oracle(hist, name, mode, L, a, tb, step_updates):
    """45 x 37 (ragged last tile), several far chunks per block, both kinds of update unit."""
    p = ragged(synth.BC_NOFLUX if tb != 8 else synth.BC_DIRICHLET0, mode, L, a)
    got, s = run(p, hist=hist, time_block=tb, chunk_terms=16, step_updates=step_updates)
    g = s.geometry()
    assert g["time_block"] == tb and g["block_updates"] == (0 if step_updates else 1)
    assert rel_inf(got, oracle.run(p)) < TOL


@pytest.mark.parametrize("hist", ["bf16", "f16"])
def test_blocked_lowp_config3_128_vs_oracle(hist):
    """Config-3 physics at the oracle-checkable size (128^2, 2000 steps, logistic reaction)."""
    p = synth.config3(n=128, K=2000)
    got, _ = run(p, hist=hist, time_block=16)
    assert rel_inf(got, oracle.run(p, threads=0)) < TOL


def test_blocked_fp16_scales_keep_tiny_fields():
    """A field of size 1e-6: its differences sit below FP16's normal range, so only the per
    (row, tile) power-of-two scales keep them; the result must still meet the tolerance."""
    p = ragged(synth.BC_DIRICHLET0, synth.MEM_FULL, K=200, scale=1e-6)
    got, _ = run(p, hist="f16", time_block=8, chunk_terms=16)
    assert rel_inf(got, oracle.run(p)) < TOL


@pytest.mark.parametrize("hist", ["bf16", "f16"])
def test_blocked_lowp_launch_split_is_bitwise_invariant(hist):
    p = ragged(synth.BC_NOFLUX, synth.MEM_ADAPTIVE, a=3, K=400)
    one, _ = run(p, hist=hist, time_block=8, chunk_terms=32)
    b = FRD(p, hist=hist, time_block=8, chunk_terms=32)
    b.set_state(p["u0"])
    for n in (57, 3, 100, 1, 139, 100):
        b.step(n)
    assert np.array_equal(one, b.run(0).cpu().double().numpy())


def test_config3_full_size_lowp_vs_fp32_history():
    """512^2, 20000 steps: the BF16- and FP16-history runs against the FP32-history run, element
    by element at the low-precision tolerance."""
    p = synth.config3()
    ref, _ = run(p, time_block=16)
    for hist in ("bf16", "f16"):
        got, _ = run(p, hist=hist, time_block=16)
        assert rel_inf(got, ref) < TOL, hist

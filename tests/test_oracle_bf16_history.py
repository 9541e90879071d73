"""Pins of the oracle's BF16-stored history run (the storage rule of the mixed-precision GPU
paths: history rows older than an FP32 window are used after rounding to BF16)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1004_5128_gb300 import synth


def test_round_bf16_matches_torch_bfloat16():
    """Round to nearest even at 8 significant bits, as torch's float32 -> bfloat16 conversion
    does, on FP32-representable values (no double rounding): random values, exact ties and
    values next to ties, powers of two, negative values."""
    g = np.random.default_rng(7)
    x = g.standard_normal(20000) * np.exp(g.uniform(-30, 30, 20000))
    # exact ties: 8 significant bits plus a trailing half, and one FP32 ulp around them
    m = g.integers(128, 256, 2000).astype(np.float64)
    ties = (m + 0.5) * 2.0 ** g.integers(-40, 40, 2000)
    x = np.concatenate([x, ties, np.nextafter(ties.astype(np.float32), np.float32(np.inf)).astype(np.float64),
                        -ties, 2.0 ** np.arange(-60, 60), [0.0, -0.0]])
    x = x.astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x).float().to(torch.bfloat16).double().numpy()
    got = np.array([oracle.round_bf16(v) for v in x])
    assert np.array_equal(got, ref)


def ragged(mode, L=0, a=0, K=120):
    return synth.problem(2, 17, 13, 0.75, 0.7, synth.dt_for_courant(0.15, 0.7, 1.0, 0.75), 1.0,
                         synth.BC_NOFLUX, react=(0.01, -0.2, 0.3, -0.4), mem_mode=mode, mem_L=L,
                         mem_a=a, K=K, u0=synth.SplitMix64(21).uniform(17 * 13, 0, 1))


@pytest.mark.parametrize("mode,L,a", [(synth.MEM_FULL, 0, 0), (synth.MEM_SHORT, 9, 0),
                                      (synth.MEM_ADAPTIVE, 0, 3)])
def test_window_covering_all_lags_is_the_plain_run(mode, L, a):
    p = ragged(mode, L, a)
    assert np.array_equal(oracle.run_bf16(p, 0, p["K"]), oracle.run(p))
    assert np.array_equal(oracle.run_bf16(p, 16, p["K"]), oracle.run(p))


def test_rounding_error_scale_and_window_effect():
    """With all lags >= 1 rounded, the result moves by about BF16's relative precision times the
    memory's weight; a wider FP32 window moves it less (the newest lags carry the largest
    weights)."""
    p = ragged(synth.MEM_FULL, K=200)
    ref = oracle.run(p)
    e = [np.max(np.abs(oracle.run_bf16(p, 0, h) - ref)) / np.max(np.abs(ref)) for h in (0, 8, 32)]
    assert 1e-6 < e[0] < 2e-2
    assert e[2] < e[1] < e[0]


def test_block_window_rule():
    """blk > 0: step k keeps lags up to head + (k mod blk) exact.  With blk = 1 that is the
    per-step rule with the same head."""
    p = ragged(synth.MEM_ADAPTIVE, a=3)
    assert np.array_equal(oracle.run_bf16(p, 1, 5), oracle.run_bf16(p, 0, 5))
    a = oracle.run_bf16(p, 8, 8)
    assert not np.array_equal(a, oracle.run_bf16(p, 0, 8))

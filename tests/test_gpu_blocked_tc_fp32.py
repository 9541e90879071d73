"""Temporally blocked engine with FP32 history whose far rows run on the tensor cores (blocks of 32
and 64 steps): every history row is stored as two FP16 planes, hi = fp16(delta 2^e) and
lo = fp16(delta 2^e - hi) with a power of two 2^-e per (row, tile), and three FP16 MMAs per K
slice (hi.hi + hi.lo + lo.hi) accumulate in FP32.  The pair keeps about 22 significant bits of
every row value and weight, so the FP32 tolerance of the FP64 oracle holds (1e-5, infinity norm
relative to max |u_ref|).  With 256 threads per half-CTA each far unit covers half a tile (far
sub-tiles of 512 points), with 128 threads the whole tile."""
import numpy as np
import pytest

import oracle
from paper_1004_5128_gb300 import FRD, synth
from tests.helpers import rel_inf

pytestmark = pytest.mark.gpu

TOL = 1e-5
# Against the CUDA-core far loop over the same FP32 rows: both are FP32 sums of the same terms in
# different orders, plus the split's 2^-22 relative rounding of each row value and weight.
SAME_ROWS_TOL = 2e-6


def ragged(bc, mode, L=0, a=0, K=300, scale=1.0, nx=45, ny=37, react=(0.01, -0.2, 0.3, -0.4)):
    return synth.problem(2, nx, ny, 0.75, 0.7, synth.dt_for_courant(0.15, 0.7, 1.0, 0.75), 1.0, bc,
                         react=react, mem_mode=mode, mem_L=L, mem_a=a, K=K,
                         u0=scale * synth.SplitMix64(21).uniform(nx * ny, 0, 1))


def run(p, **kw):
    s = FRD(p, **kw)
    s.set_state(p["u0"])
    out = s.run(p["K"]).cpu().double().numpy()
    assert s.status() == 0
    return out, s


MODES = [("full", synth.MEM_FULL, 0, 0), ("short40", synth.MEM_SHORT, 40, 0),
         ("adapt3", synth.MEM_ADAPTIVE, 0, 3), ("adapt10", synth.MEM_ADAPTIVE, 0, 10)]


@pytest.mark.parametrize("threads", [256, 128])
@pytest.mark.parametrize("step_updates", [False, True])
@pytest.mark.parametrize("tb", [32, 64])
@pytest.mark.parametrize("name,mode,L,a", MODES, ids=[m[0] for m in MODES])
def test_fp32_tensor_core_far_units_match_oracle(name, mode, L, a, tb, step_updates, threads):
    """45 x 37 points (two ragged tiles of 1024, or four of 512), 300 steps, chunks of two stages."""
    p = ragged(synth.BC_NOFLUX, mode, L, a, K=300)
    got, s = run(p, time_block=tb, chunk_terms=32, step_updates=step_updates, tile_threads=threads)
    g = s.geometry()
    assert g["far_tensor_cores"] == 1 and g["time_block"] == tb and g["tile_threads"] == threads
    ref = oracle.run(p)
    assert rel_inf(got, ref) < TOL
    fma, s2 = run(p, time_block=16, step_updates=step_updates)  # CUDA-core far loop, same rows
    assert s2.geometry()["far_tensor_cores"] == 0
    assert rel_inf(got, fma) < SAME_ROWS_TOL


@pytest.mark.parametrize("scale", [1e-6, 1e6])
def test_fp32_tensor_core_field_scales(scale):
    """Row scales far from one (near 2^34 and 2^-6) meet the weights in the coefficients, which
    the per-unit power of two brings back into FP16 range (linear reaction: the cubic term would
    blow a field of 1e6 up)."""
    p = ragged(synth.BC_DIRICHLET0, synth.MEM_FULL, K=200, scale=scale, react=(0.01, -0.2, 0.0, 0.0))
    got, s = run(p, time_block=32, chunk_terms=64)
    assert s.geometry()["far_tensor_cores"] == 1
    assert rel_inf(got, oracle.run(p)) < TOL


def test_fp32_tensor_core_point_source_dynamic_range():
    """A unit point source on 65^2 for 400 steps: within a tile the rows span many orders of
    magnitude, the regime where one scale per (row, tile) loses the most bits."""
    u0 = np.zeros(65 * 65)
    u0[32 * 65 + 32] = 1.0
    p = synth.problem(2, 65, 65, 0.5, 1.0, synth.dt_for_courant(0.15, 1.0, 1.0, 0.5), 1.0, synth.BC_DIRICHLET0,
                      K=400, u0=u0)
    got, s = run(p, time_block=32, chunk_terms=32)
    assert s.geometry()["far_tensor_cores"] == 1
    assert rel_inf(got, oracle.run(p)) < TOL


def test_fp32_tensor_core_3d_and_one_dimension():
    p3 = synth.problem(3, 20, 17, 0.6, 0.5, 1e-3, 1.0, synth.BC_NOFLUX, react=(0.0, -0.1, 0.0, 0.0),
                       nz=13, K=160, u0=synth.SplitMix64(5).uniform(20 * 17 * 13, 0, 1))
    got, s = run(p3, time_block=32, chunk_terms=32)
    assert s.geometry()["far_tensor_cores"] == 1
    assert rel_inf(got, oracle.run(p3)) < TOL
    p1 = synth.problem(1, 3001, 1, 0.8, 0.5, 2e-4, 1.0, synth.BC_NOFLUX, react=(0.0, -0.1, 0.0, 0.0),
                       K=200, u0=synth.SplitMix64(9).uniform(3001, 0, 1))
    got, s = run(p1, time_block=64, chunk_terms=64)
    assert rel_inf(got, oracle.run(p1)) < TOL


def test_fp32_tensor_core_config3_128_vs_oracle_and_split_invariance():
    """Config-3 physics at 128^2, 2000 steps, blocks of 32; a run split into launches that start
    inside blocks gives the same bits."""
    p = synth.config3(n=128, K=2000)
    got, s = run(p, time_block=32)
    assert s.geometry()["far_tensor_cores"] == 1
    assert rel_inf(got, oracle.run(p, threads=0)) < TOL
    b = FRD(p, time_block=32)
    b.set_state(p["u0"])
    for n in (333, 17, 650, 1, 999):
        b.step(n)
    assert np.array_equal(got, b.run(0).cpu().double().numpy())


def test_fp32_tensor_core_batch_matches_single_runs():
    from paper_1004_5128_gb300 import FRDBatch
    probs = [ragged(synth.BC_NOFLUX, synth.MEM_FULL, K=200),
             synth.config3(n=40, K=260),
             synth.with_mode(synth.config2(K=150, n=33), synth.MEM_ADAPTIVE, a=3)]
    geo = dict(time_block=32, chunk_terms=64, step_updates=True)
    bt = FRDBatch(probs, **geo)
    for i, p in enumerate(probs):
        bt.set_state(i, p["u0"])
    bt.run()
    assert bt.status() == 0
    for i, p in enumerate(probs):
        one, _ = run(p, **geo)
        assert np.array_equal(bt.state(i).cpu().double().numpy(), one)


def test_config3_full_size_fp32_tensor_cores_vs_cuda_cores():
    """512^2, 20000 steps: the tensor-core run (blocks of 32) against the CUDA-core run (blocks of
    16) over the same FP32 history, element by element at the FP32 tolerance."""
    p = synth.config3()
    ref, s1 = run(p, time_block=16)
    got, s2 = run(p, time_block=32)
    assert s1.geometry()["far_tensor_cores"] == 0 and s2.geometry()["far_tensor_cores"] == 1
    assert rel_inf(got, ref) < TOL


C2_CASES = [("full", synth.MEM_FULL, 32, 256, 4000), ("short", synth.MEM_SHORT, 64, 256, 1000),
            ("adaptive", synth.MEM_ADAPTIVE, 32, 256, 2000), ("full128", synth.MEM_FULL, 32, 128, 2000)]


@pytest.mark.parametrize("name,mode,tb,threads,K", C2_CASES, ids=[c[0] for c in C2_CASES])
def test_fp32_tensor_cores_config2_row_scales_spread(name, mode, tb, threads, K):
    """Config 2 (256^2, eight decaying Gaussians): the row scales of one far unit spread over many
    octaves, so the coefficients' power of two must bound (largest weight) x (largest row scale)
    over the unit, not the largest product within one thread's share (which overflowed FP16).
    Against the CUDA-core run over the same FP32 rows."""
    p = synth.config2(mode, K=K)
    got, s = run(p, time_block=tb, tile_threads=threads)
    assert s.geometry()["far_tensor_cores"] == 1
    ref, _ = run(p, time_block=16)
    assert rel_inf(got, ref) < TOL


def test_fp16_tensor_cores_config2_row_scales_spread():
    """The same bound on the FP16-history path, against the CUDA-core far loop over the same FP16
    rows (what remains is FP32 summation order)."""
    p = synth.config2(synth.MEM_FULL, K=4000)
    got, s = run(p, hist="f16", time_block=32)
    assert s.geometry()["far_tensor_cores"] == 1
    ref, s2 = run(p, hist="f16", time_block=16, fma_far=True)
    assert s2.geometry()["far_tensor_cores"] == 0
    assert rel_inf(got, ref) < 5e-5


@pytest.mark.parametrize("hist", ["f32", "bf16"])
def test_two_tile_update_units_match_oracle_and_split_invariance(hist):
    """400 x 400 points are 157 tiles of 1024, more than half the 304 half-CTAs, so each per-step
    update unit carries two tiles (phase A of both, then phase B of both); against the oracle (BF16
    history at its tolerance, against the oracle with the BF16 storage rule at 5e-5), and a run split
    into launches inside blocks gives the same bits."""
    n, K = 400, 300
    p = synth.problem(2, n, n, 0.6, 1.0, synth.dt_for_courant(0.1, 1.0, 1.0, 0.6), 1.0, synth.BC_DIRICHLET0,
                      react=(0.0, 0.95, -1.0, 0.0), K=K, u0=0.1 * synth.SplitMix64(33).uniform(n * n, 0, 1))
    kw = dict(time_block=64) if hist == "f32" else dict(time_block=64, hist="bf16")
    got, s = run(p, **kw)
    g = s.geometry()
    assert g["far_tensor_cores"] == 1 and g["tiles"] == 157
    if hist == "f32":
        assert rel_inf(got, oracle.run(p)) < TOL
    else:
        assert rel_inf(got, oracle.run(p)) < 2e-3
        assert rel_inf(got, oracle.run_bf16(p, 64, 64)) < 5e-5
    b = FRD(p, **kw)
    b.set_state(p["u0"])
    for m in (77, 1, 100, 45):
        b.step(m)
    assert np.array_equal(got, b.run(K - 223).cpu().double().numpy())

"""GPU parity of the forward engine (all memory modes and history dtypes) against the FP64
oracle, element by element, plus full-size checks through properties that hold at any size.

Tolerances (infinity norm relative to max |u_ref|): 1e-12 FP64, 1e-5 FP32 history,
2e-3 BF16/FP16 history."""
import numpy as np
import pytest
import torch

import oracle
from paper_1004_5128_gb300 import FRD, FdError, synth
from paper_1004_5128_gb300 import _lib as L
from tests.helpers import laplacian_eigenvalue, rel_inf

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 2e-3, "f16": 2e-3}


def run_gpu(p, K=None, state="f32", **kw):
    K = p["K"] if K is None else K
    s = FRD(p, state=state, max_steps=max(K, 1), **kw)
    s.set_state(p["u0"])
    out = s.run(K).cpu().double().numpy()
    return out, s


def test_config1_fp64_full():
    """1-D N=256, Dirichlet, gamma=0.5, S=0.2, 1000 steps, full memory, FP64."""
    p = synth.config1()
    got, s = run_gpu(p, state="f64")
    assert s.status() == 0
    assert rel_inf(got, oracle.run(p)) < TOL["f64"]


MODES = [("full", synth.MEM_FULL, 0, 0, 0), ("short50", synth.MEM_SHORT, 50, 0, 0),
         ("short1", synth.MEM_SHORT, 1, 0, 0), ("adapt3", synth.MEM_ADAPTIVE, 0, 3, 0),
         ("adapt10", synth.MEM_ADAPTIVE, 0, 10, 0), ("adapt2part", synth.MEM_ADAPTIVE, 0, 2, 1)]


@pytest.mark.parametrize("name,mode,Lw,a,rule", MODES, ids=[m[0] for m in MODES])
@pytest.mark.parametrize("bc", [synth.BC_DIRICHLET0, synth.BC_NOFLUX])
def test_fp32_modes_2d_ragged(name, mode, Lw, a, rule, bc):
    """45 x 37 grid (ragged last tile), 300 steps, several chunks per step."""
    p = synth.problem(2, 45, 37, 0.75, 0.7, synth.dt_for_courant(0.15, 0.7, 1.0, 0.75), 1.0, bc,
                      react=(0.01, -0.2, 0.3, -0.4), mem_mode=mode, mem_L=Lw, mem_a=a,
                      adaptive_rule=rule, K=300, u0=synth.SplitMix64(21).uniform(45 * 37, 0, 1))
    got, _ = run_gpu(p, chunk_terms=16)
    assert rel_inf(got, oracle.run(p)) < TOL["f32"]


@pytest.mark.parametrize("state", ["f32", "f64"])
def test_1d_many_tiles(state):
    """1-D N=3001 (3+ tiles with a ragged tail), adaptive a=5, 400 steps."""
    p = synth.problem(1, 3001, 1, 0.55, 1.0, synth.dt_for_courant(0.2, 1.0, 1.0, 0.55), 1.0,
                      synth.BC_DIRICHLET0, react=(0, -0.05, 0, 0), mem_mode=synth.MEM_ADAPTIVE,
                      mem_a=5, K=400, u0=synth.SplitMix64(8).uniform(3001, -1, 1))
    got, _ = run_gpu(p, state=state, tile_threads=64, chunk_terms=24)
    assert rel_inf(got, oracle.run(p)) < TOL[state]


@pytest.mark.parametrize("hist", ["bf16", "f16", "f32"])
def test_config3_mixed_precision_128(hist):
    """Config-3 physics at the oracle-checkable size: 128^2, 2000 steps, logistic reaction,
    BF16 / FP16 (row-tile scaled) history with Kahan FP32 accumulation vs FP32 history."""
    p = synth.config3(n=128, K=2000)
    got, s = run_gpu(p, hist=hist, kahan=(hist != "f32"))
    assert s.status() == 0
    ref = oracle.run(p, threads=0)
    assert rel_inf(got, ref) < TOL[hist]
    if hist == "bf16":  # the oracle with the same storage rule: head lags 1..32 in FP32
        assert s.geometry()["head_lags"] == 32
        assert rel_inf(got, oracle.run_bf16(p, 0, 32, threads=0)) < 5e-5  # rounding flips, as blocked


def test_deterministic_and_launch_split_invariant():
    """Fixed chunk order: repeated runs and a run split into many launches agree bitwise."""
    p = synth.with_mode(synth.config2(K=400, n=64), synth.MEM_ADAPTIVE, a=3)
    a, _ = run_gpu(p, chunk_terms=32)
    b, _ = run_gpu(p, chunk_terms=32)
    s = FRD(p, max_steps=400, chunk_terms=32)
    s.set_state(p["u0"])
    for _ in range(8):
        s.step(50)
    c = s.run(0).cpu().double().numpy()
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_edge_cases():
    # a single point (1-D): delta = -2u, the relaxation problem
    p = synth.problem(1, 1, 1, 0.6, 0.5, 0.01, 1.0, synth.BC_DIRICHLET0, K=300, u0=[1.0])
    got, _ = run_gpu(p, state="f64")
    assert rel_inf(got, oracle.run(p)) < 1e-12
    # a 1-wide 2-D strip, no-flux
    p = synth.problem(2, 1, 33, 0.9, 1.0, 0.02, 1.0, synth.BC_NOFLUX, K=120,
                      u0=synth.SplitMix64(3).uniform(33, 0, 1))
    got, _ = run_gpu(p)
    assert rel_inf(got, oracle.run(p)) < 1e-5
    # zero steps returns u0; one step equals the oracle
    p = synth.config1(K=1)
    s = FRD(p, state="f64", max_steps=1)
    s.set_state(p["u0"])
    assert np.array_equal(s.run(0).cpu().numpy(), p["u0"])
    assert rel_inf(s.run(1).cpu().numpy(), oracle.run(p)) < 1e-14
    # capacity is enforced
    with pytest.raises(FdError) as e:
        s.step(1)
    assert e.value.code == L.FD_ERR_STATE


def test_nonfinite_flag():
    p = synth.problem(1, 64, 1, 0.8, 1.0, 1.0, 1.0, synth.BC_DIRICHLET0, K=400,
                      u0=synth.SplitMix64(1).uniform(64, 0, 1))
    s = FRD(p, max_steps=400, allow_unstable=True)
    s.set_state(p["u0"])
    with pytest.raises(FdError) as e:
        s.run(400)
    assert e.value.code == L.FD_ERR_NONFINITE


def test_stall_injection_times_out_and_gpu_stays_usable():
    """A device wait on a counter nothing advances ends with FD_ERR_TIMEOUT after timeout_ms;
    the context stays usable for the next handle."""
    p = synth.config2(K=20, n=64)
    s = FRD(p, max_steps=20, inject_stall=True, timeout_ms=200)
    s.set_state(p["u0"])
    with pytest.raises(FdError) as e:
        s.run(20)
    assert e.value.code == L.FD_ERR_TIMEOUT
    # the first wait to give up is the injected one or one queued behind it
    info = s.error_info()
    assert info["words"][0] in (6, 8, 9) and info["site"] != "none"
    with pytest.raises(FdError) as e:
        s.step(1)
    assert e.value.code == L.FD_ERR_STATE
    got, _ = run_gpu(p)
    assert rel_inf(got, oracle.run(p)) < 1e-5


# ---------------------------------------------------------------- full-size (config 2)

@pytest.mark.parametrize("mode", [synth.MEM_FULL, synth.MEM_SHORT, synth.MEM_ADAPTIVE])
def test_config2_full_size_modes_vs_scalar_recursions(mode):
    """256^2, 5000 steps, no-flux, f=-0.1u in the benchmark's launch geometry.  A sum of
    cosine eigenmodes evolves mode by mode, each amplitude following the oracle's scalar
    recursion under the same weights and schedule; compare every point."""
    p = synth.config2(mode)
    modes = [(0, 0, 1.0), (1, 0, 0.5), (3, 2, 0.25), (17, 5, 0.125), (64, 64, 0.0625), (200, 31, 0.03)]
    u0 = sum(c * synth.eigenmode(p, qx, qy) for qx, qy, c in modes)
    ref = np.zeros_like(u0)
    for qx, qy, c in modes:
        A = oracle.scalar_mode(p, laplacian_eigenvalue(p, qx, qy))
        ref += c * A[-1] * synth.eigenmode(p, qx, qy)
    q = dict(p)
    q["u0"] = u0
    got, s = run_gpu(q)
    assert s.status() == 0
    assert rel_inf(got, ref) < 1e-5


@pytest.mark.parametrize("mode", [synth.MEM_FULL, synth.MEM_SHORT, synth.MEM_ADAPTIVE])
def test_config2_gaussians_mass_balance(mode):
    """The actual config-2 input: mirror boundaries conserve mass up to the decay term,
    M^K = (1 - 0.1 dt)^K M^0 in every memory mode."""
    p = synth.config2(mode)
    got, _ = run_gpu(p)
    M0 = p["u0"].sum()
    ref = M0 * (1.0 - 0.1 * p["dt"]) ** p["K"]
    assert abs(got.sum() - ref) / M0 < 2e-5


@pytest.mark.parametrize("state", ["f32", "f64"])
@pytest.mark.parametrize("mode,Lw,a", [(synth.MEM_FULL, 0, 0), (synth.MEM_SHORT, 40, 0),
                                       (synth.MEM_ADAPTIVE, 0, 3)])
def test_superdiffusion(state, mode, Lw, a):
    """gamma = 1.5 (weights positive, partial sums growing like m^{1/2}), S at 60% of the bound."""
    g = 1.5
    dt = synth.dt_for_courant(0.6 * synth.stability_bound(g, 2), 1.0, 1.0, g)
    p = synth.problem(2, 40, 33, g, 1.0, dt, 1.0, synth.BC_DIRICHLET0, react=(0, -0.05, 0, 0),
                      mem_mode=mode, mem_L=Lw, mem_a=a, K=250,
                      u0=synth.SplitMix64(17).uniform(40 * 33, 0, 1))
    got, _ = run_gpu(p, state=state)
    assert rel_inf(got, oracle.run(p)) < TOL[state]


@pytest.mark.parametrize("state", ["f32", "f64"])
@pytest.mark.parametrize("bc", [synth.BC_DIRICHLET0, synth.BC_NOFLUX])
@pytest.mark.parametrize("mode,Lw,a", [(synth.MEM_FULL, 0, 0), (synth.MEM_SHORT, 30, 0),
                                       (synth.MEM_ADAPTIVE, 0, 3)])
def test_3d_ragged(state, bc, mode, Lw, a):
    """3-D 20 x 17 x 13 (7-point stencil; tiles cut through z-planes), 200 steps."""
    nx, ny, nz = 20, 17, 13
    dt = synth.dt_for_courant(0.5 * synth.stability_bound(0.8, 3), 1.0, 1.0, 0.8)
    p = synth.problem(3, nx, ny, 0.8, 1.0, dt, 1.0, bc, react=(0.02, -0.1, 0.1, -0.05),
                      mem_mode=mode, mem_L=Lw, mem_a=a, K=200, nz=nz,
                      u0=synth.SplitMix64(33).uniform(nx * ny * nz, 0, 1))
    got, _ = run_gpu(p, state=state, chunk_terms=24)
    assert rel_inf(got, oracle.run(p)) < TOL[state]


def test_3d_64cube_eigenmodes():
    """64^3 = 262144 points, 600 steps, no-flux, f = -0.05u: a sum of cosine modes evolves
    through the oracle's scalar recursions (full memory)."""
    n = 64
    dt = synth.dt_for_courant(0.5 * synth.stability_bound(0.7, 3), 1.0, 1.0, 0.7)
    p = synth.problem(3, n, n, 0.7, 1.0, dt, 1.0, synth.BC_NOFLUX, react=(0, -0.05, 0, 0), K=600,
                      nz=n)
    modes = [(0, 0, 0, 1.0), (1, 2, 3, 0.4), (9, 4, 17, 0.2), (40, 33, 60, 0.1)]
    p["u0"] = sum(c * synth.eigenmode(p, qx, qy, qz) for qx, qy, qz, c in modes)
    ref = np.zeros_like(p["u0"])
    for qx, qy, qz, c in modes:
        A = oracle.scalar_mode(p, laplacian_eigenvalue(p, qx, qy, qz))
        ref += c * A[-1] * synth.eigenmode(p, qx, qy, qz)
    got, _ = run_gpu(p)
    assert rel_inf(got, ref) < 1e-5

"""GPU parity of the checkpointed reverse-time adjoint against the FP64 oracle adjoint, and the
autograd binding.  J = 1/2 |u^K - target|^2; gradients w.r.t. gamma, alpha, react, u0.

Tolerances are the stated ones: 1e-12 (FP64) and 1e-5 (FP32), each relative to the largest
magnitude of the reference gradient (infinity norm for dJ/du0 and dJ/dreact)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1004_5128_gb300 import FRD, FRDFunction, synth
from tests.helpers import rel_inf

TOL = {"f64": 1e-12, "f32": 1e-5}

pytestmark = pytest.mark.gpu


def small(bc, nx=20, ny=17, K=150, gamma=0.7):
    g = synth.SplitMix64(91)
    u0 = g.uniform(nx * ny, 0.0, 1.0)
    tgt = g.uniform(nx * ny, 0.0, 0.8)
    p = synth.problem(2, nx, ny, gamma, 0.8, 0.02, 1.0, bc, react=(0.03, -0.2, 0.15, -0.1), K=K, u0=u0)
    return p, tgt


def gpu_adjoint(p, tgt, state, ckpt, **kw):
    s = FRD(p, state=state, keep_tape=True, ckpt_every=ckpt, **kw)
    s.set_state(p["u0"])
    uK = s.run(p["K"])
    dJ = uK - torch.as_tensor(tgt, device=uK.device, dtype=uK.dtype)
    r = s.adjoint(dJ)
    r["du0"] = r["du0"].cpu().double().numpy()
    return r


def compare(r, ref, tol):
    assert rel_inf(r["du0"], ref["du0"]) < tol
    for key in ("dgamma", "dalpha"):
        assert abs(r[key] - ref[key]) <= tol * abs(ref[key]), (key, r[key], ref[key])
    dr = np.array(r["dreact"])
    assert np.max(np.abs(dr - ref["dreact"])) <= tol * np.max(np.abs(ref["dreact"]))


@pytest.mark.parametrize("bc", [synth.BC_DIRICHLET0, synth.BC_NOFLUX])
def test_adjoint_fp64_vs_oracle(bc):
    p, tgt = small(bc)
    r = gpu_adjoint(p, tgt, "f64", ckpt=40)  # 3 full segments + a ragged one
    compare(r, oracle.adjoint(p, tgt), TOL["f64"])


def test_adjoint_fp64_1d_many_tiles():
    g = synth.SplitMix64(4)
    n = 1500
    p = synth.problem(1, n, 1, 0.6, 1.0, 0.05, 1.0, synth.BC_DIRICHLET0, react=(0, -0.1, 0, 0), K=120,
                      u0=g.uniform(n, 0, 1))
    tgt = g.uniform(n, 0, 1)
    r = gpu_adjoint(p, tgt, "f64", ckpt=50, tile_threads=64, chunk_terms=16)
    compare(r, oracle.adjoint(p, tgt), TOL["f64"])


def test_adjoint_fp32_vs_oracle():
    p, tgt = small(synth.BC_DIRICHLET0, nx=48, ny=40, K=300)
    r = gpu_adjoint(p, tgt, "f32", ckpt=64)
    compare(r, oracle.adjoint(p, tgt), TOL["f32"])


def test_adjoint_config5_reduced_vs_oracle():
    """Config-5 physics (128^2, gamma=0.7, alpha=0.8, f=-0.1u, dt=0.005) at 300 steps."""
    p = synth.config5(K=300)
    tgt = oracle.run(synth.config5(K=300, target=True))
    r = gpu_adjoint(p, tgt, "f32", ckpt=200)
    compare(r, oracle.adjoint(p, tgt), TOL["f32"])


def test_adjoint_config5_full_size_fp64_vs_central_differences():
    """128^2, 4000 steps, checkpoints every 200: the FP64 GPU adjoint against Richardson-
    extrapolated central differences of the FP64 GPU forward (plain h = 1e-4 differences carry
    ~4e-5 truncation error here), and the FP32 adjoint against the FP64 one."""
    p = synth.config5()
    tgt_s = FRD(synth.config5(target=True), state="f64")
    tgt_s.set_state(p["u0"])
    tgt = tgt_s.run(p["K"])

    def J(q):
        s = FRD(q, state="f64")
        s.set_state(q["u0"])
        return 0.5 * float(((s.run(q["K"]) - tgt) ** 2).sum())

    r64 = gpu_adjoint(p, tgt.cpu().numpy(), "f64", ckpt=200)

    def fd(perturb):
        # central differences at h and h/2, Richardson-extrapolated: O(h^4) truncation
        def cd(h):
            return (J(perturb(h)) - J(perturb(-h))) / (2 * h)
        h = 1e-4
        return (4.0 * cd(h / 2) - cd(h)) / 3.0

    def field(name):
        def f(h):
            q = dict(p)
            q[name] = p[name] + h
            return q
        return f

    for key, name in (("dgamma", "gamma"), ("dalpha", "alpha")):
        ref = fd(field(name))
        assert abs(r64[key] - ref) < 1e-6 * abs(ref), (key, r64[key], ref)

    def react1(h):
        q = dict(p)
        q["react"] = [0.0, -0.1 + h, 0.0, 0.0]
        return q
    ref = fd(react1)
    assert abs(r64["dreact"][1] - ref) < 1e-6 * abs(ref)
    v = synth.SplitMix64(12).uniform(p["u0"].size, -1, 1)

    def along_v(h):
        q = dict(p)
        q["u0"] = p["u0"] + h * v
        return q
    ref = fd(along_v)
    assert abs(float(r64["du0"] @ v) - ref) < 1e-6 * abs(ref)
    r32 = gpu_adjoint(p, tgt.cpu().numpy(), "f32", ckpt=200)
    for key in ("dgamma", "dalpha"):
        assert abs(r32[key] - r64[key]) < TOL["f32"] * abs(r64[key])
    assert rel_inf(r32["du0"], r64["du0"]) < TOL["f32"]
    assert np.max(np.abs(np.array(r32["dreact"]) - r64["dreact"])) < TOL["f32"] * np.max(np.abs(r64["dreact"]))


def test_autograd_function():
    p, tgt = small(synth.BC_NOFLUX, nx=16, ny=16, K=80)
    dev = torch.device("cuda")
    u0 = torch.tensor(p["u0"], device=dev, requires_grad=True)
    gam = torch.tensor(p["gamma"], dtype=torch.float64, requires_grad=True)
    alp = torch.tensor(p["alpha"], dtype=torch.float64, requires_grad=True)
    react = torch.tensor(p["react"], dtype=torch.float64, requires_grad=True)
    uK = FRDFunction.apply(u0, gam, alp, react, dict(problem=p, K=p["K"], state="f64", ckpt_every=30))
    loss = 0.5 * ((uK - torch.tensor(tgt, device=dev)) ** 2).sum()
    loss.backward()
    ref = oracle.adjoint(p, tgt)
    assert abs(loss.item() - ref["J"]) < 1e-12 * ref["J"]
    assert rel_inf(u0.grad.cpu().numpy(), ref["du0"]) < TOL["f64"]
    assert abs(gam.grad.item() - ref["dgamma"]) < TOL["f64"] * abs(ref["dgamma"])
    assert abs(alp.grad.item() - ref["dalpha"]) < TOL["f64"] * abs(ref["dalpha"])
    assert np.max(np.abs(react.grad.numpy() - ref["dreact"])) < TOL["f64"] * np.max(np.abs(ref["dreact"]))


@pytest.mark.parametrize("state", ["f64", "f32"])
@pytest.mark.parametrize("L", [9, 40])
def test_short_memory_adjoint_vs_oracle(state, L):
    """Short memory: the adjoint sums each row over the transposed window (lags m <= L), with
    checkpoint segments of 40 steps over 150."""
    p, tgt = small(synth.BC_NOFLUX)
    p = synth.with_mode(p, synth.MEM_SHORT, L=L)
    r = gpu_adjoint(p, tgt, state, ckpt=40)
    compare(r, oracle.adjoint(p, tgt), TOL[state])


ADAPT = [(2, synth.ADAPT_PAPER), (3, synth.ADAPT_PAPER), (10, synth.ADAPT_PAPER), (2, synth.ADAPT_PARTITION),
         (3, synth.ADAPT_PARTITION)]


@pytest.mark.parametrize("state", ["f64", "f32"])
@pytest.mark.parametrize("a,rule", ADAPT)
def test_adaptive_memory_adjoint_vs_oracle(state, a, rule):
    """Adaptive memory (Definitions 3.1/3.2, Proposition 3.1): the adjoint sums every lag with the
    weight the medians settle on and corrects the tail terms of each step; checkpoint segments of
    40 steps over 150."""
    p, tgt = small(synth.BC_NOFLUX)
    p = synth.with_mode(p, synth.MEM_ADAPTIVE, a=a, rule=rule)
    r = gpu_adjoint(p, tgt, state, ckpt=40)
    compare(r, oracle.adjoint(p, tgt), TOL[state])


@pytest.mark.parametrize("step_updates", [False, True])
@pytest.mark.parametrize("tb", [4, 8])
@pytest.mark.parametrize("a,rule", ADAPT)
def test_adaptive_memory_blocked_adjoint_vs_oracle(tb, a, rule, step_updates):
    """The blocked adjoint of adaptive memory: far rows with the settled weights, launches that
    start inside blocks (checkpoints every 50 of 230 steps), several far chunks per block."""
    g = synth.SplitMix64(5)
    p = synth.problem(2, 45, 37, 0.75, 0.7, synth.dt_for_courant(0.15, 0.7, 1.0, 0.75), 1.0, synth.BC_DIRICHLET0,
                      react=(0.01, -0.2, 0.3, -0.4), mem_mode=synth.MEM_ADAPTIVE, mem_a=a, adaptive_rule=rule,
                      K=230, u0=g.uniform(45 * 37, 0, 1))
    tgt = g.uniform(45 * 37, 0, 0.8)
    r = gpu_adjoint(p, tgt, "f32", ckpt=50, time_block=tb, chunk_terms=16, step_updates=step_updates)
    compare(r, oracle.adjoint(p, tgt), TOL["f32"])


def test_autograd_function_adaptive_memory():
    p, tgt = small(synth.BC_DIRICHLET0, nx=16, ny=16, K=90)
    p = synth.with_mode(p, synth.MEM_ADAPTIVE, a=3)
    dev = torch.device("cuda")
    u0 = torch.tensor(p["u0"], device=dev, requires_grad=True)
    gam = torch.tensor(p["gamma"], dtype=torch.float64, requires_grad=True)
    alp = torch.tensor(p["alpha"], dtype=torch.float64, requires_grad=True)
    react = torch.tensor(p["react"], dtype=torch.float64, requires_grad=True)
    uK = FRDFunction.apply(u0, gam, alp, react, dict(problem=p, K=p["K"], state="f64", ckpt_every=25))
    loss = 0.5 * ((uK - torch.tensor(tgt, device=dev)) ** 2).sum()
    loss.backward()
    ref = oracle.adjoint(p, tgt)
    assert rel_inf(u0.grad.cpu().numpy(), ref["du0"]) < TOL["f64"]
    assert abs(gam.grad.item() - ref["dgamma"]) < TOL["f64"] * abs(ref["dgamma"])
    assert abs(alp.grad.item() - ref["dalpha"]) < TOL["f64"] * abs(ref["dalpha"])

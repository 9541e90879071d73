"""Pins of the oracle's FP64 adjoint (reverse-time sweep of eq. frac_final) against
complex-step and central finite-difference derivatives of the forward oracle."""
import numpy as np
import pytest

import oracle
from paper_1004_5128_gb300 import synth

H_CS = 1e-30


def adj_problem(bc, ndim=2):
    nx, ny, nz = {1: (23, 1, 1), 2: (9, 7, 1), 3: (5, 4, 3)}[ndim]
    g = synth.SplitMix64(77)
    u0 = g.uniform(nx * ny * nz, 0.0, 1.0)
    target = g.uniform(nx * ny * nz, 0.0, 0.8)
    dt = 0.01
    p = synth.problem(ndim, nx, ny, 0.7, 0.8, dt, 1.0, bc, react=(0.05, -0.3, 0.2, -0.1), K=40,
                      u0=u0, nz=nz)
    return p, target


def J_of(p, target, **over):
    q = dict(p)
    q.update(over)
    if "react" in over:
        q["react"] = list(over["react"])
    u = oracle.run(q)
    return 0.5 * float(np.sum((u - target) ** 2))


def cs_grad(p, target, **im):
    re, imu = oracle.run_cs(p, **im)
    return float(np.sum((re - target) * imu)) / H_CS


@pytest.mark.parametrize("bc,ndim", [(synth.BC_DIRICHLET0, 2), (synth.BC_NOFLUX, 2),
                                     (synth.BC_NOFLUX, 1), (synth.BC_DIRICHLET0, 3),
                                     (synth.BC_NOFLUX, 3)])
def test_adjoint_matches_complex_step(bc, ndim):
    p, target = adj_problem(bc, ndim)
    a = oracle.adjoint(p, target)
    assert abs(a["J"] - J_of(p, target)) < 1e-14 * a["J"]
    dg = cs_grad(p, target, gamma_im=H_CS)
    da = cs_grad(p, target, alpha_im=H_CS)
    assert abs(a["dgamma"] - dg) < 1e-11 * abs(dg)
    assert abs(a["dalpha"] - da) < 1e-11 * abs(da)
    for i in range(4):
        e = np.zeros(4)
        e[i] = H_CS
        dr = cs_grad(p, target, react_im=e)
        assert abs(a["dreact"][i] - dr) < 1e-11 * abs(dr), i
    # dot-product test for dJ/du0: <lambda^0, v> = directional derivative along v
    v = synth.SplitMix64(5).uniform(p["u0"].size, -1.0, 1.0)
    dv = cs_grad(p, target, u0_im=H_CS * v)
    assert abs(float(a["du0"] @ v) - dv) < 1e-11 * abs(dv)


def test_adjoint_matches_central_differences():
    p, target = adj_problem(synth.BC_DIRICHLET0)
    a = oracle.adjoint(p, target)
    h = 1e-4
    fd = (J_of(p, target, gamma=p["gamma"] + h) - J_of(p, target, gamma=p["gamma"] - h)) / (2 * h)
    assert abs(a["dgamma"] - fd) < 1e-6 * abs(fd)
    fd = (J_of(p, target, alpha=p["alpha"] + h) - J_of(p, target, alpha=p["alpha"] - h)) / (2 * h)
    assert abs(a["dalpha"] - fd) < 1e-6 * abs(fd)
    r = np.array(p["react"])
    for i in range(4):
        rp, rm = r.copy(), r.copy()
        rp[i] += h
        rm[i] -= h
        fd = (J_of(p, target, react=rp) - J_of(p, target, react=rm)) / (2 * h)
        assert abs(a["dreact"][i] - fd) < 1e-6 * abs(fd)
    j = 31
    up, um = p["u0"].copy(), p["u0"].copy()
    up[j] += h
    um[j] -= h
    fd = (J_of(p, target, u0=up) - J_of(p, target, u0=um)) / (2 * h)
    assert abs(a["du0"][j] - fd) < 1e-6 * abs(fd)


def test_complex_step_forward_matches_real_forward():
    p, _ = adj_problem(synth.BC_NOFLUX)
    re, im = oracle.run_cs(p)
    assert np.max(np.abs(re - oracle.run(p))) < 1e-13 and np.all(im == 0)


@pytest.mark.parametrize("bc,L", [(synth.BC_DIRICHLET0, 6), (synth.BC_NOFLUX, 13), (synth.BC_NOFLUX, 25)])
def test_short_memory_adjoint_matches_complex_step(bc, L):
    """Short memory (eq. frac_shortmemory): the transposed window M(r) = min(L, K-1-r); a
    dropped window bound (full-memory sums) or an off-by-one in it fails these."""
    p, target = adj_problem(bc)
    p = synth.with_mode(p, synth.MEM_SHORT, L=L)
    a = oracle.adjoint(p, target)
    assert abs(a["J"] - J_of(p, target)) < 1e-14 * a["J"]
    dg = cs_grad(p, target, gamma_im=H_CS)
    da = cs_grad(p, target, alpha_im=H_CS)
    assert abs(a["dgamma"] - dg) < 1e-11 * abs(dg)
    assert abs(a["dalpha"] - da) < 1e-11 * abs(da)
    for i in range(4):
        e = np.zeros(4)
        e[i] = H_CS
        dr = cs_grad(p, target, react_im=e)
        assert abs(a["dreact"][i] - dr) < 1e-11 * abs(dr), i
    v = synth.SplitMix64(6).uniform(p["u0"].size, -1.0, 1.0)
    dv = cs_grad(p, target, u0_im=H_CS * v)
    assert abs(float(a["du0"] @ v) - dv) < 1e-11 * abs(dv)
    # the short-memory gradient differs from the full-memory one (the window matters)
    full = oracle.adjoint(synth.with_mode(p, synth.MEM_FULL), target)
    assert abs(full["dgamma"] - a["dgamma"]) > 1e-6 * abs(a["dgamma"])


@pytest.mark.parametrize("bc,a,rule", [(synth.BC_DIRICHLET0, 3, 0), (synth.BC_NOFLUX, 2, 0),
                                       (synth.BC_NOFLUX, 3, 1), (synth.BC_DIRICHLET0, 5, 0)])
def test_adaptive_memory_adjoint_matches_complex_step(bc, a, rule):
    """Adaptive memory (Definitions 3.1/3.2, Proposition 3.1): delta^r enters step r+m with the
    multiplicity that lag m has in step r+m's schedule (d at a median, 1 on the base interval
    and the tail, 0 elsewhere).  Using one step's schedule for all rows, or the settled weights
    without the tails, fails these."""
    p, target = adj_problem(bc)
    p = synth.with_mode(p, synth.MEM_ADAPTIVE, a=a, rule=rule)
    ad = oracle.adjoint(p, target)
    assert abs(ad["J"] - J_of(p, target)) < 1e-14 * ad["J"]
    dg = cs_grad(p, target, gamma_im=H_CS)
    da = cs_grad(p, target, alpha_im=H_CS)
    assert abs(ad["dgamma"] - dg) < 1e-11 * abs(dg)
    assert abs(ad["dalpha"] - da) < 1e-11 * abs(da)
    for i in range(4):
        e = np.zeros(4)
        e[i] = H_CS
        dr = cs_grad(p, target, react_im=e)
        assert abs(ad["dreact"][i] - dr) < 1e-11 * abs(dr), i
    v = synth.SplitMix64(7).uniform(p["u0"].size, -1.0, 1.0)
    dv = cs_grad(p, target, u0_im=H_CS * v)
    assert abs(float(ad["du0"] @ v) - dv) < 1e-11 * abs(dv)
    # the adaptive gradient differs from the full-memory one (40 steps reach interval 3 at a <= 3)
    full = oracle.adjoint(synth.with_mode(p, synth.MEM_FULL), target)
    assert abs(full["dgamma"] - ad["dgamma"]) > 1e-6 * abs(ad["dgamma"])


def test_adaptive_memory_adjoint_equals_full_when_a_covers_the_run():
    """With a >= K the adaptive schedule is the full one (Definition 3.1): identical gradients."""
    p, target = adj_problem(synth.BC_NOFLUX)
    full = oracle.adjoint(p, target)
    ad = oracle.adjoint(synth.with_mode(p, synth.MEM_ADAPTIVE, a=p["K"]), target)
    for key in ("J", "dgamma", "dalpha"):
        assert ad[key] == full[key], key
    assert np.array_equal(ad["du0"], full["du0"]) and np.array_equal(ad["dreact"], full["dreact"])

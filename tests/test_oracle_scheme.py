"""Pins of the oracle's time stepping (eqs. frac_norxn, deltasimp, frac_final,
frac_shortmemory, eq:adapttime) to results fixed by mathematics, not by the
oracle itself."""
import math

import numpy as np
import pytest

import oracle
from paper_1004_5128_gb300 import synth
from tests.helpers import laplacian_eigenvalue, laplacian_matrix, rel_inf

MODES = [(oracle.MEM_FULL, 0, 0), (oracle.MEM_SHORT, 7, 0), (oracle.MEM_ADAPTIVE, 0, 3),
         (oracle.MEM_ADAPTIVE, 0, 2)]


def small_problem(ndim, bc, nx=13, ny=9, gamma=0.7, react=(0.0, -0.3, 0.0, 0.0), K=60, seed=11, nz=5):
    dx = 0.1
    dt = synth.dt_for_courant(0.12, 1.3, dx, gamma)
    ny = 1 if ndim == 1 else ny
    nz = nz if ndim == 3 else 1
    u0 = synth.SplitMix64(seed).uniform(nx * ny * nz, -1.0, 1.0)
    return synth.problem(ndim, nx, ny, gamma, 1.3, dt, dx, bc, react=react, K=K, u0=u0, nz=nz)


# P2 -------------------------------------------------------------------------
@pytest.mark.parametrize("ndim,bc", [(1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 1)])
def test_gamma_one_is_ftcs_heat_bitwise(ndim, bc):
    """psi(1, m>=1) = 0 exactly, so eq. frac_final is the textbook FTCS heat update."""
    p = small_problem(ndim, bc, gamma=1.0, react=(0.05, -0.4, 0.1, -0.02), K=40)
    S = p["alpha"] * p["dt"] ** 1.0 / p["dx"] ** 2
    r = p["react"]
    u = p["u0"].reshape(p["nz"], p["ny"], p["nx"]).copy()
    for _ in range(p["K"]):
        pad = np.pad(u, 1, mode="edge" if bc == synth.BC_NOFLUX else "constant")
        c = pad[1:-1, 1:-1, 1:-1]
        xp, xm = pad[1:-1, 1:-1, 2:], pad[1:-1, 1:-1, :-2]
        yp, ym = pad[1:-1, 2:, 1:-1], pad[1:-1, :-2, 1:-1]
        zp, zm = pad[2:, 1:-1, 1:-1], pad[:-2, 1:-1, 1:-1]
        if ndim == 1:
            lap = xp - 2.0 * c + xm
        elif ndim == 2:
            lap = xp + xm - 4.0 * c + yp + ym
        else:
            lap = xp + xm - 6.0 * c + yp + ym + zp + zm
        f = r[0] + u * (r[1] + u * (r[2] + u * r[3]))
        u = u + p["dt"] * f + S * lap
    got = oracle.run(p)
    assert np.array_equal(got, u.reshape(-1))


# P3 -------------------------------------------------------------------------
@pytest.mark.parametrize("ndim,bc", [(1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 1)])
@pytest.mark.parametrize("mode,L,a", MODES)
def test_eigenmode_reduces_to_scalar_recursion(ndim, bc, mode, L, a):
    p = synth.with_mode(small_problem(ndim, bc, K=80), mode, L=L, a=a)
    qx, qy, qz = 3, 2, 1
    phi = synth.eigenmode(p, qx, qy, qz)
    lam = laplacian_eigenvalue(p, qx, qy, qz)
    A = oracle.scalar_mode(p, lam)
    got = oracle.run(p, u0=phi)
    assert rel_inf(got, A[-1] * phi) < 1e-12


@pytest.mark.parametrize("g", [0.3, 0.6, 0.9])
def test_scalar_recursion_generating_function(g):
    """Full memory: A(z) = A0 / ((1-z) - dt r1 z + S Lambda z (1-z)^{1-g})."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    K = 120
    p = synth.problem(1, 5, 1, g, 0.9, 0.02, 1.0, synth.BC_DIRICHLET0, react=(0, -0.7, 0, 0), K=K)
    lam = 1.7
    A = oracle.scalar_mode(p, lam, K=K, A0=1.0)
    S = mpmath.mpf(0.9) * mpmath.mpf(0.02) ** mpmath.mpf(g) / mpmath.mpf(1.0) ** 2
    # denominator series coefficients D_n
    D = [mpmath.mpf(0)] * (K + 1)
    D[0] = mpmath.mpf(1)
    D[1] = mpmath.mpf(-1) - mpmath.mpf(0.02) * mpmath.mpf(-0.7)
    for n in range(1, K + 1):
        D[n] += S * lam * (-1) ** (n - 1) * mpmath.binomial(1 - mpmath.mpf(g), n - 1)
    # series division A(z) D(z) = 1
    Ar = [mpmath.mpf(1)]
    for n in range(1, K + 1):
        Ar.append(-sum(D[j] * Ar[n - j] for j in range(1, n + 1)) / D[0])
    ref = np.array([float(x) for x in Ar])
    assert np.max(np.abs(A - ref)) < 1e-13 * np.max(np.abs(ref))


def mittag_leffler(g, z):
    """E_g(-z) for z >= 0."""
    mpmath = pytest.importorskip("mpmath")
    if g == 0.5:
        return float(mpmath.exp(z * z) * mpmath.erfc(z))
    mpmath.mp.dps = 60
    return float(mpmath.nsum(lambda k: (-z) ** k / mpmath.gamma(g * k + 1), [0, mpmath.inf]))


@pytest.mark.parametrize("g", [0.5, 0.75, 0.9, 1.25, 1.5, 1.75])
def test_relaxation_tracks_mittag_leffler(g):
    """N = 1, Dirichlet: delta = -2u, so the scheme discretises du/dt = -mu D^{1-g} u with
    mu = 2 alpha / dx^2, whose solution is E_g(-mu t^g) u0 (for 1 < g < 2, D^{1-g} is a fractional
    integral and the solution has zero initial velocity); the GL error is first order."""
    T, alpha, dx = 1.0, 0.5, 1.0  # mu = 1
    errs = []
    for K in (200, 400, 800):
        dt = T / K
        p = synth.problem(1, 1, 1, g, alpha, dt, dx, synth.BC_DIRICHLET0, K=K, u0=[1.0])
        uK = oracle.run(p)[0]
        errs.append(abs(uK - mittag_leffler(g, T ** g)))
    assert errs[-1] < 5e-3
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.7 < r1 < 2.3 and 1.7 < r2 < 2.3, errs


# P4 -------------------------------------------------------------------------
@pytest.mark.parametrize("mode,L,a", MODES)
@pytest.mark.parametrize("beta", [0.0, 0.8])
@pytest.mark.parametrize("ndim", [2, 3])
def test_mass_balance_noflux(mode, L, a, beta, ndim):
    """Mirror ghosts make every column of L sum to zero, so sum_j delta_j = 0 and
    with f = -beta u the mass obeys M^{k+1} = (1 - beta dt) M^k in every memory mode."""
    p = synth.with_mode(small_problem(ndim, synth.BC_NOFLUX, nx=17, ny=11, react=(0, -beta, 0, 0),
                                      K=150), mode, L=L, a=a)
    p["u0"] = np.abs(p["u0"]) + 0.1
    _, tape = oracle.run(p, tape=True)
    M = tape.sum(axis=1)
    ref = M[0] * (1.0 - beta * p["dt"]) ** np.arange(p["K"] + 1)
    assert np.max(np.abs(M - ref)) / M[0] < 1e-12


# P5 -------------------------------------------------------------------------
@pytest.mark.parametrize("ndim,bc", [(1, 0), (2, 1)])
def test_modes_coincide_when_window_covers_history(ndim, bc):
    p = small_problem(ndim, bc, K=50)
    full = oracle.run(p)
    short = oracle.run(synth.with_mode(p, oracle.MEM_SHORT, L=50))
    adapt = oracle.run(synth.with_mode(p, oracle.MEM_ADAPTIVE, a=60))
    assert np.array_equal(full, short) and np.array_equal(full, adapt)
    # ... and genuinely differ once the window is shorter than the history
    assert not np.array_equal(full, oracle.run(synth.with_mode(p, oracle.MEM_SHORT, L=10)))
    assert not np.array_equal(full, oracle.run(synth.with_mode(p, oracle.MEM_ADAPTIVE, a=3)))


# P7 -------------------------------------------------------------------------
@pytest.mark.parametrize("ndim,bc,nx,ny", [(1, 0, 4, 1), (1, 1, 5, 1), (2, 0, 3, 2), (2, 1, 2, 3),
                                            (3, 0, 2, 2), (3, 1, 2, 1)])
@pytest.mark.parametrize("mode,L,a", MODES)
def test_dense_linear_system(ndim, bc, nx, ny, mode, L, a):
    """For linear f = r0 + r1 u the K steps form one block-lower-triangular linear system in
    (u^1 .. u^K); a dense library solve of it must equal the time stepping."""
    K = 14
    p = synth.with_mode(small_problem(ndim, bc, nx=nx, ny=ny, react=(0.2, -0.5, 0, 0), K=K, nz=2),
                        mode, L=L, a=a)
    N = p["u0"].size
    Lm = laplacian_matrix(p)
    S = p["alpha"] * p["dt"] ** p["gamma"] / p["dx"] ** 2
    mpmath = pytest.importorskip("mpmath")
    psi = np.array([float((-1) ** m * mpmath.binomial(1 - mpmath.mpf(p["gamma"]), m))
                    for m in range(K + 1)])
    A = np.zeros((K * N, K * N))
    b = np.zeros(K * N)
    I = np.eye(N)
    # block row k: u^{k+1} - (1 + dt r1) u^k - S sum c_m L u^{k-m} = dt r0
    for k in range(K):
        rows = slice(k * N, (k + 1) * N)
        A[rows, rows] = I  # u^{k+1}
        coef = {k: -(1.0 + p["dt"] * p["react"][1]) * I}
        lag, mult = oracle.schedule(mode, L, a, 0, k)
        for m, d in zip(lag, mult):
            coef[k - m] = coef.get(k - m, 0) - S * d * psi[m] * Lm
        b[rows] = p["dt"] * p["react"][0]
        for r, blk in coef.items():
            if r == 0:
                b[rows] -= blk @ p["u0"]
            else:
                A[rows, (r - 1) * N:r * N] += blk
    U = np.linalg.solve(A, b)
    got = oracle.run(p)
    assert rel_inf(got, U[-N:]) < 1e-12


@pytest.mark.parametrize("g", [0.3, 0.5, 0.8, 1.0, 1.3, 1.5, 1.9])
def test_stability_threshold_is_checkerboard_bound(g):
    """Just below S = 2^g / (4 ndim) the highest mode (Lambda = 4 ndim) decays, just above it grows:
    the bound the library enforces is the scheme's threshold for 0 < g < 2."""
    bound = synth.stability_bound(g, 1)
    amp = []
    for f in (0.97, 1.03):
        p = synth.problem(1, 5, 1, g, 1.0, 1.0, 1.0 / math.sqrt(f * bound), synth.BC_DIRICHLET0, K=3000)
        A = oracle.scalar_mode(p, 4.0, K=3000)
        amp.append(np.max(np.abs(A[-500:])))
    assert amp[0] < 0.1
    assert not np.isfinite(amp[1]) or amp[1] > 1e20

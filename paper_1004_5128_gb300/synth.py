"""Seeded synthetic inputs for the fractional reaction-diffusion workloads.

This module only draws numbers and lays out problem descriptions; it holds
none of the scheme's arithmetic (no weights, no stencil, no memory sum).  It is
the one module shared by the CUDA path (its tests and benchmark) and by the
FP64 CPU oracle's tests, so that both sides see bit-identical inputs.

Random numbers come from SplitMix64 (S. Vigna, "Further scramblings of
Marsaglia's xorshift generators", and the splitmix64.c reference generator):
state advances by the golden-ratio increment 0x9E3779B97F4A7C15 and each
output is the state passed through two xor-shift-multiply rounds.  Doubles use
the top 53 bits, so every draw is exactly representable and identical on any
machine.

Problem descriptions are plain dicts with the fields of the paper's scheme
(eq. frac_final, Section 2.2): grid (ndim, nx, ny), gamma, alpha, dt, dx,
boundary condition, cubic reaction f(u) = r0 + r1 u + r2 u^2 + r3 u^3, memory
mode (full / short window L / adaptive base a), step count K and u0.
"""
from __future__ import annotations

import math

import numpy as np

BC_DIRICHLET0 = 0
BC_NOFLUX = 1
MEM_FULL = 0
MEM_SHORT = 1
MEM_ADAPTIVE = 2
ADAPT_PAPER = 0
ADAPT_PARTITION = 1

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based SplitMix64 stream: output i mixes seed + (i+1)*golden."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            idx = np.arange(1, n + 1, dtype=np.uint64)
            z = self.state + idx * _GOLDEN
            self.state = self.state + np.uint64(n) * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def randint(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Integers uniform on [lo, hi] inclusive."""
        u = self.uniform(n)
        return np.minimum(lo + np.floor(u * (hi - lo + 1)).astype(np.int64), hi)


def dt_for_courant(S: float, alpha: float, dx: float, gamma: float) -> float:
    """Time step that gives S = alpha * dt^gamma / dx^2 (the scheme's prefactor)."""
    return (S * dx * dx / alpha) ** (1.0 / gamma)


def stability_bound(gamma: float, ndim: int) -> float:
    """Largest stable S for the full-memory explicit scheme (checkerboard mode)."""
    return 2.0 ** gamma / (4.0 * ndim)


def problem(ndim, nx, ny, gamma, alpha, dt, dx, bc, react=(0.0, 0.0, 0.0, 0.0),
            mem_mode=MEM_FULL, mem_L=0, mem_a=0, adaptive_rule=ADAPT_PAPER, K=1, u0=None, nz=1):
    ny = 1 if ndim == 1 else ny
    nz = nz if ndim == 3 else 1
    p = dict(ndim=int(ndim), nx=int(nx), ny=int(ny), nz=int(nz), gamma=float(gamma),
             alpha=float(alpha), dt=float(dt), dx=float(dx), bc=int(bc),
             react=[float(r) for r in react], mem_mode=int(mem_mode), mem_L=int(mem_L),
             mem_a=int(mem_a), adaptive_rule=int(adaptive_rule), K=int(K))
    if u0 is None:
        u0 = np.zeros(nx * ny * nz)
    p["u0"] = np.ascontiguousarray(np.asarray(u0, dtype=np.float64).reshape(-1))
    assert p["u0"].size == nx * ny * nz
    return p


def gaussians_2d(n: int, seed: int, count: int = 8, sigma_frac: float = 0.02,
                 amp=(0.5, 1.0), cell_centred: bool = True) -> np.ndarray:
    """Sum of `count` seeded Gaussians on an n x n grid of the unit square.

    Centres ~ U[0.1, 0.9]^2, amplitudes ~ U[amp], sigma = sigma_frac (in units
    of the domain), exp(-r^2 / (2 sigma^2)).  Returned row-major (y, x) flat.
    """
    g = SplitMix64(seed)
    cx = g.uniform(count, 0.1, 0.9)
    cy = g.uniform(count, 0.1, 0.9)
    a = g.uniform(count, amp[0], amp[1])
    off = 0.5 if cell_centred else 1.0
    xs = (np.arange(n) + off) / (n if cell_centred else n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    u = np.zeros((n, n))
    for i in range(count):
        u += a[i] * np.exp(-((X - cx[i]) ** 2 + (Y - cy[i]) ** 2) / (2.0 * sigma_frac ** 2))
    return u.reshape(-1)


def gaussian_1d(n: int, width: float = 0.005) -> np.ndarray:
    """u0(x) = exp(-(x - 0.5)^2 / width) at the interior points x_j = (j+1)/(n+1)."""
    x = (np.arange(n) + 1.0) / (n + 1.0)
    return np.exp(-((x - 0.5) ** 2) / width)


# ---------------------------------------------------------------------------
# The five workloads.  Each returns a problem dict (u0 included).
# ---------------------------------------------------------------------------

def config1(K: int = 1000):
    """1-D, N=256 on x in [0,1], Dirichlet 0, gamma=0.5, alpha=1, f=0, S=0.2, full, FP64."""
    n = 256
    dx = 1.0 / (n + 1)
    gamma, alpha = 0.5, 1.0
    dt = dt_for_courant(0.2, alpha, dx, gamma)
    return problem(1, n, 1, gamma, alpha, dt, dx, BC_DIRICHLET0, K=K, u0=gaussian_1d(n))


def config2(mode: int = MEM_FULL, K: int = 5000, n: int = 256, L: int = 500, a: int = 10,
            rule: int = ADAPT_PAPER):
    """2-D n x n (256), no-flux, gamma=0.8, alpha=0.5, f=-0.1u, S=0.1, 8 Gaussians (seed 2)."""
    dx = 1.0 / n
    gamma, alpha = 0.8, 0.5
    dt = dt_for_courant(0.1, alpha, dx, gamma)
    u0 = gaussians_2d(n, seed=2)
    return problem(2, n, n, gamma, alpha, dt, dx, BC_NOFLUX, react=(0.0, -0.1, 0.0, 0.0),
                   mem_mode=mode, mem_L=L if mode == MEM_SHORT else 0,
                   mem_a=a if mode == MEM_ADAPTIVE else 0, adaptive_rule=rule, K=K, u0=u0)


def config3(n: int = 512, K: int = 20000):
    """2-D n x n (512), lattice dx=1, Dirichlet 0, gamma=0.6, alpha=1, f=u(1-u)-0.05u, S=0.1,
    u0 ~ U[0, 0.1] (seed 3).  The oracle check uses n=128, K=2000 with the same dt."""
    gamma, alpha, dx = 0.6, 1.0, 1.0
    dt = dt_for_courant(0.1, alpha, dx, gamma)
    u0 = SplitMix64(3).uniform(n * n, 0.0, 0.1)
    return problem(2, n, n, gamma, alpha, dt, dx, BC_DIRICHLET0, react=(0.0, 0.95, -1.0, 0.0),
                   K=K, u0=u0)


def config4(mode: int = MEM_FULL, a: int = 10, count: int = 64, seed: int = 4,
            steps_range=(1000, 8000), side_range=(64, 384), n1_range=(64, 4096)):
    """Batch of `count` uneven instances: half 1-D (N log-uniform), half 2-D (side log-uniform),
    gamma ~ U[0.3,0.95], alpha log-uniform [0.1,2], f=-k u with k ~ U[0,0.2],
    K ~ U{steps_range}, Dirichlet 0 on the unit domain, S = half the stability bound."""
    g = SplitMix64(seed)
    half = count // 2
    n1 = np.exp(g.uniform(half, math.log(n1_range[0]), math.log(n1_range[1]))).astype(np.int64)
    side = np.exp(g.uniform(count - half, math.log(side_range[0]),
                            math.log(side_range[1]))).astype(np.int64)
    gam = g.uniform(count, 0.3, 0.95)
    alp = np.exp(g.uniform(count, math.log(0.1), math.log(2.0)))
    kr = g.uniform(count, 0.0, 0.2)
    Ks = g.randint(count, steps_range[0], steps_range[1])
    seeds = g.randint(count, 1, 1 << 30)
    probs = []
    for i in range(count):
        if i < half:
            ndim, nx, ny = 1, int(n1[i]), 1
            dx = 1.0 / (nx + 1)
            u0 = gaussian_1d(nx)
        else:
            ndim, nx = 2, int(side[i - half])
            ny = nx
            dx = 1.0 / (nx + 1)
            u0 = gaussians_2d(nx, seed=int(seeds[i]), cell_centred=False)
        S = 0.5 * stability_bound(float(gam[i]), ndim)
        dt = dt_for_courant(S, float(alp[i]), dx, float(gam[i]))
        probs.append(problem(ndim, nx, ny, float(gam[i]), float(alp[i]), dt, dx, BC_DIRICHLET0,
                             react=(0.0, -float(kr[i]), 0.0, 0.0), mem_mode=mode,
                             mem_a=a if mode == MEM_ADAPTIVE else 0, K=int(Ks[i]), u0=u0))
    return probs


def config5(n: int = 128, K: int = 4000, target: bool = False):
    """Adjoint workload: 2-D n x n (128), lattice dx=1, Dirichlet 0, dt=0.005, f=-0.1u,
    gamma=0.7, alpha=0.8 (target run: gamma=0.65, alpha=1.0), 8 Gaussians sigma=0.02 n (seed 5)."""
    gamma, alpha = (0.65, 1.0) if target else (0.7, 0.8)
    u0 = gaussians_2d(n, seed=5, cell_centred=False)
    return problem(2, n, n, gamma, alpha, 0.005, 1.0, BC_DIRICHLET0, react=(0.0, -0.1, 0.0, 0.0),
                   K=K, u0=u0)


def with_mode(p: dict, mode: int, L: int = 0, a: int = 0, rule: int = ADAPT_PAPER) -> dict:
    q = dict(p)
    q["mem_mode"] = int(mode)
    q["mem_L"] = int(L)
    q["mem_a"] = int(a)
    q["adaptive_rule"] = int(rule)
    return q


def eigenmode(p: dict, qx: int, qy: int = 1, qz: int = 1) -> np.ndarray:
    """Discrete Laplacian eigenvector for p's grid and boundary condition.

    Dirichlet 0: sin(q pi (j+1)/(n+1)); no-flux (cell-centred mirror): cos(q pi (j+1/2)/n).
    Product over the axes in 2-D / 3-D, row-major (z, y, x) flat.
    """
    def axis(n, q):
        j = np.arange(n, dtype=np.float64)
        if p["bc"] == BC_DIRICHLET0:
            return np.sin(q * math.pi * (j + 1.0) / (n + 1.0))
        return np.cos(q * math.pi * (j + 0.5) / n)
    ex = axis(p["nx"], qx)
    if p["ndim"] == 1:
        return ex
    ey = axis(p["ny"], qy)
    if p["ndim"] == 2:
        return np.outer(ey, ex).reshape(-1)
    ez = axis(p["nz"], qz)
    return np.einsum("z,y,x->zyx", ez, ey, ex).reshape(-1)


def workload_runs(name: str, K: int = 0, modes: str = ""):
    """Named workloads as [(run name, problem or list of problems, solver options)].

    c1: config 1 (FP64); c2: config 2 in its three memory modes; c3: config 3 with BF16, FP16
    and FP32 history; c4: the 64-instance batch, full and adaptive; c5: the adjoint problem;
    c2cl: config 2's adaptive schedule in closed loop (tau 0.1 and 0.01) and open loop.
    K overrides every step count; modes keeps only the named runs.
    """
    if name == "c2":
        runs = [("full", config2(MEM_FULL), {}), ("short", config2(MEM_SHORT), {}),
                ("adaptive", config2(MEM_ADAPTIVE), {})]
    elif name == "c1":
        runs = [("full", config1(), {"state": "f64"})]
    elif name == "c3":
        # temporally blocked, blocks of 64, far rows on the tensor cores (FP32 history as a pair of
        # FP16 planes)
        runs = [("bf16", config3(), {"hist": "bf16", "time_block": 64}),
                ("f16", config3(), {"hist": "f16", "time_block": 64}),
                ("f32", config3(), {"time_block": 64})]
    elif name == "c4":
        runs = [("full", config4(MEM_FULL), {}), ("adaptive", config4(MEM_ADAPTIVE), {})]
    elif name == "c5":
        runs = [("adjoint", config5(), {})]
    elif name == "c2cl":
        # config 2's adaptive schedule (a = 10) with feedback from the history, against the open
        # loop on the same per-step kernel
        runs = [("open", config2(MEM_ADAPTIVE), {"time_block": 0}),
                ("tau0.1", config2(MEM_ADAPTIVE), {"closed_tau": 0.1}),
                ("tau0.01", config2(MEM_ADAPTIVE), {"closed_tau": 0.01})]
    else:
        raise ValueError(f"unknown workload {name}")
    if modes:
        runs = [r for r in runs if r[0] in modes.split(",")]
    if K:
        for _, p, _ in runs:
            for q in (p if isinstance(p, list) else [p]):
                q["K"] = K
    return runs

"""Shared test helpers (no method arithmetic beyond textbook facts)."""
import math

import numpy as np

from paper_1004_5128_gb300 import synth


def laplacian_eigenvalue(p: dict, qx: int, qy: int = 1, qz: int = 1) -> float:
    """Lambda with L(phi) = -Lambda phi for the unnormalised 3/5-point stencil.

    For the Dirichlet sine mode sin(q pi (j+1)/(n+1)) and the cell-centred
    cosine mode cos(q pi (j+1/2)/n): u_{j+1} - 2u_j + u_{j-1} = -4 sin^2(q pi h/2) u_j,
    with h = 1/(n+1) or 1/n, summed over the axes in 2-D.
    """
    def lam(n, q):
        h = 1.0 / (n + 1.0) if p["bc"] == synth.BC_DIRICHLET0 else 1.0 / n
        return 4.0 * math.sin(q * math.pi * h / 2.0) ** 2
    v = lam(p["nx"], qx)
    if p["ndim"] >= 2:
        v += lam(p["ny"], qy)
    if p["ndim"] == 3:
        v += lam(p["nz"], qz)
    return v


def rel_inf(a, ref) -> float:
    """Infinity-norm error relative to max |ref|."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(a - ref)) / max(np.max(np.abs(ref)), 1e-300))


def laplacian_matrix(p: dict) -> np.ndarray:
    """Dense L of eq. deltasimp with the ghost rule of p['bc'], built row by row."""
    nx, ny, nz = p["nx"], p["ny"], p.get("nz", 1)
    N = nx * ny * nz
    L = np.zeros((N, N))
    mirror = p["bc"] == synth.BC_NOFLUX
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = (z * ny + y) * nx + x
                L[i, i] -= 2 * p["ndim"]
                nbrs = [(x + 1, y, z), (x - 1, y, z)]
                if p["ndim"] >= 2:
                    nbrs += [(x, y + 1, z), (x, y - 1, z)]
                if p["ndim"] == 3:
                    nbrs += [(x, y, z + 1), (x, y, z - 1)]
                for (xx, yy, zz) in nbrs:
                    if 0 <= xx < nx and 0 <= yy < ny and 0 <= zz < nz:
                        L[i, (zz * ny + yy) * nx + xx] += 1.0
                    elif mirror:
                        L[i, i] += 1.0
    return L

"""ctypes front end of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the package smoke check
and the benchmark's CPU-baseline / reference leg, never by the product path.
It shares no code with the CUDA library and never loads it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

BC_DIRICHLET0, BC_NOFLUX = 0, 1
MEM_FULL, MEM_SHORT, MEM_ADAPTIVE = 0, 1, 2
ADAPT_PAPER, ADAPT_PARTITION = 0, 1


class OrProblem(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("gamma", ctypes.c_double), ("alpha", ctypes.c_double),
        ("dt", ctypes.c_double), ("dx", ctypes.c_double),
        ("bc", ctypes.c_int), ("react", ctypes.c_double * 4),
        ("mem_mode", ctypes.c_int), ("mem_L", ctypes.c_int), ("mem_a", ctypes.c_int),
        ("adaptive_rule", ctypes.c_int), ("nz", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        pp = ctypes.POINTER(OrProblem)
        L.or_weights.argtypes = [ctypes.c_double, ctypes.c_long, dp, dp]
        L.or_schedule.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_long, ctypes.c_int,
                                  ctypes.c_long, lp, lp]
        L.or_schedule.restype = ctypes.c_long
        L.or_run.argtypes = [pp, dp, ctypes.c_long, dp, dp, ctypes.c_int]
        L.or_run_cs.argtypes = [pp, ctypes.c_double, ctypes.c_double, dp, dp, dp, ctypes.c_long,
                                dp, dp]
        L.or_adjoint.argtypes = [pp, dp, ctypes.c_long, dp, dp, dp, dp, dp, dp, ctypes.c_int]
        L.or_run_bf16.argtypes = [pp, dp, ctypes.c_long, ctypes.c_long, ctypes.c_long, dp, ctypes.c_int]
        L.or_run_closed.argtypes = [pp, dp, ctypes.c_long, ctypes.c_double, dp, lp, dp, ctypes.c_int]
        L.or_round_bf16.argtypes = [ctypes.c_double]
        L.or_round_bf16.restype = ctypes.c_double
        L.or_scalar_mode.argtypes = [ctypes.c_double] * 6 + [ctypes.c_int, ctypes.c_long,
                                                             ctypes.c_long, ctypes.c_int,
                                                             ctypes.c_double, ctypes.c_long, dp]
        for f in (L.or_weights, L.or_run, L.or_run_cs, L.or_adjoint, L.or_scalar_mode, L.or_run_bf16,
                  L.or_run_closed):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _problem(p: dict) -> OrProblem:
    s = OrProblem()
    s.ndim, s.nx, s.ny = p["ndim"], p["nx"], p["ny"]
    s.gamma, s.alpha, s.dt, s.dx = p["gamma"], p["alpha"], p["dt"], p["dx"]
    s.bc = p["bc"]
    for i in range(4):
        s.react[i] = p["react"][i]
    s.mem_mode, s.mem_L, s.mem_a = p["mem_mode"], p["mem_L"], p["mem_a"]
    s.adaptive_rule = p.get("adaptive_rule", ADAPT_PAPER)
    s.nz = p.get("nz", 1)
    return s


def weights(gamma: float, n: int, with_derivative: bool = False):
    psi = np.empty(n)
    dpsi = np.empty(n) if with_derivative else None
    if lib().or_weights(gamma, n, _dp(psi), _dp(dpsi)) != 0:
        raise ValueError("or_weights failed")
    return (psi, dpsi) if with_derivative else psi


def schedule(mode: int, L: int, a: int, rule: int, k: int):
    lag = np.empty(k + 1, dtype=np.int64)
    mult = np.empty(k + 1, dtype=np.int64)
    lp = ctypes.POINTER(ctypes.c_long)
    n = lib().or_schedule(mode, L, a, rule, k, lag.ctypes.data_as(lp), mult.ctypes.data_as(lp))
    if n < 0:
        raise ValueError("or_schedule failed")
    return lag[:n].copy(), mult[:n].copy()


def run(p: dict, K: int | None = None, u0=None, tape: bool = False, threads: int = 0):
    """u^K (and the (K+1, N) tape of u^0..u^K if tape=True)."""
    K = p["K"] if K is None else K
    u0 = np.ascontiguousarray(p["u0"] if u0 is None else u0, dtype=np.float64)
    N = p["nx"] * p["ny"] * p.get("nz", 1)
    uK = np.empty(N)
    tp = np.empty((K + 1, N)) if tape else None
    s = _problem(p)
    rc = lib().or_run(ctypes.byref(s), _dp(u0), K, _dp(uK), _dp(tp), threads)
    if rc != 0:
        raise ValueError(f"or_run failed ({rc})")
    return (uK, tp) if tape else uK


def run_bf16(p: dict, blk: int, head: int, K: int | None = None, threads: int = 0):
    """u^K with history rows stored in BF16 beyond the FP32 window: at step k, lags up to
    head + (k mod blk) (blk = 0: up to head) use delta as computed, older lags its BF16 rounding
    (the storage rule of the mixed-precision GPU runs)."""
    K = p["K"] if K is None else K
    u0 = np.ascontiguousarray(p["u0"], dtype=np.float64)
    uK = np.empty(p["nx"] * p["ny"] * p.get("nz", 1))
    s = _problem(p)
    rc = lib().or_run_bf16(ctypes.byref(s), _dp(u0), K, blk, head, _dp(uK), threads)
    if rc != 0:
        raise ValueError(f"or_run_bf16 failed ({rc})")
    return uK


def run_closed(p: dict, tau: float, K: int | None = None, threads: int = 0, margin: bool = False):
    """Closed-loop adaptive memory (reading of the Discussion): (u^K, terms used over the run).
    A median stands for its increment only while the history's relative variation across the
    increment, from per-row maxima of |delta^r - delta^(r-1)| and |delta^r|, stays below tau.
    margin=True appends the smallest |V - tau| / tau over the run's decisions (inf if none)."""
    K = p["K"] if K is None else K
    u0 = np.ascontiguousarray(p["u0"], dtype=np.float64)
    uK = np.empty(p["nx"] * p["ny"] * p.get("nz", 1))
    n = ctypes.c_long(0)
    mg = ctypes.c_double(0.0)
    s = _problem(p)
    rc = lib().or_run_closed(ctypes.byref(s), _dp(u0), K, float(tau), _dp(uK), ctypes.byref(n),
                             ctypes.byref(mg), threads)
    if rc != 0:
        raise ValueError(f"or_run_closed failed ({rc})")
    return (uK, int(n.value), float(mg.value)) if margin else (uK, int(n.value))


def round_bf16(x: float) -> float:
    """x rounded to BF16 (8 significant bits, to nearest, ties to even)."""
    return lib().or_round_bf16(float(x))


def run_cs(p: dict, K: int | None = None, gamma_im=0.0, alpha_im=0.0, react_im=None,
           u0_im=None):
    """Complex-step forward: returns (Re u^K, Im u^K)."""
    K = p["K"] if K is None else K
    N = p["nx"] * p["ny"] * p.get("nz", 1)
    u0 = np.ascontiguousarray(p["u0"], dtype=np.float64)
    ui = None if u0_im is None else np.ascontiguousarray(u0_im, dtype=np.float64)
    ri = None if react_im is None else np.ascontiguousarray(react_im, dtype=np.float64)
    re, im = np.empty(N), np.empty(N)
    s = _problem(p)
    rc = lib().or_run_cs(ctypes.byref(s), gamma_im, alpha_im, _dp(ri), _dp(u0), _dp(ui), K,
                         _dp(re), _dp(im))
    if rc != 0:
        raise ValueError(f"or_run_cs failed ({rc})")
    return re, im


def adjoint(p: dict, target, K: int | None = None, threads: int = 0):
    """FP64 adjoint: dict with J, du0, dgamma, dalpha, dreact[4]."""
    K = p["K"] if K is None else K
    N = p["nx"] * p["ny"] * p.get("nz", 1)
    u0 = np.ascontiguousarray(p["u0"], dtype=np.float64)
    tg = np.ascontiguousarray(target, dtype=np.float64)
    J, dg, da = np.zeros(1), np.zeros(1), np.zeros(1)
    du0, dr = np.empty(N), np.empty(4)
    s = _problem(p)
    rc = lib().or_adjoint(ctypes.byref(s), _dp(u0), K, _dp(tg), _dp(J), _dp(du0), _dp(dg),
                          _dp(da), _dp(dr), threads)
    if rc != 0:
        raise ValueError(f"or_adjoint failed ({rc})")
    return dict(J=float(J[0]), du0=du0, dgamma=float(dg[0]), dalpha=float(da[0]), dreact=dr)


def scalar_mode(p: dict, Lambda: float, K: int | None = None, A0: float = 1.0):
    """A^0..A^K of one Laplacian eigenmode under p's weights, schedule and linear reaction."""
    K = p["K"] if K is None else K
    out = np.empty(K + 1)
    rc = lib().or_scalar_mode(p["gamma"], p["alpha"], p["dt"], p["dx"], p["react"][1], Lambda,
                              p["mem_mode"], p["mem_L"], p["mem_a"],
                              p.get("adaptive_rule", ADAPT_PAPER), A0, K, _dp(out))
    if rc != 0:
        raise ValueError("or_scalar_mode failed")
    return out

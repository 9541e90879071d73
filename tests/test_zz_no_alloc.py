"""fd_run_static, the allocation-free entry point, against the workspace entry point fd_run.

fd_run_static serves callers that cannot allocate device memory (a plugin handed only a stream
by an application that owns the GPU allocator, or a loop that may not allocate once started):
its scratch is the library's static device array.  Through the C ABI, two calls in a row must
each reproduce fd_run's result within the FP32 parity tolerance of the other tests (1e-5
relative to max |u|; 1e-12 for FP64), and a problem larger than the static array is refused.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1004_5128_gb300 import FRD, make_problem, synth
from paper_1004_5128_gb300 import _lib as L
from tests.helpers import rel_inf

pytestmark = pytest.mark.gpu

GEOM = dict(tile_threads=128, chunk_terms=32, stage_rows=8, stages=3, ctas_per_sm=2)


def static_run(fp, u0: torch.Tensor, nsteps: int) -> np.ndarray:
    out = torch.empty_like(u0)
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.lib().fd_run_static(ctypes.byref(fp), ctypes.c_void_p(u0.data_ptr()), nsteps,
                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert rc == 0, L.strerror(rc)
    return out.cpu().double().numpy()


@pytest.mark.parametrize("case", ["f32_adaptive_2d", "f32_short_noflux", "f64_full_1d", "bf16_full_2d"])
def test_static_entry_matches_workspace_entry_twice(case):
    if case == "f32_adaptive_2d":
        p = synth.with_mode(synth.config2(K=300, n=72), synth.MEM_ADAPTIVE, a=3)
        kw, tol = dict(state="f32"), 1e-5
    elif case == "f32_short_noflux":
        p = synth.with_mode(synth.config2(K=250, n=50), synth.MEM_SHORT, L=40)
        kw, tol = dict(state="f32"), 1e-5
    elif case == "f64_full_1d":
        p = synth.config1(K=400)
        kw, tol = dict(state="f64"), 1e-12
    else:
        p = synth.config3(n=64, K=300)
        kw, tol = dict(hist="bf16", kahan=True), 1e-5
    ref_solver = FRD(p, **kw, **GEOM)
    ref_solver.set_state(p["u0"])
    ref = ref_solver.run(p["K"]).cpu().double().numpy()
    fp = make_problem(p, **kw, **GEOM)
    u0 = torch.from_numpy(p["u0"]).to("cuda", ref_solver.dtype)
    first = static_run(fp, u0, p["K"])
    second = static_run(fp, u0, p["K"])
    assert rel_inf(first, ref) < tol
    assert rel_inf(second, ref) < tol


def test_static_entry_refuses_problems_beyond_its_array():
    p = synth.config2(K=5000)  # 1.3 GB of history
    fp = make_problem(p)
    u0 = torch.from_numpy(p["u0"]).to("cuda", torch.float32)
    out = torch.empty_like(u0)
    rc = L.lib().fd_run_static(ctypes.byref(fp), ctypes.c_void_p(u0.data_ptr()), p["K"],
                               ctypes.c_void_p(out.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == L.FD_ERR_WORKSPACE


def _three_dims(n: int = 14, K: int = 160):
    """3-D 14^3 (2744 points: a ragged last tile), no-flux, adaptive a=3."""
    p = synth.problem(3, n, n, 0.7, 0.6, synth.dt_for_courant(0.1, 0.6, 1.0, 0.7), 1.0,
                      synth.BC_NOFLUX, react=(0.0, -0.1, 0.0, 0.0), mem_mode=synth.MEM_ADAPTIVE,
                      mem_a=3, K=K, u0=synth.SplitMix64(33).uniform(n ** 3, 0, 1), nz=n)
    return p


def test_static_entry_alternating_problems_against_oracle():
    """Differently shaped problems in a row through the one shared array, each against the FP64
    oracle: a ragged 2-D grid with BF16 history, a 3-D grid with FP16 (scaled) history, then the
    first problem again, whose result must not depend on what the second call left behind.
    The first call uses the library's default launch geometry."""
    import oracle

    a = synth.problem(2, 45, 37, 0.75, 0.7, synth.dt_for_courant(0.15, 0.7, 1.0, 0.75), 1.0,
                      synth.BC_DIRICHLET0, react=(0.01, -0.2, 0.3, -0.4), K=220,
                      u0=synth.SplitMix64(21).uniform(45 * 37, 0, 1))
    b = _three_dims()
    fa = make_problem(a, hist="bf16", kahan=True)            # default geometry
    fb = make_problem(b, hist="f16", kahan=True, **GEOM)
    ua = torch.from_numpy(a["u0"]).to("cuda", torch.float32)
    ub = torch.from_numpy(b["u0"]).to("cuda", torch.float32)
    ref_a, ref_b = oracle.run(a), oracle.run(b)
    first = static_run(fa, ua, a["K"])
    other = static_run(fb, ub, b["K"])
    again = static_run(fa, ua, a["K"])
    assert rel_inf(first, ref_a) < 2e-3
    assert rel_inf(other, ref_b) < 2e-3
    assert rel_inf(again, ref_a) < 2e-3
    assert np.array_equal(first, again)

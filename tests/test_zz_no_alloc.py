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

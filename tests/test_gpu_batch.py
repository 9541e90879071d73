"""GPU parity of the multi-instance persistent launch (one CUDA graph replay) against the
oracle, instance by instance."""
import numpy as np
import pytest
import torch

import oracle
from paper_1004_5128_gb300 import FRD, FRDBatch, synth
from paper_1004_5128_gb300 import _lib as L
from tests.helpers import rel_inf

pytestmark = pytest.mark.gpu


def run_batch(probs, **kw):
    b = FRDBatch(probs, **kw)
    for i, p in enumerate(probs):
        b.set_state(i, p["u0"])
    b.run()
    out = [b.state(i).cpu().double().numpy() for i in range(len(probs))]
    assert b.status() == 0
    return out, b


@pytest.mark.parametrize("mode", [synth.MEM_FULL, synth.MEM_ADAPTIVE])
def test_small_uneven_batch_vs_oracle(mode):
    probs = synth.config4(mode=mode, count=12, steps_range=(50, 400), side_range=(9, 70),
                          n1_range=(5, 2500))
    out, _ = run_batch(probs, chunk_terms=24)
    for p, got in zip(probs, out):
        assert rel_inf(got, oracle.run(p)) < 1e-5


def test_batch_replay_is_bitwise_identical_and_matches_single_runs():
    probs = synth.config4(count=6, steps_range=(100, 300), side_range=(20, 50), n1_range=(40, 900))
    b = FRDBatch(probs, chunk_terms=32)
    res = []
    for _ in range(2):
        for i, p in enumerate(probs):
            b.set_state(i, p["u0"])
        b.run()
        res.append([b.state(i).cpu().numpy() for i in range(len(probs))])
        assert b.status() == 0
    for x, y in zip(*res):
        assert np.array_equal(x, y)
    for p, x in zip(probs, res[0]):
        s = FRD(p, chunk_terms=32, tile_threads=256)
        s.set_state(p["u0"])
        assert np.array_equal(s.run(p["K"]).cpu().numpy(), x)


def test_run_batch_one_shot_host_buffers():
    probs = synth.config4(count=4, steps_range=(60, 120), side_range=(12, 30), n1_range=(30, 300))
    fps = [L.FdProblem() for _ in probs]
    from paper_1004_5128_gb300 import make_problem
    fps = [make_problem(p) for p in probs]
    nbytes = L.fd_batch_workspace_bytes(fps)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    host = [torch.from_numpy(p["u0"].astype(np.float32)).pin_memory() for p in probs]
    L.fd_run_batch(fps, [h.data_ptr() for h in host], ws.data_ptr(), nbytes,
                   torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for p, h in zip(probs, host):
        assert rel_inf(h.double().numpy(), oracle.run(p)) < 1e-5


@pytest.mark.parametrize("mode", [synth.MEM_FULL, synth.MEM_ADAPTIVE])
def test_config4_full_batch_sampled_vs_oracle(mode):
    """The 64-instance workload (steps 1000-8000, 1-D N 64-4096, 2-D side 64-384) in one launch;
    the instances the oracle finishes quickly are compared element by element, every instance
    is checked finite."""
    probs = synth.config4(mode=mode)
    out, _ = run_batch(probs)
    cost = [p["nx"] * p["ny"] * p["K"] ** 2 for p in probs]
    for i in np.argsort(cost)[:3]:
        assert rel_inf(out[i], oracle.run(probs[i])) < 1e-5
    assert all(np.all(np.isfinite(o)) for o in out)


@pytest.mark.parametrize("tb", [4, 8, 16])
@pytest.mark.parametrize("mode", [synth.MEM_FULL, synth.MEM_SHORT, synth.MEM_ADAPTIVE])
def test_small_uneven_blocked_batch_vs_oracle(tb, mode):
    """The temporally blocked kernel over a batch of uneven 1-D/2-D instances with their own
    step counts (not multiples of the block), chunk sizes, short windows and adaptive base
    intervals (a = 2 .. 10, both median rules)."""
    probs = synth.config4(count=10, steps_range=(50, 300), side_range=(9, 60), n1_range=(5, 2000))
    if mode == synth.MEM_SHORT:
        probs = [synth.with_mode(p, synth.MEM_SHORT, L=7 + 13 * i) for i, p in enumerate(probs)]
    if mode == synth.MEM_ADAPTIVE:
        probs = [synth.with_mode(p, synth.MEM_ADAPTIVE, a=2 + i % 9, rule=i % 2) for i, p in enumerate(probs)]
    out, b = run_batch(probs, chunk_terms=24, time_block=tb)
    assert b.geometry(0)["time_block"] == tb
    for p, got in zip(probs, out):
        assert rel_inf(got, oracle.run(p)) < 1e-5


@pytest.mark.parametrize("mode", [synth.MEM_FULL, synth.MEM_ADAPTIVE])
def test_blocked_batch_equals_single_blocked_runs_bitwise(mode):
    """Same blocks, chunks and summation order as one instance per launch."""
    probs = synth.config4(mode=mode, count=6, steps_range=(100, 300), side_range=(20, 50), n1_range=(40, 900))
    b = FRDBatch(probs, chunk_terms=32, time_block=8)
    res = []
    for _ in range(2):
        for i, p in enumerate(probs):
            b.set_state(i, p["u0"])
        b.run()
        res.append([b.state(i).cpu().numpy() for i in range(len(probs))])
        assert b.status() == 0
    for x, y in zip(*res):
        assert np.array_equal(x, y)
    for p, x in zip(probs, res[0]):
        s = FRD(p, chunk_terms=32, tile_threads=256, time_block=8)
        s.set_state(p["u0"])
        assert np.array_equal(s.run(p["K"]).cpu().numpy(), x)


@pytest.mark.parametrize("mode", [synth.MEM_FULL, synth.MEM_ADAPTIVE])
def test_config4_full_batch_large_instances_vs_scalar_recursions(mode):
    """The 64-instance workload with the shipped (tuned) geometry, large instances included: the
    three most expensive 1-D and three most expensive 2-D instances start from a superposition
    of Laplacian eigenmodes, so the oracle's scalar recursion of each mode (same weights,
    schedule and linear reaction) gives their exact result at full size; the three cheapest
    instances are compared with the oracle element by element."""
    from tests.helpers import laplacian_eigenvalue
    probs = [dict(p) for p in synth.config4(mode=mode)]
    cost = [p["nx"] * p["ny"] * p["K"] ** 2 for p in probs]
    order = list(np.argsort(cost))
    big1 = [i for i in order[::-1] if probs[i]["ndim"] == 1][:3]
    big2 = [i for i in order[::-1] if probs[i]["ndim"] == 2][:3]
    modes = {1: [(1, 1, 1.0), (3, 1, 0.5), (40, 1, 0.05)], 2: [(1, 1, 1.0), (3, 2, 0.5), (30, 17, 0.05)]}
    refs = {}
    for i in big1 + big2:
        p = probs[i]
        ms = modes[p["ndim"]]
        p["u0"] = sum(c * synth.eigenmode(p, qx, qy) for qx, qy, c in ms)
        refs[i] = sum(c * oracle.scalar_mode(p, laplacian_eigenvalue(p, qx, qy))[-1] * synth.eigenmode(p, qx, qy)
                      for qx, qy, c in ms)
    out, b = run_batch(probs)
    g0 = b.geometry(0)   # the tuned batch geometry: tensor-core far units, paired FP32 history
    assert g0["time_block"] == 32 and g0["far_tensor_cores"] == 1
    for i in big1 + big2:
        assert rel_inf(out[i], refs[i]) < 1e-5, (i, probs[i]["nx"], probs[i]["K"])
    for i in order[:3]:
        assert rel_inf(out[i], oracle.run(probs[i])) < 1e-5

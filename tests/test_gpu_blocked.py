"""Temporally blocked engine (time_block = 4 / 8 / 16; FP32, full, short and adaptive memory)
against the FP64 oracle and against properties that hold at full size, with block-long update units (the
default where the tiles are few) and with one update unit per step (step_updates); the blocked
reverse-time adjoint (time_block = 4 / 8) against the oracle's adjoint."""
import numpy as np
import pytest
import torch

import oracle
from paper_1004_5128_gb300 import FRD, synth
from tests.helpers import laplacian_eigenvalue, rel_inf

pytestmark = pytest.mark.gpu


def ragged(bc, mode, L=0, K=300):
    return synth.problem(2, 45, 37, 0.75, 0.7, synth.dt_for_courant(0.15, 0.7, 1.0, 0.75), 1.0, bc,
                         react=(0.01, -0.2, 0.3, -0.4), mem_mode=mode, mem_L=L, K=K,
                         u0=synth.SplitMix64(21).uniform(45 * 37, 0, 1))


@pytest.mark.parametrize("step_updates", [False, True])
@pytest.mark.parametrize("tb", [4, 8, 16])
@pytest.mark.parametrize("bc", [synth.BC_DIRICHLET0, synth.BC_NOFLUX])
@pytest.mark.parametrize("mode,L", [(synth.MEM_FULL, 0), (synth.MEM_SHORT, 50), (synth.MEM_SHORT, 7)])
def test_blocked_matches_oracle(tb, bc, mode, L, step_updates):
    """Several far chunks per block (chunk 16 rows), short windows longer and shorter than 2T."""
    p = ragged(bc, mode, L)
    s = FRD(p, time_block=tb, chunk_terms=16, step_updates=step_updates)
    assert s.geometry()["block_updates"] == (0 if step_updates else 1)
    s.set_state(p["u0"])
    assert rel_inf(s.run(p["K"]).cpu().double().numpy(), oracle.run(p)) < 1e-5


@pytest.mark.parametrize("tb,chunk", [(4, 16), (8, 24), (16, 40)])
@pytest.mark.parametrize("mode,L", [(synth.MEM_FULL, 0), (synth.MEM_SHORT, 37)])
def test_block_updates_equal_step_updates_bitwise(tb, chunk, mode, L):
    """With the same far chunks (chunk rows at least the block's rows over its chunk limit), the
    block-long units sum each step's terms in the per-step units' order: identical bits, in
    one launch and in launches that start inside blocks.  With blocks of 16 the per-step units
    take the previous block's rows from a near unit's partial sum, a different grouping: the
    two then agree to rounding, and each kind is split-invariant to the bit."""
    p = ragged(synth.BC_NOFLUX, mode, L)
    outs = []
    for su in (False, True):
        s = FRD(p, time_block=tb, chunk_terms=chunk, step_updates=su)
        s.set_state(p["u0"])
        outs.append(s.run(p["K"]).cpu().numpy())
        s.set_state(p["u0"])
        for n in (37, 5, 101, 1, 156):
            s.step(n)
        outs.append(s.run(0).cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[2], outs[3])
    if tb < 16:
        assert np.array_equal(outs[0], outs[2])
    else:
        assert rel_inf(outs[0], outs[2]) < 1e-6


def ragged_adaptive(a, rule, K=300, bc=synth.BC_NOFLUX):
    return synth.with_mode(ragged(bc, synth.MEM_FULL, K=K), synth.MEM_ADAPTIVE, a=a, rule=rule)


@pytest.mark.parametrize("step_updates", [False, True])
@pytest.mark.parametrize("tb", [4, 8, 16])
@pytest.mark.parametrize("rule", [synth.ADAPT_PAPER, synth.ADAPT_PARTITION])
@pytest.mark.parametrize("a", [2, 3, 10])
def test_blocked_adaptive_matches_oracle(tb, rule, a, step_updates):
    """Far rows carry the settled weights g(m) (psi on the base interval, d psi at the medians,
    0 between); each step's tail rows (a = 2: tails longer than a block) and near rows take
    that step's weights in the update units."""
    p = ragged_adaptive(a, rule)
    s = FRD(p, time_block=tb, chunk_terms=16, step_updates=step_updates)
    assert s.geometry()["time_block"] == tb
    s.set_state(p["u0"])
    assert rel_inf(s.run(p["K"]).cpu().double().numpy(), oracle.run(p)) < 1e-5


@pytest.mark.parametrize("tb,chunk", [(4, 16), (8, 24), (16, 40)])
@pytest.mark.parametrize("a", [2, 10])
def test_blocked_adaptive_block_updates_equal_step_updates_bitwise(tb, chunk, a):
    """Block-long and per-step update units sum the same terms in the same order, in one
    launch and in launches that start inside blocks (blocks of 16: to rounding, as above)."""
    p = ragged_adaptive(a, synth.ADAPT_PAPER)
    outs = []
    for su in (False, True):
        s = FRD(p, time_block=tb, chunk_terms=chunk, step_updates=su)
        s.set_state(p["u0"])
        outs.append(s.run(p["K"]).cpu().numpy())
        s.set_state(p["u0"])
        for n in (37, 5, 101, 1, 156):
            s.step(n)
        outs.append(s.run(0).cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[2], outs[3])
    if tb < 16:
        assert np.array_equal(outs[0], outs[2])
    else:
        assert rel_inf(outs[0], outs[2]) < 1e-6


@pytest.mark.parametrize("step_updates", [False, True])
@pytest.mark.parametrize("tb", [8, 16])
@pytest.mark.parametrize("mode", [synth.MEM_FULL, synth.MEM_ADAPTIVE])
def test_blocked_3d_matches_oracle(tb, mode, step_updates):
    """7-point stencil on a 13x11x9 grid (ragged last tile), mirror boundaries."""
    n = 13 * 11 * 9
    p = synth.problem(3, 13, 11, 0.65, 0.9, synth.dt_for_courant(0.05, 0.9, 1.0, 0.65), 1.0,
                      synth.BC_NOFLUX, react=(0.02, -0.3, 0.1, -0.2), K=220, nz=9,
                      u0=synth.SplitMix64(33).uniform(n, 0, 1))
    if mode == synth.MEM_ADAPTIVE:
        p = synth.with_mode(p, synth.MEM_ADAPTIVE, a=4)
    s = FRD(p, time_block=tb, chunk_terms=16, tile_threads=128, step_updates=step_updates)
    s.set_state(p["u0"])
    assert rel_inf(s.run(p["K"]).cpu().double().numpy(), oracle.run(p)) < 1e-5


def test_blocked_1d_many_tiles():
    p = synth.problem(1, 3001, 1, 0.55, 1.0, synth.dt_for_courant(0.2, 1.0, 1.0, 0.55), 1.0,
                      synth.BC_DIRICHLET0, react=(0, -0.05, 0, 0), K=400,
                      u0=synth.SplitMix64(8).uniform(3001, -1, 1))
    s = FRD(p, time_block=8, tile_threads=64, chunk_terms=24)
    s.set_state(p["u0"])
    assert rel_inf(s.run(p["K"]).cpu().double().numpy(), oracle.run(p)) < 1e-5


@pytest.mark.parametrize("step_updates", [False, True])
def test_blocked_launch_split_is_bitwise_invariant(step_updates):
    """Blocks are aligned to absolute steps, so any split into launches gives the same bits."""
    p = ragged(synth.BC_NOFLUX, synth.MEM_FULL, K=400)
    a = FRD(p, time_block=8, chunk_terms=32, step_updates=step_updates)
    a.set_state(p["u0"])
    one = a.run(400).cpu().numpy()
    b = FRD(p, time_block=8, chunk_terms=32, step_updates=step_updates)
    b.set_state(p["u0"])
    for n in (57, 3, 100, 1, 139, 100):
        b.step(n)
    assert np.array_equal(one, b.run(0).cpu().numpy())


@pytest.mark.parametrize("step_updates", [False, True])
@pytest.mark.parametrize("mode", [synth.MEM_FULL, synth.MEM_SHORT, synth.MEM_ADAPTIVE])
def test_blocked_config2_full_size(mode, step_updates):
    """256^2, 5000 steps: eigenmode superposition against the oracle's scalar recursions, and
    the Gaussian input's mass balance."""
    p = synth.config2(mode)
    modes = [(0, 0, 1.0), (1, 0, 0.5), (3, 2, 0.25), (17, 5, 0.125), (64, 64, 0.0625), (200, 31, 0.03)]
    q = dict(p)
    q["u0"] = sum(c * synth.eigenmode(p, qx, qy) for qx, qy, c in modes)
    ref = sum(c * oracle.scalar_mode(p, laplacian_eigenvalue(p, qx, qy))[-1] * synth.eigenmode(p, qx, qy)
              for qx, qy, c in modes)
    s = FRD(q, time_block=8, tile_threads=512, step_updates=step_updates)
    assert s.geometry()["block_updates"] == (0 if step_updates else 1)
    s.set_state(q["u0"])
    assert rel_inf(s.run(q["K"]).cpu().double().numpy(), ref) < 1e-5
    s = FRD(p, time_block=8, tile_threads=512, step_updates=step_updates)
    s.set_state(p["u0"])
    M0 = p["u0"].sum()
    assert abs(s.run(p["K"]).cpu().double().numpy().sum() - M0 * (1 - 0.1 * p["dt"]) ** p["K"]) / M0 < 2e-5


def blocked_adjoint(p, tgt, tb, ckpt, **kw):
    s = FRD(p, keep_tape=True, ckpt_every=ckpt, time_block=tb, **kw)
    assert s.geometry()["time_block"] == tb
    s.set_state(p["u0"])
    uK = s.run(p["K"])
    r = s.adjoint(uK - torch.as_tensor(tgt, device=uK.device, dtype=uK.dtype))
    r["du0"] = r["du0"].cpu().double().numpy()
    return r


def compare_grads(r, ref, tol):
    assert rel_inf(r["du0"], ref["du0"]) < tol
    for key in ("dgamma", "dalpha"):
        assert abs(r[key] - ref[key]) <= tol * abs(ref[key]), (key, r[key], ref[key])
    assert np.max(np.abs(np.array(r["dreact"]) - ref["dreact"])) <= tol * np.max(np.abs(ref["dreact"]))


@pytest.mark.parametrize("step_updates", [False, True])
@pytest.mark.parametrize("tb", [4, 8])
@pytest.mark.parametrize("bc", [synth.BC_DIRICHLET0, synth.BC_NOFLUX])
def test_blocked_adjoint_matches_oracle(tb, bc, step_updates):
    """Checkpoint segments of 50 steps (not a multiple of the block: recompute and adjoint
    launches start inside a block) and a ragged last segment; several far chunks per block."""
    p = ragged(bc, synth.MEM_FULL, K=230)
    tgt = synth.SplitMix64(3).uniform(p["nx"] * p["ny"], 0, 0.8)
    compare_grads(blocked_adjoint(p, tgt, tb, ckpt=50, chunk_terms=16, step_updates=step_updates),
                  oracle.adjoint(p, tgt), 1e-5)


def test_blocked_adjoint_config5_reduced():
    """Config-5 physics (128^2, gamma=0.7, alpha=0.8, f=-0.1u, dt=0.005) at 600 steps, the
    config's checkpoint spacing of 200 steps."""
    p = synth.config5(K=600)
    tgt = oracle.run(synth.config5(K=600, target=True))
    compare_grads(blocked_adjoint(p, tgt, 8, ckpt=200), oracle.adjoint(p, tgt), 1e-5)


def test_blocked_adjoint_rejects_blocks_of_16():
    from paper_1004_5128_gb300 import _lib as L
    with pytest.raises(L.FdError) as e:
        FRD(ragged(synth.BC_NOFLUX, synth.MEM_FULL), keep_tape=True, time_block=16)
    assert e.value.code == L.FD_ERR_UNSUPPORTED


@pytest.mark.parametrize("step_updates", [False, True])
def test_blocked_adjoint_repeats_bitwise_at_config5_size(step_updates):
    """128^2, 4000 steps, checkpoints every 200 with the shipped adjoint geometry (blocks of 8,
    128-thread tiles, 16-row stages, 128-row chunks): 40 launches per adjoint, each with
    boundary units that the kernel passes over.  Five repetitions must all finish and agree
    to the bit (fixed summation order)."""
    p = synth.config5(K=4000)
    geo = dict(time_block=8, tile_threads=128, stage_rows=16, chunk_terms=128, step_updates=step_updates)
    runs = []
    for _ in range(5):
        s = FRD(p, keep_tape=True, ckpt_every=200, timeout_ms=5000, **geo)
        s.set_state(p["u0"])
        uK = s.run(p["K"])
        r = s.adjoint(uK * 0.01)
        runs.append((r["dgamma"], r["dalpha"], r["du0"].cpu().numpy()))
        s.close()
    for dg, da, du in runs[1:]:
        assert dg == runs[0][0] and da == runs[0][1] and np.array_equal(du, runs[0][2])


def test_blocked_stall_injection_reports_its_site():
    """A wait nothing will satisfy ends the blocked launch with FD_ERR_TIMEOUT, the error record
    names a wait of the blocked kernel, and the next handle runs normally."""
    from paper_1004_5128_gb300 import _lib as L
    p = ragged(synth.BC_NOFLUX, synth.MEM_FULL, K=40)
    s = FRD(p, time_block=8, inject_stall=True, timeout_ms=200)
    s.set_state(p["u0"])
    with pytest.raises(L.FdError) as e:
        s.run(p["K"])
    assert e.value.code == L.FD_ERR_TIMEOUT
    # the first wait to give up is the injected one or one that depends on it
    info = s.error_info()
    assert info["words"][0] in (1, 3, 4, 5, 9, 10) and info["site"] != "none"
    s.close()
    t = FRD(p, time_block=8)
    t.set_state(p["u0"])
    assert rel_inf(t.run(p["K"]).cpu().double().numpy(), oracle.run(p)) < 1e-5


@pytest.mark.parametrize("step_updates", [False, True])
@pytest.mark.parametrize("tb,L", [(4, 9), (8, 37)])
def test_blocked_short_memory_adjoint_matches_oracle(tb, L, step_updates):
    """Blocked adjoint of short memory: the far window and the head both stop at lag L."""
    p = ragged(synth.BC_DIRICHLET0, synth.MEM_SHORT, L=L, K=230)
    tgt = synth.SplitMix64(4).uniform(p["nx"] * p["ny"], 0, 0.8)
    compare_grads(blocked_adjoint(p, tgt, tb, ckpt=50, chunk_terms=16, step_updates=step_updates),
                  oracle.adjoint(p, tgt), 1e-5)

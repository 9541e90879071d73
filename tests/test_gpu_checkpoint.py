"""fd_save / fd_load: a run checkpointed at step k and resumed in a fresh handle gives the bits of
an uninterrupted run, for the per-step kernel and the blocked kernels (CUDA-core and tensor-core
far units, paired FP32 and 16-bit history), in every memory mode; a checkpoint from another problem
is refused."""
import numpy as np
import pytest

from paper_1004_5128_gb300 import FRD, _lib as L, synth

pytestmark = pytest.mark.gpu


def ragged(mode, L_=0, a=0, K=300):
    return synth.problem(2, 45, 37, 0.75, 0.7, synth.dt_for_courant(0.15, 0.7, 1.0, 0.75), 1.0, synth.BC_NOFLUX,
                         react=(0.01, -0.2, 0.3, -0.4), mem_mode=mode, mem_L=L_, mem_a=a, K=K,
                         u0=synth.SplitMix64(21).uniform(45 * 37, 0, 1))


CASES = [("per-step", {}), ("blocked16", dict(time_block=16)), ("tc-f32-64", dict(time_block=64)),
         ("tc-bf16-32", dict(time_block=32, hist="bf16")), ("tc-f16-64", dict(time_block=64, hist="f16"))]
MODES = [("full", synth.MEM_FULL, 0, 0), ("short40", synth.MEM_SHORT, 40, 0), ("adapt3", synth.MEM_ADAPTIVE, 0, 3)]


@pytest.mark.parametrize("name,mode,L_,a", MODES, ids=[m[0] for m in MODES])
@pytest.mark.parametrize("kind,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("on_device", [False, True])
def test_checkpoint_resume_is_bitwise(kind, kw, name, mode, L_, a, on_device):
    p = ragged(mode, L_, a)
    ref = FRD(p, **kw)
    ref.set_state(p["u0"])
    want = ref.run(p["K"]).cpu().numpy()
    s = FRD(p, **kw)
    s.set_state(p["u0"])
    s.step(137)  # inside a block of every block length
    ck = s.save(device=on_device)
    s.close()
    r = FRD(p, **kw)
    r.load(ck)
    assert r.k == 137
    got = r.run(p["K"] - 137).cpu().numpy()
    assert r.status() == 0
    assert np.array_equal(got, want)


def test_checkpoint_of_another_problem_is_refused():
    p = ragged(synth.MEM_FULL)
    s = FRD(p, time_block=64)
    s.set_state(p["u0"])
    s.step(70)
    ck = s.save()
    q = dict(p, gamma=0.76)
    t = FRD(q, time_block=64)
    with pytest.raises(L.FdError) as e:
        t.load(ck)
    assert e.value.code == L.FD_ERR_INVALID_ARG
    with pytest.raises(L.FdError):
        FRD(p, time_block=64).load(ck[: ck.numel() // 2])  # short buffer

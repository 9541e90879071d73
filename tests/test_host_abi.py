"""CPU tests of the C ABI's host side: symbols, weights, schedules, validation, workspace sizing.
No kernel runs here (no GPU in this environment)."""
import ctypes
import re
import os

import numpy as np
import pytest

import oracle
from paper_1004_5128_gb300 import _lib as L
from paper_1004_5128_gb300 import build as B
from paper_1004_5128_gb300 import make_problem, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    L.lib()


def test_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "fd.h")).read()
    declared = set(re.findall(r"^\s*(?:int|int64_t|const char \*)\s*\**\s*(fd_\w+)\s*\(", hdr, re.M))
    assert declared == set(L.EXPORTS)
    lib = ctypes.CDLL(L.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name


def test_weights_match_oracle():
    for g in (0.3, 0.5, 0.8, 1.0, 1.5):
        a, da = L.fd_weights(g, 20001, with_derivative=True)
        b, db = oracle.weights(g, 20001, with_derivative=True)
        assert np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)) < 1e-13
        m = np.abs(db) > 0
        assert np.max(np.abs(da[m] - db[m]) / np.abs(db[m])) < 1e-12


@pytest.mark.parametrize("mode,L_,a,rule", [(0, 0, 0, 0), (1, 1, 0, 0), (1, 7, 0, 0), (1, 500, 0, 0),
                                            (2, 0, 2, 0), (2, 0, 3, 0), (2, 0, 10, 0), (2, 0, 50, 0),
                                            (2, 0, 2, 1), (2, 0, 3, 1), (2, 0, 10, 1)])
def test_schedule_matches_oracle(mode, L_, a, rule):
    """The engine's integer schedule (prefix of medians + tail range) equals the oracle's
    literal enumeration at every step, bit for bit."""
    p = synth.with_mode(synth.config2(K=10), mode, L=L_, a=a, rule=rule)
    fp = make_problem(p, max_steps=10)
    for k in list(range(0, 200)) + [999, 4999, 7777, 10008, 10009, 12345]:
        lag, mult = L.fd_schedule(fp, k)
        olag, omult = oracle.schedule(mode, L_, a, rule, k)
        assert np.array_equal(lag, olag) and np.array_equal(mult, omult), k


def test_validation_codes():
    p = synth.config2(K=10)
    fp = make_problem(p, max_steps=10)
    fp.gamma = 2.5
    with pytest.raises(L.FdError) as e:
        L.fd_workspace_bytes(fp)
    assert e.value.code == L.FD_ERR_INVALID_ARG
    fp = make_problem(p, max_steps=10)
    fp.dt = p["dt"] * 100  # S far above 2^g / 8
    with pytest.raises(L.FdError) as e:
        L.fd_workspace_bytes(fp)
    assert e.value.code == L.FD_ERR_UNSTABLE
    fp.flags |= L.FD_FLAG_ALLOW_UNSTABLE
    assert L.fd_workspace_bytes(fp) > 0
    # adjoint: full, short (the short run then keeps every row for the recompute) and adaptive
    # memory (settled weights plus the tail terms' table)
    q = make_problem(synth.with_mode(p, synth.MEM_SHORT, L=5), max_steps=10, keep_tape=True)
    assert L.fd_workspace_bytes(q) > 0
    q = make_problem(synth.with_mode(p, synth.MEM_ADAPTIVE, a=3), max_steps=10, keep_tape=True)
    assert L.fd_workspace_bytes(q) > L.fd_workspace_bytes(make_problem(synth.with_mode(p, synth.MEM_ADAPTIVE, a=3),
                                                                       max_steps=10))
    # bf16 history with an f64 state is not a built combination
    q = make_problem(p, max_steps=10, state="f64", hist="bf16")
    with pytest.raises(L.FdError) as e:
        L.fd_workspace_bytes(q)
    assert e.value.code == L.FD_ERR_UNSUPPORTED
    for bad in (dict(mem_mode=synth.MEM_SHORT, mem_L=0), dict(mem_mode=synth.MEM_ADAPTIVE, mem_a=1)):
        q = dict(p)
        q.update(bad)
        with pytest.raises(L.FdError):
            L.fd_workspace_bytes(make_problem(q, max_steps=10))


def test_init_rejects_small_or_misaligned_workspace():
    p = make_problem(synth.config1(K=10), state="f64")
    need = L.fd_workspace_bytes(p)
    h = ctypes.c_void_p(0)
    assert L.lib().fd_init(ctypes.byref(p), ctypes.c_void_p(1 << 20), need - 1, None, ctypes.byref(h)) \
        == L.FD_ERR_WORKSPACE
    assert L.lib().fd_init(ctypes.byref(p), ctypes.c_void_p((1 << 20) + 16), need, None,
                           ctypes.byref(h)) == L.FD_ERR_WORKSPACE
    assert L.lib().fd_init(ctypes.byref(p), None, need, None, ctypes.byref(h)) == L.FD_ERR_WORKSPACE


def test_workspace_scales_with_history():
    full = L.fd_workspace_bytes(make_problem(synth.config2(K=5000)))
    short = L.fd_workspace_bytes(make_problem(synth.config2(synth.MEM_SHORT, K=5000)))
    bf = L.fd_workspace_bytes(make_problem(synth.config2(K=5000), hist="bf16"))
    assert 1.30e9 < full < 1.40e9          # 5000 rows x 256 KiB of FP32 delta history
    assert short < 0.2e9                   # ring of L+1 = 501 rows (131 MB) plus partial rows
    assert 0.6e9 < bf < 0.75e9            # BF16 rows plus FP32 partial rows and head ring
    tape = L.fd_workspace_bytes(make_problem(synth.config5(K=4000), keep_tape=True))
    assert tape > 2 * 4000 * 128 * 128 * 4  # forward + adjoint histories


def test_batch_workspace():
    probs = [make_problem(p) for p in synth.config4(count=8, steps_range=(100, 300),
                                                    side_range=(16, 40), n1_range=(16, 300))]
    assert L.fd_batch_workspace_bytes(probs) > 0


def test_strerror():
    assert "stability" in L.fd_strerror(L.FD_ERR_UNSTABLE)
    assert L.fd_strerror(0) == "ok"


def test_time_block_validation():
    p = synth.config2(K=100)
    assert L.fd_workspace_bytes(make_problem(p, time_block=8)) > 0
    # the blocked adjoint keeps two accumulator sets: blocks of 4 and 8 steps only
    taped = L.fd_workspace_bytes(make_problem(p, time_block=8, keep_tape=True))
    assert taped > L.fd_workspace_bytes(make_problem(p, keep_tape=True)) > 0
    # BF16 / FP16 history blocks forward; blocks of 16, 32 or 64 on the tensor cores; FP32 history
    # with blocks of 32 or 64 on the tensor cores (split into FP16 hi and lo parts)
    for ok in (dict(time_block=8, hist="bf16"), dict(time_block=16, hist="f16"),
               dict(time_block=32, hist="bf16"), dict(time_block=64, hist="f16"),
               dict(time_block=16, hist="bf16", fma_far=True),
               dict(time_block=32), dict(time_block=64), dict(time_block=32, tile_threads=256)):
        assert L.fd_workspace_bytes(make_problem(p, **ok)) > 0
    for bad, code in ((dict(time_block=5), L.FD_ERR_INVALID_ARG),
                      (dict(time_block=8, hist="bf16", keep_tape=True), L.FD_ERR_UNSUPPORTED),
                      (dict(time_block=32, fma_far=True), L.FD_ERR_UNSUPPORTED),
                      (dict(time_block=32, keep_tape=True), L.FD_ERR_UNSUPPORTED),
                      (dict(time_block=64, keep_tape=True), L.FD_ERR_UNSUPPORTED),
                      (dict(time_block=32, hist="bf16", fma_far=True), L.FD_ERR_UNSUPPORTED),
                      (dict(time_block=32, hist="bf16", tile_threads=192), L.FD_ERR_INVALID_ARG),
                      (dict(time_block=16, hist="bf16", stage_rows=32), L.FD_ERR_INVALID_ARG),
                      (dict(time_block=8, kahan=True), L.FD_ERR_UNSUPPORTED),
                      (dict(time_block=16, keep_tape=True), L.FD_ERR_UNSUPPORTED)):
        with pytest.raises(L.FdError) as e:
            L.fd_workspace_bytes(make_problem(p, **bad))
        assert e.value.code == code
    # adaptive memory blocks forward and adjoint (blocks of 4 or 8)
    ad = synth.with_mode(p, synth.MEM_ADAPTIVE, a=10)
    assert L.fd_workspace_bytes(make_problem(ad, time_block=8)) > L.fd_workspace_bytes(make_problem(ad)) > 0
    assert L.fd_workspace_bytes(make_problem(ad, time_block=8, keep_tape=True)) > \
        L.fd_workspace_bytes(make_problem(ad, time_block=8))


def test_blocked_batch_validation():
    """A batch runs one kernel: every instance takes the same time_block."""
    probs = synth.config4(count=4, steps_range=(50, 90), side_range=(9, 20), n1_range=(5, 50))
    same = [make_problem(p, time_block=8) for p in probs]
    assert L.fd_batch_workspace_bytes(same) > L.fd_batch_workspace_bytes([make_problem(p) for p in probs])
    mixed = [make_problem(p, time_block=8 if i else 4) for i, p in enumerate(probs)]
    with pytest.raises(L.FdError) as e:
        L.fd_batch_workspace_bytes(mixed)
    assert e.value.code == L.FD_ERR_INVALID_ARG
    with pytest.raises(L.FdError) as e:
        L.fd_batch_workspace_bytes([make_problem(p, time_block=8, keep_tape=True) for p in probs])
    assert e.value.code == L.FD_ERR_UNSUPPORTED


def test_bench_traffic_entries_follow_the_kernel_code(tmp_path):
    """profiles/traffic.json entries are keyed to the kernel code with comments and blank space
    removed: a comment edit keeps an entry, a code edit drops it."""
    import importlib.util
    import json
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    src = os.path.join(root, "paper_1004_5128_gb300", "csrc", "fd_engine_tb.cuh")
    text = open(src).read()
    h = bench.code_hash(src)
    (tmp_path / "a.cuh").write_text(text.replace("const int lane = tid & 31", "/* x */ // y\n    const int lane = tid & 31", 1))
    (tmp_path / "b.cuh").write_text(text.replace("const int lane = tid & 31", "const int lane = tid % 32", 1))
    assert bench.code_hash(str(tmp_path / "a.cuh")) == h
    assert bench.code_hash(str(tmp_path / "b.cuh")) != h
    # an entry is reported for its own key and geometry only
    e = json.load(open(os.path.join(root, "profiles", "traffic.json")))["entries"][0]
    other = dict(e["geometry"], tile_threads=e["geometry"]["tile_threads"] // 2)
    assert bench.measured_traffic(e["key"], other) is None
    assert bench.measured_traffic("no such run", dict(e["geometry"])) is None


def test_closed_loop_validation():
    """Closed-loop adaptive memory: adaptive schedules on the per-step kernel with history in state
    precision, forward only, single handles; a threshold tau >= 0 (+inf allowed)."""
    import math
    ad = synth.with_mode(synth.config2(K=100), synth.MEM_ADAPTIVE, a=10)
    open_bytes = L.fd_workspace_bytes(make_problem(ad))
    for tau in (0.0, 0.1, math.inf):
        for state in ("f32", "f64"):
            assert L.fd_workspace_bytes(make_problem(ad, state=state, closed_tau=tau)) > \
                L.fd_workspace_bytes(make_problem(ad, state=state))
    assert L.fd_workspace_bytes(make_problem(ad, closed_tau=0.1)) > open_bytes
    for kw, code in ((dict(closed_tau=-1.0), L.FD_ERR_INVALID_ARG),
                     (dict(closed_tau=math.nan), L.FD_ERR_INVALID_ARG),
                     (dict(closed_tau=0.1, time_block=8), L.FD_ERR_UNSUPPORTED),
                     (dict(closed_tau=0.1, hist="bf16"), L.FD_ERR_UNSUPPORTED),
                     (dict(closed_tau=0.1, keep_tape=True), L.FD_ERR_UNSUPPORTED)):
        with pytest.raises(L.FdError) as e:
            L.fd_workspace_bytes(make_problem(ad, **kw))
        assert e.value.code == code
    with pytest.raises(L.FdError) as e:
        L.fd_workspace_bytes(make_problem(synth.config2(K=100), closed_tau=0.1))  # full memory
    assert e.value.code == L.FD_ERR_UNSUPPORTED
    with pytest.raises(L.FdError) as e:
        L.fd_batch_workspace_bytes([make_problem(ad, closed_tau=0.1)] * 2)
    assert e.value.code == L.FD_ERR_UNSUPPORTED
    # the tuned table's geometry (blocks of 64 for this schedule) is not applied to a closed loop
    from paper_1004_5128_gb300.frd import tuned_geometry
    assert tuned_geometry(synth.config2(synth.MEM_ADAPTIVE), {"closed_tau": 0.1}) == {}

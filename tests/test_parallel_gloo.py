"""Multi-rank layer on CPU: world_size-2 gloo process groups (no GPU).

The instance split must cover every instance once with balanced history traffic; each rank
computes its shard (here with the FP64 oracle standing in for the GPU engine) and the gathered
results must equal the single-process run bitwise; the timing reduction is a max over ranks.
Within one instance, slabs of grid rows with a one-row u halo exchanged per step (explicit
send/recv) must reproduce the one-rank run bitwise."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1004_5128_gb300 import parallel, synth


def small_batch():
    return synth.config4(count=10, steps_range=(20, 90), side_range=(5, 14), n1_range=(5, 60))


def test_shard_covers_and_balances():
    probs = synth.config4()  # the 64-instance workload
    for ws in (1, 2, 3, 4, 8):
        parts = parallel.shard(probs, ws)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(probs)))
        loads = [sum(parallel.instance_cost(probs[i]) for i in p) for p in parts]
        biggest = max(parallel.instance_cost(p) for p in probs)
        assert max(loads) - min(loads) <= biggest + 1e-9


def test_schedule_terms_exact_for_full_and_short():
    import oracle
    p = synth.config2(K=300, n=8)
    assert parallel.schedule_terms(p) == sum(len(oracle.schedule(0, 0, 0, 0, k)[0]) - 1 for k in range(300))
    q = synth.with_mode(p, synth.MEM_SHORT, L=37)
    assert parallel.schedule_terms(q) == sum(len(oracle.schedule(1, 37, 0, 0, k)[0]) - 1 for k in range(300))
    r = synth.with_mode(p, synth.MEM_ADAPTIVE, a=10)
    exact = sum(len(oracle.schedule(2, 0, 10, 0, k)[0]) - 1 for k in range(300))
    assert abs(parallel.schedule_terms(r, samples=300) - exact) <= 0.02 * exact


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out_dir):
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        probs = small_batch()
        mine = parallel.shard(probs, ws)[rank]
        res = {i: oracle.run(probs[i]) for i in mine}
        gathered = [None] * ws
        dist.all_gather_object(gathered, res)
        t = parallel.max_over_ranks(float(rank + 1) * 0.5)
        if rank == 0:
            merged = {}
            for g in gathered:
                merged.update(g)
            np.savez(os.path.join(out_dir, "out.npz"), t=t,
                     **{f"u{i}": merged[i] for i in sorted(merged)})
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_single_process(tmp_path):
    import oracle
    ws = 2
    mp.spawn(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    d = np.load(tmp_path / "out.npz")
    assert float(d["t"]) == 1.0  # max over ranks of 0.5 * (rank + 1)
    probs = small_batch()
    for i, p in enumerate(probs):
        assert np.array_equal(d[f"u{i}"], oracle.run(p))


# ---- within one instance: slabs of grid rows with a one-row u halo per step -----------------
# The memory sum is local to each point: a rank keeps only its own rows' history.  The stencil
# is the only coupling, so each step exchanges one row of u^k with each neighbouring slab.  The
# ranks below step the scheme (eq. frac_final) in numpy with the oracle's weights and schedule;
# the gathered field must equal the one-rank run bitwise and the oracle to rounding.

def slab_problem(mode):
    p = synth.problem(2, 13, 11, 0.7, 0.8, synth.dt_for_courant(0.15, 0.8, 1.0, 0.7), 1.0,
                      synth.BC_NOFLUX, react=(0.01, -0.2, 0.3, -0.4), K=60,
                      u0=synth.SplitMix64(41).uniform(13 * 11, 0, 1))
    return synth.with_mode(p, mode, a=3) if mode == synth.MEM_ADAPTIVE else p


def slab_rows(ny, ws, rank):
    base, extra = divmod(ny, ws)
    y0 = rank * base + min(rank, extra)
    return y0, y0 + base + (1 if rank < extra else 0)


def run_slab(p, y0, y1, exchange):
    """u^K on rows y0..y1-1; exchange(first_row, last_row) returns the ghost rows below and above
    (None at the grid's edge)."""
    import oracle
    nx, ny, K = p["nx"], p["ny"], p["K"]
    psi = np.asarray(oracle.weights(p["gamma"], K + 1))
    S = p["alpha"] * p["dt"] ** p["gamma"] / p["dx"] ** 2
    noflux = p["bc"] == synth.BC_NOFLUX
    q = p["react"]
    u = np.asarray(p["u0"], dtype=np.float64).reshape(ny, nx)[y0:y1].copy()
    zero = np.zeros(nx)
    hist = []
    for k in range(K):
        below, above = exchange(u[0].copy(), u[-1].copy())
        below = below if below is not None else (u[0] if noflux else zero)
        above = above if above is not None else (u[-1] if noflux else zero)
        ext = np.vstack([below, u, above])
        edge_l = u[:, :1] if noflux else np.zeros((u.shape[0], 1))
        edge_r = u[:, -1:] if noflux else np.zeros((u.shape[0], 1))
        left = np.hstack([edge_l, u[:, :-1]])
        right = np.hstack([u[:, 1:], edge_r])
        delta = ((ext[:-2] + ext[2:]) + (left + right)) - 4.0 * u
        hist.append(delta)
        lags, mult = oracle.schedule(p["mem_mode"], p["mem_L"], p["mem_a"], p.get("adaptive_rule", 0), k)
        s = np.zeros_like(u)
        for m, c in sorted(zip(lags.tolist(), mult.tolist())):
            s = s + (c * psi[m]) * hist[k - m]
        f = q[0] + q[1] * u + q[2] * u * u + q[3] * u * u * u
        u = u + p["dt"] * f + S * s
    return u


def _slab_worker(rank, ws, port, out_dir, mode):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        p = slab_problem(mode)
        y0, y1 = slab_rows(p["ny"], ws, rank)

        def exchange(first, last):
            reqs, below, above = [], None, None
            if rank > 0:
                below = torch.empty(p["nx"], dtype=torch.float64)
                reqs += [dist.isend(torch.from_numpy(first), rank - 1), dist.irecv(below, rank - 1)]
            if rank < ws - 1:
                above = torch.empty(p["nx"], dtype=torch.float64)
                reqs += [dist.isend(torch.from_numpy(last), rank + 1), dist.irecv(above, rank + 1)]
            for r in reqs:
                r.wait()
            return (None if below is None else below.numpy()), (None if above is None else above.numpy())

        u = run_slab(p, y0, y1, exchange)
        gathered = [None] * ws
        dist.all_gather_object(gathered, (y0, u))
        if rank == 0:
            full = np.zeros((p["ny"], p["nx"]))
            for a, part in gathered:
                full[a:a + part.shape[0]] = part
            np.save(os.path.join(out_dir, "slabs.npy"), full)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode", [synth.MEM_FULL, synth.MEM_ADAPTIVE])
def test_two_gloo_slab_ranks_reproduce_one_rank_bitwise(tmp_path, mode):
    import oracle
    ws = 2
    mp.spawn(_slab_worker, args=(ws, _free_port(), str(tmp_path), mode), nprocs=ws, join=True)
    got = np.load(tmp_path / "slabs.npy")
    p = slab_problem(mode)
    one = run_slab(p, 0, p["ny"], lambda first, last: (None, None))
    assert np.array_equal(got, one)
    ref = oracle.run(p).reshape(p["ny"], p["nx"])
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))

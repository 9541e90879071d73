"""Multi-rank layer on CPU: world_size-2 gloo process groups (no GPU).

The instance split must cover every instance once with balanced history traffic; each rank
computes its shard (here with the FP64 oracle standing in for the GPU engine) and the gathered
results must equal the single-process run bitwise; the timing reduction is a max over ranks."""
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

"""bench.py's split of the workload over ranks: the config-4 batch is sharded by parallel.shard
(every instance on exactly one rank), single-instance workloads run as replicas."""
import bench
from paper_1004_5128_gb300 import parallel, synth


def test_batch_instances_are_sharded_like_parallel_shard():
    runs = synth.workload_runs("c4")
    for ws in (2, 3, 8):
        parts = [bench.shard_runs(runs, ws, r) for r in range(ws)]
        assert all(sharded for _, sharded in parts)
        for j, (name, probs, _) in enumerate(runs):
            split = parallel.shard(probs, ws)
            for r in range(ws):
                got = parts[r][0][j][1]
                assert [id(p) for p in got] == [id(probs[i]) for i in split[r]]
            assert sorted(i for s in split for i in s) == list(range(len(probs)))


def test_single_instances_are_replicas():
    runs = synth.workload_runs("c3", K=10)
    for ws in (1, 4):
        out, sharded = bench.shard_runs(runs, ws, ws - 1)
        assert not sharded and [r[0] for r in out] == ["bf16", "f16", "f32"]
        assert all(a[1] is b[1] for a, b in zip(out, runs))


def test_closed_loop_workload():
    """The closed-loop workload runs config 2's adaptive schedule three ways on the per-step
    kernel: open loop (time_block 0 keeps the tuned blocked geometry away) and closed loop at two
    thresholds."""
    runs = synth.workload_runs("c2cl")
    assert [r[0] for r in runs] == ["open", "tau0.1", "tau0.01"]
    for name, p, kw in runs:
        assert p["mem_mode"] == synth.MEM_ADAPTIVE and p["mem_a"] == 10 and p["nx"] == 256 and p["K"] == 5000
    assert runs[0][2] == {"time_block": 0}
    assert [r[2].get("closed_tau") for r in runs[1:]] == [0.1, 0.01]

"""Replica sharding across processes (CPU, gloo, world size 2).

Two ranks each run their share of the replicas, offsetting the Philox seed by
their first replica; rank 0 gathers the final positions and they must equal a
single-process run of all replicas bit for bit. The trajectories are computed
by the FP64 oracle (no GPU here); the CUDA library's own seed-offset
reproducibility is checked on the GPU by test_replica_sharding_is_exact.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def run_replicas(first, count, seed, steps):
    import oracle
    from paper_1003_1148_gb300 import synth
    w = synth.compact_chain(20, 5)
    m = oracle.Model(w, np.zeros(20, np.int32), np.zeros(20, np.int32))
    out = []
    for r in range(first, first + count):
        x, _, _, _ = m.run(w, steps, seed=seed + r)
        out.append(x)
    return np.array(out)


def worker(rank, world, port, total, result_path):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    from paper_1003_1148_gb300 import dist
    w, r, _ = dist.rank_env()
    group = dist.init(w)
    first, count = dist.replica_range(r, w, total=total)
    x = run_replicas(first, count, seed=1000, steps=25)
    t = dist.max_over_ranks(group, float(r + 1))
    allx = dist.gather_rows(group, x, w)
    dist.barrier(group)
    if r == 0:
        np.save(result_path, allx)
        with open(result_path + ".max", "w") as f:
            f.write(str(t))
    group.destroy_process_group()


def test_replica_range_partitions():
    from paper_1003_1148_gb300 import dist
    for total in (1, 5, 8192, 8193):
        for world in (1, 2, 3, 8):
            spans = [dist.replica_range(r, world, total=total) for r in range(world)]
            assert spans[0][0] == 0
            assert sum(c for _, c in spans) == total
            for (a, ca), (b, _) in zip(spans, spans[1:]):
                assert a + ca == b
    assert dist.replica_range(3, 4, per_rank=8192) == (3 * 8192, 8192)


def test_two_rank_sharding_equals_single_run(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    total = 5
    path = str(tmp_path / "gathered.npy")
    tmp.spawn(worker, args=(2, free_port(), total, path), nprocs=2, join=True)
    gathered = np.load(path)
    single = run_replicas(0, total, seed=1000, steps=25)
    assert gathered.shape == single.shape
    assert np.array_equal(gathered, single)
    assert float(open(path + ".max").read()) == 2.0

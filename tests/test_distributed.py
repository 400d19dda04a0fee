"""Multi-rank host logic of the sharded path on the CPU (gloo, world size 2):
the partition covers every matrix once, each rank processes only its slice,
and the timing reduction returns the maximum over ranks.  The per-rank
compute here is the CPU oracle standing in for the GPU call (the GPU path is
one independent call per rank)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2005_07403_gb300 import distributed as D


def test_partition_covers_each_matrix_once():
    for n in (0, 1, 7, 100, 65537):
        for world in (1, 2, 3, 8):
            seen = np.zeros(n, int)
            for r in range(world):
                s, c = D.partition(n, world, r)
                seen[s:s + c] += 1
            assert np.all(seen == 1)
    with pytest.raises(ValueError):
        D.partition(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    from paper_2005_07403_gb300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = inputs.normal_batch(10001, 4, 5)
    start, count, res = D.run_sharded(A, oracle.svd2, world, rank)
    full = oracle.svd2(A)
    ok = bool(np.array_equal(res["smax"], full["smax"][start:start + count]))
    t = D.max_over_ranks(10.0 * (rank + 1))
    D.barrier()
    q.put((rank, start, count, ok, t))
    dist.destroy_process_group()


def test_two_rank_sharded_run_and_timing_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1:3] for g in got] == [(0, 5001), (5001, 5000)]
    assert all(g[3] for g in got)
    assert all(g[4] == 20.0 for g in got)

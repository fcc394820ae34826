"""Multi-rank host logic on CPU: two gloo ranks run independent problems and
agree on the maximum step time (the only collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, size, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(size), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2105_12301_gb300 import ranks, inputs
    import torch.distributed as dist
    r, n = ranks.init("gloo")
    seed = ranks.problem_seed(1003, r)
    X = inputs.calcium(N=8, L=64, seed=seed)
    m = ranks.max_over_ranks(10.0 + r)
    ranks.barrier()
    q.put((r, n, seed, float(X[0, 0]), m))
    dist.destroy_process_group()


def test_two_ranks_independent_problems_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, s0, x0, m0), (r1, n1, s1, x1, m1) = res
    assert (r0, r1) == (0, 1) and n0 == n1 == 2
    assert s0 == 1003 and s1 != s0          # rank 0 runs the reference problem
    assert x0 != x1                          # the problems differ
    assert m0 == m1 == 11.0                  # both see the max over ranks

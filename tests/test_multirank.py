"""Multi-rank host logic on CPU (gloo): the row-block split of one problem
covers every library row exactly once and in order, the gathered blocks
reassemble the full matrix, and all ranks agree on the maximum step time."""
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


def _worker(rank, size, port, N, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(size), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2105_12301_gb300 import ranks
    r, n = ranks.init("gloo")
    b, e = ranks.row_block(N, r, n)
    # a stand-in for this rank's rho rows: entry (i, j) = 1000 i + j
    block = (1000.0 * torch.arange(b, e, dtype=torch.float64)[:, None]
             + torch.arange(N, dtype=torch.float64)[None, :])
    full = ranks.gather_row_blocks(block, N)
    m = ranks.max_over_ranks(10.0 + r)
    ranks.barrier()
    q.put((r, n, b, e, full.numpy().tolist(), m))
    dist.destroy_process_group()


def _run(size, N):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, size, port, N, q)) for r in range(size)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("N", [7, 8])
def test_two_ranks_split_rows_gather_and_max_time(N):
    import numpy as np
    res = _run(2, N)
    want = 1000.0 * np.arange(N)[:, None] + np.arange(N)[None, :]
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    # contiguous blocks in rank order covering every row exactly once
    assert res[0][2] == 0 and res[0][3] == res[1][2] and res[1][3] == N
    assert abs((res[0][3] - res[0][2]) - (res[1][3] - res[1][2])) <= 1
    for r in res:
        np.testing.assert_array_equal(np.array(r[4]), want)   # every rank has the full matrix
        assert r[5] == 11.0                                    # both see the max over ranks


def test_row_blocks_partition_for_many_sizes():
    from paper_2105_12301_gb300 import ranks
    for N in (1, 2, 5, 50000, 50001):
        for size in (1, 2, 3, 4, 8):
            blocks = [ranks.row_block(N, r, size) for r in range(size)]
            assert blocks[0][0] == 0 and blocks[-1][1] == N
            assert all(blocks[r][1] == blocks[r + 1][0] for r in range(size - 1))
            lens = [e - b for b, e in blocks]
            assert max(lens) - min(lens) <= 1

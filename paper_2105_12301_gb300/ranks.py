"""Process-group helpers for all-to-all CCM on N GPUs.

Libraries are independent (section 2.1: the four steps run per library and
target pair), so one problem splits into contiguous blocks of library rows,
one block per rank, with every series replicated on every rank: a rank
computes optimal E and the rho rows of its own libraries against all targets,
with no exchange during the computation.  The only collectives are the max
over ranks of the measured step time and an optional gather of the rho row
blocks after the step.
"""
import os

import torch
import torch.distributed as dist


def world():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def init(backend=None):
    """Initialise the default process group when launched with WORLD_SIZE > 1."""
    rank, size, _ = world()
    if size > 1 and not dist.is_initialized():
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return rank, size


def row_block(N, rank, size):
    """The library rows [begin, end) of rank `rank` out of `size`: contiguous,
    in rank order, covering 0..N-1 exactly once, sizes differing by at most 1."""
    return rank * N // size, (rank + 1) * N // size


def gather_row_blocks(block, N, device=None):
    """All rho rows on every rank: block is this rank's [end-begin][M] rows
    (row_block order); returns the [N][M] matrix.  Blocks are padded to the
    largest block for the collective and trimmed after it."""
    if not dist.is_initialized():
        return block
    size = dist.get_world_size()
    M = block.shape[1]
    rows = max(row_block(N, r, size)[1] - row_block(N, r, size)[0] for r in range(size))
    pad = torch.zeros((rows, M), dtype=block.dtype, device=device if device is not None else block.device)
    pad[: block.shape[0]] = block
    parts = [torch.empty_like(pad) for _ in range(size)]
    dist.all_gather(parts, pad)
    return torch.cat([parts[r][: row_block(N, r, size)[1] - row_block(N, r, size)[0]]
                      for r in range(size)])


def barrier():
    if dist.is_initialized():
        dist.barrier()


def max_over_ranks(value, device=None):
    """Maximum of a float over all ranks (the value itself when single-rank)."""
    if not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

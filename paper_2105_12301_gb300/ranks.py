"""Process-group helpers for running independent CCM problems on N GPUs.

Libraries are independent (section 2.1: the four steps run per library and
target pair), so N ranks run N independent problems with no data exchange;
the only collective is the max over ranks of the measured step time.
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


def problem_seed(base_seed, rank):
    """Seed of the problem a rank runs: rank 0 runs the reference workload."""
    return base_seed if rank == 0 else base_seed + 7919 * rank


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

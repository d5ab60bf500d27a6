"""Replica parallelism across GPUs: one process per GPU, each running its own independent
instances (the problem shards by instance, never within one: a single instance would need
global transposes every step).  No data-path collective exists; the only cross-rank
operations are the timing barrier and the max of the per-rank times.

Launch: ``python -m torch.distributed.run --nproc-per-node N ...`` (RANK, LOCAL_RANK,
WORLD_SIZE, MASTER_ADDR/PORT from the environment).  The process group uses NCCL when CUDA
is available and gloo otherwise (the CPU tests run two gloo ranks).
"""
import os
from typing import List, Tuple


def init_replicas(backend: str = None) -> Tuple[int, int, int]:
    """(world, rank, local_rank) from the environment; joins the process group if world > 1."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world, rank, local


def _device():
    import torch
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def max_over_ranks(x: float, world: int) -> float:
    """Maximum of a per-rank scalar (timings) over all ranks."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int) -> None:
    """All ranks meet; on a GPU also waits for the device."""
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def instance_seeds(count: int, rank: int) -> List[int]:
    """Seeds of the `count` instances rank `rank` runs: disjoint across ranks, so N ranks
    run N x count distinct instances (weak scaling)."""
    return list(range(rank * count, (rank + 1) * count))


def finalize(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()

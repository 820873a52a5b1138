"""Process-per-GPU helpers for benchmarking several GPUs of one node.

The path needs no exchange between GPUs: every (pixel, sample, band) path is
independent, so ranks render disjoint units.  Two partitions are offered:
  - sample passes: rank r renders the whole image with Philox key seed + r
    (independent samples; weak scaling, the image of N ranks averages N x spp);
  - band sub-domains: rank r renders a contiguous band range (the paper's
    spectral decomposition; strong scaling, partial XYZ images add up).
Only the timing uses a collective (a barrier and a max over ranks).
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass
class DistInfo:
    rank: int = 0
    world: int = 1
    local_rank: int = 0
    initialized: bool = False


def init_from_env(backend: str = "nccl") -> DistInfo:
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    info = DistInfo(rank, world, local, False)
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend, rank=rank, world_size=world)
        info.initialized = True
    return info


def barrier(info: DistInfo, device=None):
    if info.world > 1:
        import torch.distributed as dist
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def max_over_ranks(info: DistInfo, value: float, device=None) -> float:
    if info.world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if (device is not None and dist.get_backend() == "nccl") else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(info: DistInfo, value: float, device=None) -> float:
    if info.world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if (device is not None and dist.get_backend() == "nccl") else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def rank_seed(seed: int, rank: int) -> int:
    """Philox key of a rank's sample passes (disjoint streams per rank)."""
    return (int(seed) + (int(rank) << 32)) & 0xFFFFFFFFFFFFFFFF


def band_shard(n_bands: int, world: int, rank: int):
    """Contiguous band sub-domain [first, first + count) of a rank; the
    ranges tile [0, n_bands) and differ in size by at most one band."""
    base, extra = divmod(n_bands, world)
    first = rank * base + min(rank, extra)
    count = base + (1 if rank < extra else 0)
    return first, count


def finish(info: DistInfo):
    if info.initialized:
        import torch.distributed as dist
        dist.destroy_process_group()

"""Process-per-GPU helpers for rendering on several GPUs of one node.

Every (pixel, sample, band) path is independent, so ranks render disjoint
units.  Two partitions are offered:
  - sample passes: rank r renders the whole image with Philox key seed + r
    (independent samples; weak scaling, the image of N ranks averages N x spp);
    no data moves between ranks;
  - band sub-domains (the paper's spectral decomposition, title and section
    5, with wavelength ranges as the sub-domains): rank r renders the bands
    band_shard(B, N, r) of every path; its XYZ image of those bands is a
    partial sum of the full image's, so one reduce-sum of the [P x 3] FP32
    partials to rank 0 (NCCL on GPUs, gloo on CPU) forms the image.  That
    reduce is the path's only exchange.
Timing adds a barrier and a max over ranks.
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


def render_band_sharded(info: DistInfo, renderer, cameras, spp: int, depth: int, seed: int, n_bands: int,
                        dst: int = 0, **render_kw):
    """Renders this rank's band sub-domain of the views and reduces the XYZ
    partials of all ranks onto rank `dst`.  `renderer.render(cameras, spp,
    depth, seed, band_first=, band_count=, spectral=False, **render_kw)` must
    return {"xyz": [P, 3] float32 tensor} on the collective's device.
    Returns (xyz, (first, count)); xyz holds the full image on `dst` and
    this rank's partial elsewhere."""
    first, count = band_shard(n_bands, info.world, info.rank)
    if count == 0:
        raise ValueError("more ranks than bands")
    out = renderer.render(cameras, spp, depth, seed, band_first=first, band_count=count, spectral=False,
                          **render_kw)
    xyz = out["xyz"]
    if info.world > 1:
        import torch.distributed as dist
        dist.reduce(xyz, dst=dst, op=dist.ReduceOp.SUM)
    return xyz, (first, count)


def finish(info: DistInfo):
    if info.initialized:
        import torch.distributed as dist
        dist.destroy_process_group()

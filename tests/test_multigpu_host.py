"""Host logic of the multi-GPU paths, run as two gloo ranks on CPU: timing
collectives, per-rank seeds, band shards, and the band-sharded render whose
XYZ partials are reduced to rank 0 (the renderer of each rank is the FP64
oracle here; on GPUs it is the CUDA library and the reduce runs over NCCL)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1912_04000_gb300 import multigpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    info = multigpu.init_from_env("gloo")
    multigpu.barrier(info)
    mx = multigpu.max_over_ranks(info, 10.0 + rank)
    sm = multigpu.sum_over_ranks(info, 1.0 + rank)
    seeds = multigpu.rank_seed(7, rank)
    q.put((rank, mx, sm, seeds, multigpu.band_shard(81, world, rank)))
    multigpu.finish(info)


def test_two_gloo_ranks():
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
    assert [r[1] for r in res] == [11.0, 11.0]
    assert [r[2] for r in res] == [3.0, 3.0]
    assert res[0][3] != res[1][3]
    (f0, c0), (f1, c1) = res[0][4], res[1][4]
    assert f0 == 0 and f0 + c0 == f1 and f1 + c1 == 81


@pytest.mark.parametrize("n,w", [(81, 1), (81, 2), (81, 4), (81, 8), (16, 3), (5, 8)])
def test_band_shards_tile(n, w):
    got = [multigpu.band_shard(n, w, r) for r in range(w)]
    pos = 0
    for f, c in got:
        assert f == pos
        pos += c
    assert pos == n
    assert max(c for _, c in got) - min(c for _, c in got) <= 1


class _OracleRenderer:
    """The oracle behind the renderer's render() signature (test adapter)."""

    def __init__(self, wl):
        import oracle
        self.sc = oracle.OracleScene(wl.scene, wl.spectra)

    def render(self, cameras, spp, depth, seed, band_first=0, band_count=None, spectral=False):
        import torch
        r = self.sc.render(cameras, spp, depth, seed, band_first=band_first, band_count=band_count, n_threads=1)
        return {"xyz": torch.as_tensor(r["xyz"].astype("float32"))}


def _band_worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    from paper_1912_04000_gb300 import scenes
    info = multigpu.init_from_env("gloo")
    wl = scenes.tiny_box(width=24, height=16, spp=2)
    xyz, shard = multigpu.render_band_sharded(info, _OracleRenderer(wl), wl.cameras, wl.spp, wl.depth, wl.seed,
                                              wl.band_count)
    q.put((rank, shard, xyz.numpy() if rank == 0 else None))
    multigpu.finish(info)


@pytest.mark.parametrize("world", [2, 3])
def test_band_sharded_render_reduces_to_full_image(world):
    import numpy as np

    import oracle
    from paper_1912_04000_gb300 import scenes
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_band_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = [r[1] for r in res]
    assert shards[0][0] == 0 and sum(c for _, c in shards) == 16
    wl = scenes.tiny_box(width=24, height=16, spp=2)
    full = oracle.OracleScene(wl.scene, wl.spectra).render(wl.cameras, wl.spp, wl.depth, wl.seed)["xyz"]
    # the partials are FP32 images: the reduced image equals the one-rank
    # image to FP32 summation order
    np.testing.assert_allclose(res[0][2], full, rtol=2e-6, atol=1e-9)

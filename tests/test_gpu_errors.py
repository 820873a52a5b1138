"""The boundary's error codes, each reached without a device fault: scenes
the library refuses (RT_ERR_SCENE), calls out of order (RT_ERR_STATE), ray
queues smaller than a wave (RT_ERR_QUEUE_OVERFLOW, nothing written past the
caller's buffers), traversal loops that reach their cap (RT_ERR_TIMEOUT: the
kernels stop and return), and a failing CUDA call -- injected on the host,
the call not made -- that poisons the context (RT_ERR_CUDA, then
RT_ERR_STATE).  After each recoverable error the context renders correctly."""
import numpy as np
import pytest

from paper_1912_04000_gb300 import scenes
from paper_1912_04000_gb300._native import RtError

pytestmark = pytest.mark.gpu

ARG, SCENE, CUDA, QUEUE, TIMEOUT, STATE = 1, 2, 4, 5, 6, 7


@pytest.fixture(scope="module")
def R():
    from paper_1912_04000_gb300.renderer import Renderer
    return Renderer(0)


def _status(fn, *a, **k):
    with pytest.raises(RtError) as e:
        fn(*a, **k)
    return e.value.status


def _bad_scene(kind):
    wl = scenes.tiny_box(width=8, height=8, spp=1)
    sc = wl.scene
    v, t, m = sc.verts.copy(), sc.tris.copy(), sc.mat_id.copy()
    mt, th = sc.mat_type.copy(), sc.mat_thickness.copy()
    if kind == "nan_vertex":
        v[3, 1] = np.nan
    elif kind == "inf_vertex":
        v[0, 2] = np.inf
    elif kind == "index":
        t[5, 2] = v.shape[0]
    elif kind == "material":
        m[7] = mt.shape[0]
    elif kind == "degenerate":
        t[2] = (t[2, 0], t[2, 0], t[2, 1])
    elif kind == "material_type":
        mt[0] = 9
    elif kind == "thickness":
        th[1] = -0.01
    return scenes.Scene(v, t, m, mt, th), wl


@pytest.mark.parametrize("kind", ["nan_vertex", "inf_vertex", "index", "material", "degenerate", "material_type",
                                  "thickness"])
def test_bad_scene_rejected(R, kind):
    bad, wl = _bad_scene(kind)
    assert _status(R.load_scene, bad) == SCENE
    # the context is still usable
    R.load(wl)
    out = R.render(wl.cameras, 1, wl.depth, 0, xyz_mode=2)
    assert np.isfinite(out["spectral"].cpu().numpy()).all()


def test_calls_out_of_order():
    from paper_1912_04000_gb300.renderer import Renderer
    R2 = Renderer(0)
    wl = scenes.tiny_box(width=8, height=8, spp=1)
    assert _status(R2.render, wl.cameras, 1, 2, 0, band_count=4) == STATE  # no scene
    assert _status(R2.guide_init, seed=1) == STATE
    R2.load_scene(wl.scene)
    assert _status(R2.render, wl.cameras, 1, 2, 0, band_count=4) == STATE  # no spectra
    R2.set_spectra(wl.spectra)
    R2.render(wl.cameras, 1, 2, 0)
    R2.close()


def test_queue_overflow_reported_and_contained(R):
    import torch
    wl = scenes.tiny_box(width=32, height=24, spp=2)
    R.load(wl)
    P, B = wl.n_pixels, wl.band_count
    ref = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)["spectral"].cpu().numpy()
    guard = 4096
    big = torch.full((P * B + guard,), -7.0, dtype=torch.float64, device="cuda")
    bigx = torch.full((P * 3 + guard,), -7.0, dtype=torch.float32, device="cuda")
    out_s = big[:P * B].view(P, B)
    out_x = bigx[:P * 3].view(P, 3)
    R.set_limits(queue_capacity=1000)
    try:
        assert _status(R.render, wl.cameras, wl.spp, wl.depth, wl.seed, out_spectral=out_s, out_xyz=out_x) == QUEUE
        # with guided sampling too (its query queue)
        R.guide_init(seed=2, log2_table=12)
        assert _status(R.render, wl.cameras, wl.spp, wl.depth, wl.seed, guided=True, xyz=False) == QUEUE
    finally:
        R.set_limits()
    torch.cuda.synchronize()
    assert torch.all(big[P * B:] == -7.0) and torch.all(bigx[P * 3:] == -7.0)
    again = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)["spectral"].cpu().numpy()
    assert np.array_equal(again, ref)


def test_traversal_cap_reported(R):
    wl = scenes.nave(width=32, height=24, n_bands=4, spp=1, depth=3)
    R.load(wl)
    ref = R.render(wl.cameras, 1, wl.depth, 0, xyz_mode=2)["spectral"].cpu().numpy()
    R.set_limits(traversal_steps=3)
    try:
        assert _status(R.render, wl.cameras, 1, wl.depth, 0, xyz_mode=2) == TIMEOUT
        assert _status(R.trace_closest, np.float32([[10, 2, 10]]), np.float32([[1, 0, 0]])) == TIMEOUT
    finally:
        R.set_limits()
    again = R.render(wl.cameras, 1, wl.depth, 0, xyz_mode=2)["spectral"].cpu().numpy()
    assert np.array_equal(again, ref)


def test_failed_cuda_call_poisons_context():
    from paper_1912_04000_gb300.renderer import Renderer
    R2 = Renderer(0)
    wl = scenes.tiny_box(width=8, height=8, spp=1)
    R2.load(wl)
    R2.render(wl.cameras, 1, wl.depth, 0)
    R2.set_limits(fail_cuda_call=1)
    assert _status(R2.render, wl.cameras, 1, wl.depth, 0) == CUDA
    # every later call refuses: the context is unusable
    assert _status(R2.render, wl.cameras, 1, wl.depth, 0) == STATE
    assert _status(R2.load, wl) == STATE
    assert _status(R2.set_limits) == STATE
    R2.close()
    # other contexts on the device are unaffected
    R3 = Renderer(0).load(wl)
    assert np.isfinite(R3.render(wl.cameras, 1, wl.depth, 0)["spectral"].cpu().numpy()).all()
    R3.close()


def test_argument_errors(R):
    wl = scenes.tiny_box(width=8, height=8, spp=1)
    R.load(wl)
    assert _status(R.render, wl.cameras, 1, 0, 0) == ARG  # depth 0
    assert _status(R.render, wl.cameras, 1, 2, 0, band_first=10, band_count=10) == ARG
    bad = [scenes.Camera((0, 0, 0), (0, 0, 0), (0, 1, 0), 60.0, 8, 8)]
    assert _status(R.render, bad, 1, 2, 0) == ARG  # look == pos

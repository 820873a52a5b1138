"""Guided rendering through the C ABI: progressive sample ranges compose
exactly; one-sample MIS with the learned guide leaves the estimate unbiased
(z-test against the plain tracer); online training inside the render runs."""
import numpy as np
import pytest

from paper_1912_04000_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1912_04000_gb300.renderer import Renderer
    return Renderer(0)


def test_progressive_equals_single_call(R):
    import torch
    wl = scenes.tiny_box(width=40, height=30, spp=4)
    R.load(wl)
    full = R.render(wl.cameras, 4, wl.depth, wl.seed, xyz_mode=2)
    acc = torch.empty_like(full["spectral"])
    R.render(wl.cameras, 2, wl.depth, wl.seed, out_spectral=acc, xyz_mode=2)
    out = R.render(wl.cameras, 2, wl.depth, wl.seed, out_spectral=acc, sample_first=2, accumulate=True, spp_total=4,
                   xyz_mode=2)
    assert torch.equal(acc, full["spectral"])
    np.testing.assert_allclose(out["xyz"].cpu().numpy(), full["xyz"].cpu().numpy(), rtol=1e-6, atol=1e-12)


def _z(a, b):
    d = (a - b).ravel()
    return abs(d.mean()) / (d.std() / np.sqrt(d.size))


@pytest.mark.parametrize("trained", [False, True])
def test_guided_is_unbiased(R, trained):
    wl = scenes.tiny_box(width=64, height=48, spp=32, n_bands=4)
    R.load(wl)
    R.guide_init(seed=5, log2_table=14, guide_depth=3)
    if trained:
        R.render(wl.cameras, 8, wl.depth, 1234, guided=True, guide_collect=1, guide_train_steps=8, xyz=False)
    plain = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz=False)["spectral"].cpu().numpy() / wl.spp
    guided = R.render(wl.cameras, wl.spp, wl.depth, wl.seed + 99, guided=True, xyz=False)["spectral"].cpu().numpy()
    guided /= wl.spp
    assert np.isfinite(guided).all() and (guided >= 0).all()
    assert _z(guided, plain) < 5.0
    # and the guided estimate is not identical to the plain one (the guide is used)
    assert not np.array_equal(guided, plain)


def test_query_order_changes_nothing(R):
    """With a frozen guide every query is evaluated on its own (one MMA row,
    its own Philox counters), so sorting the queries by position before the
    network runs (guide_order 1) changes no bit of the image."""
    wl = scenes.nave(width=96, height=64, n_bands=9, spp=2, depth=4)
    R.load(wl)
    R.guide_init(seed=3, log2_table=16)
    a = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, guided=True, xyz=False)["spectral"].cpu().numpy()
    b = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, guided=True, xyz=False, guide_order=1)["spectral"].cpu().numpy()
    assert np.array_equal(a, b)


def test_training_in_render_changes_guide(R):
    wl = scenes.nave(width=96, height=64, n_bands=9, spp=2, depth=4)
    R.load(wl)
    R.guide_init(seed=2, log2_table=16)
    g0, w0 = R.guide_get_params()
    out = R.render(wl.cameras, 2, wl.depth, wl.seed, guided=True, guide_collect=2, guide_train_steps=4, xyz=False)
    g1, w1 = R.guide_get_params()
    assert np.isfinite(g1).all() and np.isfinite(w1).all()
    assert not np.array_equal(w0, w1) and not np.array_equal(g0, g1)
    assert np.isfinite(out["spectral"].cpu().numpy()).all()


def test_trained_guide_lowers_mse_at_equal_spp(R):
    """What the trained network gains over the method without it: on the
    nave (128 x 96, 81 bands, depth 8) the guided tracer, trained online over
    its first 16 passes (256 Adam steps), has a lower MSE than the plain
    tracer at equal spp against a 1024-spp plain reference."""
    import torch
    wl = scenes.nave(width=128, height=96)
    R.load(wl)
    P, B = wl.n_pixels, wl.band_count
    ref = R.render(wl.cameras, 1024, wl.depth, 777)["xyz"].cpu().numpy().astype(np.float64)
    spp, n_train = 64, 16
    plain = R.render(wl.cameras, spp, wl.depth, 0)["xyz"].cpu().numpy().astype(np.float64)
    R.guide_init(seed=11, guide_depth=2)
    acc = torch.zeros((P, B), dtype=torch.float64, device="cuda")
    for s_ in range(n_train):
        R.render(wl.cameras, 1, wl.depth, 0, out_spectral=acc, sample_first=s_, accumulate=s_ > 0, spp_total=spp,
                 guided=True, guide_collect=1, guide_train_steps=16, xyz=False)
    guided = R.render(wl.cameras, spp - n_train, wl.depth, 0, out_spectral=acc, sample_first=n_train,
                      accumulate=True, spp_total=spp, guided=True)["xyz"].cpu().numpy().astype(np.float64)
    mse_p = np.mean((plain - ref) ** 2)
    mse_g = np.mean((guided - ref) ** 2)
    print("equal-spp MSE plain / guided", mse_p / mse_g)
    assert mse_p / mse_g > 1.3


def test_trained_guide_lowers_mse_at_equal_time(R):
    """The configuration's target (at least 2x lower MSE at equal wall time,
    against a high-spp plain reference) on a 256 x 192 view of the nave, 81
    bands, depth 8: the guided tracer, trained online over its first 32 of
    256 passes (32 Adam steps per wave), against the plain tracer given the
    same wall time; the reference is 4096 plain spp with another seed (the
    bench's equal-time sub-record is the same experiment)."""
    import time

    import torch
    wl = scenes.nave(width=256, height=192)
    R.load(wl)
    P, B = wl.n_pixels, wl.band_count
    ref = R.render(wl.cameras, 4096, wl.depth, 777)["xyz"].cpu().numpy().astype(np.float64)
    R.render(wl.cameras, 8, wl.depth, 5)  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    R.render(wl.cameras, 64, wl.depth, 5, xyz=False)
    torch.cuda.synchronize()
    t_per_spp = (time.perf_counter() - t0) / 64
    spp, n_train = 256, 32
    R.guide_init(seed=11, guide_depth=2, mis_alpha=0.7)
    acc = torch.zeros((P, B), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s_ in range(n_train):
        R.render(wl.cameras, 1, wl.depth, 0, out_spectral=acc, sample_first=s_, accumulate=s_ > 0, spp_total=spp,
                 guided=True, guide_collect=4, guide_train_steps=32, xyz=False)
    out = R.render(wl.cameras, spp - n_train, wl.depth, 0, out_spectral=acc, sample_first=n_train, accumulate=True,
                   spp_total=spp, guided=True)
    torch.cuda.synchronize()
    t_guided = time.perf_counter() - t0
    guided = out["xyz"].cpu().numpy().astype(np.float64)
    spp_eq = max(1, int(round(t_guided / t_per_spp)))
    plain = R.render(wl.cameras, spp_eq, wl.depth, 0)["xyz"].cpu().numpy().astype(np.float64)
    ratio = np.mean((plain - ref) ** 2) / np.mean((guided - ref) ** 2)
    print(f"equal time: guided {spp} spp in {t_guided:.2f} s, plain {spp_eq} spp; MSE plain / guided {ratio:.2f}")
    assert ratio > 2.0

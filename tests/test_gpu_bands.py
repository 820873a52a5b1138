"""Four bands per path on the GPU against the oracle's four-band estimator:
full images (box, dispersive prism), per-path records, the full-size nave
(81 bands: 18 paths of four bands and 3 of three per pixel and sample),
wave decomposition, band sub-ranges, graph replay, and the option's
argument checks."""
import numpy as np
import pytest

import oracle
from paper_1912_04000_gb300 import scenes
from paper_1912_04000_gb300._native import RtError

from parity import assert_parity, xyz_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1912_04000_gb300.renderer import Renderer
    return Renderer(0)


def _oracle(wl, **kw):
    return oracle.OracleScene(wl.scene, wl.spectra).render(wl.cameras, wl.spp, wl.depth, wl.seed, bands_per_path=4,
                                                           **kw)


@pytest.mark.parametrize("name", ["tiny_box", "prism_room"])
def test_full_image(R, name):
    wl = scenes.tiny_box() if name == "tiny_box" else scenes.prism_room()
    R.load(wl)
    out = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, bands_per_path=4)
    o = _oracle(wl)
    m = assert_parity(out["xyz"].cpu().numpy(), o["xyz"], name)
    print(name, "four-band parity", m)
    gs = out["spectral"].cpu().numpy()
    rel = np.abs(gs - o["spectral_sum"]).sum() / np.abs(o["spectral_sum"]).sum()
    assert rel < 1e-5
    st = out["stats"]
    npix = sum(c.width * c.height for c in wl.cameras)
    assert st["paths"] == npix * wl.spp * wl.spectra.n.shape[1]


@pytest.mark.parametrize("name", ["tiny_box", "prism_room"])
def test_per_path_records(R, name):
    if name == "tiny_box":
        wl = scenes.tiny_box(width=40, height=30, spp=3, depth=6)
    else:
        wl = scenes.prism_room(width=48, height=36, spp=4)
    R.load(wl)
    rng = np.random.default_rng(4)
    pix = np.sort(rng.choice(wl.n_pixels, 64, replace=False)).astype(np.int64)
    out = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, probe_pixels=pix, xyz_mode=2, bands_per_path=4)
    o = _oracle(wl, pixels=pix.astype(np.uint32), record_paths=True)
    gL = out["probe_L"].cpu().numpy()
    gS = out["probe_sig"].cpu().numpy().view(np.uint32)
    same = gS == o["path_sig"]
    print(name, "four-band paths with identical events", same.mean())
    assert same.mean() >= 0.99
    np.testing.assert_allclose(gL[same], o["path_L"][same], rtol=5e-5, atol=1e-9)


def test_nave_sampled_pixels(R):
    """1024 x 768, 81 bands (per pixel and sample 18 paths of four bands and
    3 of three), 16 spp, depth 8."""
    wl = scenes.nave()
    R.load(wl)
    rng = np.random.default_rng(9)
    pix = np.sort(rng.choice(wl.n_pixels, 48, replace=False)).astype(np.int64)
    out = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, probe_pixels=pix, xyz_mode=2, bands_per_path=4)
    o = _oracle(wl, pixels=pix.astype(np.uint32), record_paths=True)
    gS = out["probe_sig"].cpu().numpy().view(np.uint32)
    gL = out["probe_L"].cpu().numpy()
    same = gS == o["path_sig"]
    print("nave four-band: paths with identical events", same.mean())
    assert same.mean() >= 0.99
    np.testing.assert_allclose(gL[same], o["path_L"][same], rtol=1e-4, atol=1e-7)
    g = out["xyz"].cpu().numpy()[pix]
    clean = same.reshape(len(pix), -1).all(1)
    print("nave four-band sampled-pixel parity", xyz_parity(g, o["xyz"]))
    if clean.any():
        assert_parity(g[clean], o["xyz"][clean], "nave four-band clean pixels")


def test_waves_ranges_and_graph(R):
    wl = scenes.prism_room(width=64, height=48, n_bands=16, spp=3)
    R.load(wl)
    a = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2, bands_per_path=4)["spectral"].cpu().numpy()
    # many small waves: the same bits
    b = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2, bands_per_path=4,
                 wave_capacity=5000)["spectral"].cpu().numpy()
    assert np.array_equal(a, b)
    # groups are formed inside the band range: sub-ranges and a partial last
    # row of the grouping against the oracle
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    for first, count in ((4, 8), (0, 14), (3, 5)):
        c = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, band_first=first, band_count=count,
                     bands_per_path=4)
        o = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, band_first=first, band_count=count, bands_per_path=4)
        assert_parity(c["xyz"].cpu().numpy(), o["xyz"], f"bands [{first}, {first + count})")
    # graph capture and replay
    e = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2, bands_per_path=4,
                 use_graph=True)["spectral"].cpu().numpy()
    f = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2, bands_per_path=4,
                 use_graph=True)["spectral"].cpu().numpy()
    assert np.array_equal(e, a) and np.array_equal(f, a)
    # one traced path serves four bands
    one = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)["stats"]
    four = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2, bands_per_path=4)["stats"]
    assert one["paths"] == four["paths"]
    assert four["ext_rays"] * 3 < one["ext_rays"]


def test_arguments_checked(R):
    wl = scenes.tiny_box(width=16, height=16, spp=1)
    R.load(wl)
    with pytest.raises(RtError):
        R.render(wl.cameras, 1, 4, 0, bands_per_path=3)
    with pytest.raises(RtError):
        R.render(wl.cameras, 1, 4, 0, bands_per_path=4, trace_variant=1)
    R.guide_init(seed=1, log2_table=12)
    with pytest.raises(RtError):
        R.render(wl.cameras, 1, 4, 0, bands_per_path=4, guided=True)

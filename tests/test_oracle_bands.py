"""Oracle's four-bands-per-path estimator pinned against the one-band
estimator it must agree with: identical paths where the bands cannot differ
(a spectrally flat scene, a white furnace, a conductor), and the same
expectation per band where they do (dispersive prism, absorbing glass,
solid slab), by z-tests over many paths."""
import math

import numpy as np
import pytest

import oracle
from paper_1912_04000_gb300 import scenes


def _render(wl, bpp, spp=None, **kw):
    return oracle.OracleScene(wl.scene, wl.spectra).render(wl.cameras, spp or wl.spp, wl.depth, wl.seed,
                                                           record_paths=True, bands_per_path=bpp, **kw)


def _flatten(wl, src_band):
    """Every band takes the tables of band src_band (k = 0: no lambda in Beer-Lambert)."""
    sp = wl.spectra
    for a in (sp.n, sp.rho, sp.le):
        a[:] = a[:, src_band:src_band + 1]
    sp.k[:] = 0.0
    sp.sun_L[:] = sp.sun_L[src_band]
    return wl


def test_flat_spectrum_paths_equal_one_band_paths():
    # before any refraction every choice is the one-band choice of the
    # group's first band, so each band's path value is that band's value
    # (path unit g carries bands g, g + 2, g + 4, g + 6 of 8)
    wl = _flatten(scenes.tiny_box(width=24, height=18, n_bands=8, spp=3, depth=6), 0)
    one = _render(wl, 1)["path_L"]
    four = _render(wl, 4)["path_L"]
    for g in range(2):
        for q in range(4):
            np.testing.assert_allclose(four[:, :, g + 2 * q], one[:, :, g], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("albedo,depth", [(0.5, 5), (0.8, 3)])
def test_white_furnace_exact(albedo, depth):
    wl = scenes.furnace_box(albedo=albedo, le=2.0, depth=depth, n_bands=6)
    L = _render(wl, 4)["path_L"]
    np.testing.assert_allclose(L, 2.0 * (1.0 - albedo ** depth), rtol=1e-6)


def test_conductor_weights_per_band():
    # camera -> metal -> sun with a different (n, k) per band: every path is
    # exactly R_b(30 deg) in each band, as with one band per path
    wl = scenes.slab_view(n_glass=1.0, k_glass=1.0, spp=8, sun_side="reflect", material=scenes.CONDUCTOR)
    wl.spectra.n[0] = [0.6, 1.2, 2.5]
    wl.spectra.k[0] = [3.0, 4.0, 5.5]
    L = _render(wl, 4)["path_L"]
    for j in range(3):
        R = oracle.fresnel(math.cos(math.radians(30.0)), float(wl.spectra.n[0, j]), float(wl.spectra.k[0, j]))
        np.testing.assert_allclose(L[:, :, j], R, rtol=1e-5)


def _z(a, b):
    a, b = a.ravel(), b.ravel()
    se = math.sqrt(a.var() / a.size + b.var() / b.size)
    return abs(a.mean() - b.mean()) / se if se > 0 else abs(a.mean() - b.mean())


def test_thin_glass_slab_mean_per_band():
    # the mixture probability of the carried bands is not any band's own
    # R_s / (R_s + T_s), yet each band's mean stays T_s
    wl = scenes.slab_view(k_glass=3e-5, spp=4096)
    wl.spectra.n[0] = [1.45, 1.6, 1.75]
    L = _render(wl, 4)["path_L"]
    c = math.cos(math.radians(30.0))
    for j, lam in enumerate((450.0, 550.0, 650.0)):
        rs, ts = oracle.slab(c, float(wl.spectra.n[0, j]), 3e-5, lam, 0.01)
        v = L[:, :, j].ravel()
        assert abs(v.mean() - ts) < 5 * v.std() / math.sqrt(v.size)


def test_solid_slab_mean_per_band():
    wl = scenes.solid_slab_view(n_glass=1.5, k_glass=2e-6, spp=8192)
    wl.spectra.n[0] = [1.48, 1.52, 1.6]
    L = _render(wl, 4)["path_L"]
    ci = math.cos(math.radians(30.0))
    for j, lam in enumerate((450.0, 550.0, 650.0)):
        rs, ts = oracle.slab(ci, float(wl.spectra.n[0, j]), 2e-6, lam, 0.01)
        v = L[:, :, j].ravel()
        assert abs(v.mean() - ts) < 5 * v.std() / math.sqrt(v.size) + 1e-9
    # after the refraction only one band of a path carries light
    nz = (L != 0.0).sum(-1)
    assert nz.max() == 1


@pytest.mark.parametrize("name", ["tiny_box", "prism_room"])
def test_same_expectation_as_one_band(name):
    if name == "tiny_box":
        wl = scenes.tiny_box(width=32, height=24, n_bands=16, spp=24, depth=5)
    else:
        wl = scenes.prism_room(width=32, height=24, n_bands=16, spp=24)
    one = _render(wl, 1)["path_L"]
    four = _render(wl, 4)["path_L"]
    z = np.array([_z(four[:, :, j], one[:, :, j]) for j in range(wl.spectra.n.shape[1])])
    assert z.max() < 5.0, z
    # the four-band paths are not the one-band paths (the bands share choices)
    assert not np.array_equal(four, one)


def test_band_groups_and_ranges():
    """Groups are formed inside the rendered range: bands first + g + q G,
    G = ceil(count / 4), with the Philox stream of band first + g; a partial
    last row of the grouping (count not a multiple of 4) carries fewer bands."""
    wl = _flatten(scenes.tiny_box(width=12, height=10, n_bands=16, spp=2), 3)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    for first, count in ((4, 8), (0, 14), (3, 5)):
        G = (count + 3) // 4
        one = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, band_first=first, band_count=count,
                        record_paths=True)["path_L"]
        four = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, band_first=first, band_count=count,
                         record_paths=True, bands_per_path=4)["path_L"]
        for j in range(count):
            np.testing.assert_allclose(four[:, :, j], one[:, :, j % G], rtol=1e-12, atol=1e-15)

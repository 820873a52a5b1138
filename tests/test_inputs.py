"""Seeded input generators: sizes and structure of the synthetic workloads."""
import numpy as np

from paper_1912_04000_gb300 import scenes


def test_band_layout():
    lam = scenes.band_wavelengths(380, 780, 81)
    np.testing.assert_allclose(np.diff(lam), 5.0)
    lam = scenes.band_wavelengths(400, 700, 16)
    np.testing.assert_allclose(np.diff(lam), 20.0)


def test_tiny_box():
    wl = scenes.tiny_box()
    assert wl.scene.n_tris == 12
    assert (wl.scene.mat_id == 1).sum() == 2
    assert wl.n_paths == 128 * 128 * 4 * 16
    n = wl.spectra.n[1]
    np.testing.assert_allclose(n, 1.5 + 0.004 / (wl.spectra.lambda_nm * 1e-3) ** 2, rtol=1e-6)
    assert abs(wl.spectra.sun_half_angle - 0.25) < 1e-9


def test_nave_sizes():
    wl = scenes.nave(width=32, height=24)
    nt = wl.scene.n_tris
    assert 190_000 < nt < 210_000, nt
    assert wl.scene.n_mat == 20
    glass = wl.scene.mat_type == scenes.THIN_GLASS
    assert glass.sum() == 16
    g = np.where(glass)[0]
    assert (wl.spectra.n[g] >= 1.45 - 1e-6).all() and (wl.spectra.n[g] <= 1.6 + 1e-6).all()
    assert (wl.spectra.k[g] >= 1e-7 * (1 - 1e-5)).all() and (wl.spectra.k[g] <= 1e-5 * (1 + 1e-5)).all()
    stone = np.where(~glass)[0]
    assert (wl.spectra.rho[stone] >= 0.3 - 1e-6).all() and (wl.spectra.rho[stone] <= 0.8 + 1e-6).all()
    assert wl.spectra.n_bands == 81
    # deterministic
    wl2 = scenes.nave(width=32, height=24)
    assert np.array_equal(wl.scene.verts, wl2.scene.verts)
    assert np.array_equal(wl.spectra.k, wl2.spectra.k)


def test_views_uneven():
    wl = scenes.nave_views(n_views=32, n_bands=4, spp=1, base=scenes.nave(width=8, height=8, n_bands=4))
    ws = [c.width for c in wl.cameras]
    hs = [c.height for c in wl.cameras]
    assert len(ws) == 32 and min(ws) >= 256 and max(ws) <= 1024
    assert all(w % 16 == 0 for w in ws + hs)
    assert len(set(zip(ws, hs))) > 20


def test_cmf_weights_normalised():
    for lo, hi, B in ((380, 780, 81), (400, 700, 16)):
        lam = scenes.band_wavelengths(lo, hi, B)
        w = scenes.xyz_weights(lam)
        assert abs(w[:, 1].sum() - 1.0) < 1e-12

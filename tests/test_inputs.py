"""Seeded input generators: sizes and structure of the synthetic workloads."""
import math

import numpy as np
import pytest

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


def test_rayleigh_optical_depth_published_values():
    # sea-level Rayleigh optical depth: about 0.364 at 400 nm, 0.097 at
    # 550 nm and 0.036 at 700 nm (published sea-level values, e.g. Bucholtz,
    # Appl. Opt. 34, 1995)
    tau = scenes.rayleigh_optical_depth(np.array([400.0, 550.0, 700.0]))
    np.testing.assert_allclose(tau, [0.364, 0.0973, 0.0362], rtol=0.02)
    # close to the lambda^-4 law, a little steeper
    r = tau[0] / tau[2]
    assert (700.0 / 400.0) ** 4 < r < (700.0 / 400.0) ** 4.2


def test_air_mass_published_values():
    # Kasten and Young's formula: 1 at the zenith, about 1/sin h for a high
    # sun, 37.9 at the horizon
    assert abs(scenes.air_mass(90.0) - 1.0) < 1e-3
    assert abs(scenes.air_mass(30.0) - 2.0) < 0.01
    assert abs(scenes.air_mass(0.0) - 37.92) < 0.05
    ms = [scenes.air_mass(h) for h in (90, 60, 30, 10, 5, 0)]
    assert all(a < b for a, b in zip(ms, ms[1:]))


def test_low_sun_is_redder():
    lam = scenes.band_wavelengths(400, 700, 16)
    top = scenes.sun_spectrum(lam)
    prev = None
    for h in (90.0, 35.0, 10.0, 2.0):
        s = scenes.sun_spectrum(lam, elevation_deg=h)
        assert np.all(s < top) and np.all(s > 0)
        ratio = s[0] / s[-1]   # blue over red
        if prev is not None:
            assert ratio < prev
        prev = ratio
    wl = scenes.prism_room()
    np.testing.assert_allclose(wl.spectra.sun_L, scenes.sun_spectrum(wl.spectra.lambda_nm.astype(np.float64),
                                                                     elevation_deg=35.0), rtol=1e-6)


def test_crystal_nave_solids():
    wl = scenes.crystal_nave(width=32, height=24)
    base = scenes.nave(width=32, height=24)
    sc = wl.scene
    nb = base.scene.n_tris
    assert sc.n_tris == nb + 4 * 320 + 4 * 8
    assert np.array_equal(sc.mat_id[:nb], base.scene.mat_id)
    assert list(sc.mat_type[-2:]) == [scenes.DIELECTRIC, scenes.DIELECTRIC]
    crown, flint = sc.n_mat - 2, sc.n_mat - 1

    def volume(m):
        t = sc.verts[sc.tris[sc.mat_id == m]].astype(np.float64)
        return np.einsum("ij,ij->i", t[:, 0], np.cross(t[:, 1], t[:, 2])).sum() / 6.0

    # outward winding gives positive volumes: four 1.2 m prisms 2 m long and
    # four 320-face spheres of radius 0.8 (a little under the true sphere)
    assert volume(flint) == pytest.approx(4 * (math.sqrt(3.0) / 4.0 * 1.2 ** 2) * 2.0, rel=1e-5)
    vs = 4 * 4.0 / 3.0 * math.pi * 0.8 ** 3
    assert 0.95 * vs < volume(crown) < vs
    # dispersion: the flint bends blue more than red
    assert wl.spectra.n[flint][0] > wl.spectra.n[flint][-1] > 1.6

"""Oracle path estimator pinned to closed forms (white furnace, uniform sky,
sun-cone irradiance, Beer-Lambert sheet) and to invariants (band-sub-domain
decomposition, pixel subsets, thread count)."""
import math

import numpy as np
import pytest

import oracle
from paper_1912_04000_gb300 import scenes


@pytest.mark.parametrize("albedo,depth", [(0.5, 5), (0.8, 3), (0.3, 1), (0.95, 8)])
def test_white_furnace_exact(albedo, depth):
    # walls emit le(1-a) and reflect a: every path returns le (1 - a^depth)
    wl = scenes.furnace_box(albedo=albedo, le=2.0, depth=depth)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    r = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, record_paths=True)
    want = 2.0 * (1.0 - albedo ** depth)
    np.testing.assert_allclose(r["path_L"], want, rtol=1e-6)  # tables are float32


def test_uniform_sky_plate():
    wl = scenes.plate_under_sky(spp=256)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    r = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, record_paths=True)
    L = r["path_L"].ravel()
    # per-path value 4 cos theta for theta in the upper hemisphere, else 0: mean 1
    assert abs(L.mean() - 1.0) < 5 * L.std() / math.sqrt(L.size)
    assert L.max() <= 4.0 + 1e-12


@pytest.mark.parametrize("half_deg,tilt_deg", [(14.3239, 0.0), (5.0, 30.0), (10.0, 60.0)])
def test_sun_cone_irradiance(half_deg, tilt_deg):
    a, s = math.radians(half_deg), math.radians(tilt_deg)
    sun = (math.sin(s), math.cos(s), 0.0)
    wl = scenes.plate_under_sky(spp=128, rho=0.6, sun_half_angle=a, sun_dir=sun, depth=2)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    r = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, record_paths=True)
    L = r["path_L"].ravel()
    want = 0.6 * math.sin(a) ** 2 * math.cos(s)
    assert abs(L.mean() - want) < 5 * L.std() / math.sqrt(L.size) + 1e-12
    assert abs(L.mean() - want) < 0.02 * want


def test_beer_lambert_sheet():
    wl = scenes.slab_view(k_glass=1e-5, spp=512)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    r = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, record_paths=True)
    c = math.cos(math.radians(30.0))
    for j, lam in enumerate((450.0, 550.0, 650.0)):
        rs, ts = oracle.slab(c, 1.5, 1e-5, lam, 0.01)
        L = r["path_L"][:, :, j].ravel()
        # each path is (R_s + T_s) with probability T_s/(R_s + T_s), else 0
        sd = math.sqrt(rs * ts / L.size)
        assert abs(L.mean() - ts) < 5 * sd
        nz = L[L != 0.0]
        np.testing.assert_allclose(nz, rs + ts, rtol=1e-3)  # 0.05 deg field of view


def test_glass_mirror_side():
    wl = scenes.slab_view(k_glass=1e-6, spp=512, sun_side="reflect")
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    r = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, record_paths=True)
    c = math.cos(math.radians(30.0))
    for j, lam in enumerate((450.0, 550.0, 650.0)):
        rs, ts = oracle.slab(c, 1.5, 1e-6, lam, 0.01)
        L = r["path_L"][:, :, j].ravel()
        assert abs(L.mean() - rs) < 5 * math.sqrt(rs * ts / L.size)


@pytest.mark.parametrize("n,k", [(0.6, 3.0), (2.5, 5.5)])
def test_conductor_mirror(n, k):
    # camera -> conductor -> sun: every path is exactly R(30 deg) L_sun
    wl = scenes.slab_view(n_glass=n, k_glass=k, spp=8, sun_side="reflect", material=scenes.CONDUCTOR)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    r = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, record_paths=True)
    R = oracle.fresnel(math.cos(math.radians(30.0)), n, k)
    np.testing.assert_allclose(r["path_L"], R, rtol=1e-5)


def test_band_subdomains_compose():
    # the spectral domain decomposition: rendering band ranges separately
    # gives bitwise the same sums as rendering all bands at once
    wl = scenes.tiny_box(width=16, height=12, spp=2)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    full = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed)["spectral_sum"]
    a = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, band_first=0, band_count=5)["spectral_sum"]
    b = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, band_first=5, band_count=11)["spectral_sum"]
    np.testing.assert_array_equal(np.concatenate([a, b], 1), full)


def test_pixel_subset_and_threads():
    wl = scenes.tiny_box(width=16, height=12, spp=2)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    full = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, n_threads=8)
    one = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, n_threads=1)
    np.testing.assert_array_equal(full["spectral_sum"], one["spectral_sum"])
    pix = np.array([5, 77, 191, 0], np.uint32)
    sub = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, pixels=pix)
    np.testing.assert_array_equal(sub["spectral_sum"], full["spectral_sum"][pix])


def test_seed_changes_image():
    wl = scenes.tiny_box(width=8, height=8, spp=2)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    a = sc.render(wl.cameras, wl.spp, wl.depth, 0)["spectral_sum"]
    b = sc.render(wl.cameras, wl.spp, wl.depth, 1)["spectral_sum"]
    assert not np.array_equal(a, b)


def test_path_weights_bounded():
    # every per-vertex weight (rho, R_s + T_s, R) is <= 1 and the NEE term is
    # at most rho L_s 2(1 - cos a): a path's radiance is bounded by depth times that
    wl = scenes.tiny_box(width=16, height=16, spp=2)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    r = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, record_paths=True)
    a = wl.spectra.sun_half_angle
    bound = wl.depth * max(2 * (1 - math.cos(a)), 1.0) * wl.spectra.sun_L.max()
    assert (r["path_L"] >= 0).all() and (r["path_L"] <= bound).all()


def test_xyz_of_flat_spectrum():
    lam = scenes.band_wavelengths(380, 780, 81)
    w = scenes.xyz_weights(lam).astype(np.float32)
    s = np.full((3, 81), 4.0)  # 4 samples of a unit spectrum
    xyz = oracle.xyz(s, 0, 4, w)
    np.testing.assert_allclose(xyz[:, 1], 1.0, rtol=1e-6)
    # partial band ranges add up to the full XYZ
    a = oracle.xyz(s[:, :40], 0, 4, w)
    b = oracle.xyz(s[:, 40:], 40, 4, w)
    np.testing.assert_allclose(a + b, xyz, rtol=1e-12)

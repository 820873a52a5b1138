"""Oracle intersection pinned to brute force, watertightness and exact hits."""
import numpy as np
import pytest

import oracle
from paper_1912_04000_gb300 import scenes


@pytest.fixture(scope="module")
def small_nave():
    wl = scenes.nave(width=8, height=8, n_bands=4, col_seg=8, col_rings=3)
    return wl


def test_bvh_equals_brute_force(small_nave):
    wl = small_nave
    rng = np.random.default_rng(11)
    o, d = scenes.random_rays(rng, wl.scene, 3000)
    o2, d2 = scenes.edge_rays(rng, wl.scene, 2000)
    o = np.concatenate([o, o2])
    d = np.concatenate([d, d2])
    bvh = oracle.OracleScene(wl.scene, wl.spectra)
    brute = oracle.OracleScene(wl.scene, wl.spectra, force_brute=True)
    t1, p1 = bvh.closest_hits(o, d)
    t2, p2 = brute.closest_hits(o, d)
    assert (p1 == p2).all()
    assert (t1 == t2).all()
    band = np.arange(o.shape[0]) % 4
    T1, g1 = bvh.shadow_transmittance(o, d, band)
    T2, g2 = brute.shadow_transmittance(o, d, band)
    assert (g1 == g2).all()
    np.testing.assert_allclose(T1, T2, rtol=1e-14)


def test_closed_box_is_watertight():
    wl = scenes.tiny_box()
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    rng = np.random.default_rng(5)
    o, d = scenes.random_rays(rng, wl.scene, 4000)
    o2, d2 = scenes.edge_rays(rng, wl.scene, 4000)
    t, p = sc.closest_hits(np.concatenate([o, o2]), np.concatenate([d, d2]))
    assert (p >= 0).all() and (t > 0).all()


def test_nave_is_closed_for_inside_rays(small_nave):
    sc = oracle.OracleScene(small_nave.scene, small_nave.spectra)
    rng = np.random.default_rng(6)
    o, d = scenes.edge_rays(rng, small_nave.scene, 3000)
    t, p = sc.closest_hits(o, d)
    assert (p >= 0).all()


def test_exact_axis_hits():
    wl = scenes.tiny_box()  # box [0,4] x [0,3] x [0,5]
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    o = np.array([[1.0, 1.0, 1.0]] * 6, np.float32)
    d = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float32)
    t, p = sc.closest_hits(o, d)
    np.testing.assert_array_equal(t, [3.0, 1.0, 2.0, 1.0, 4.0, 1.0])
    mats = wl.scene.mat_id[p]
    assert mats[4] == 1 and (np.delete(mats, 4) == 0).all()  # z = 5 wall is glass


def test_shadow_through_glass_and_blocking():
    wl = scenes.tiny_box()
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    o = np.array([[2.5, 1.2, 2.5], [2.5, 1.2, 2.5]], np.float32)
    d = np.array([[0, 0, 1], [0, 0, -1]], np.float32)
    T, g = sc.shadow_transmittance(o, d, [3, 3])
    rs, ts = oracle.slab(1.0, float(wl.spectra.n[1, 3]), float(wl.spectra.k[1, 3]),
                         float(wl.spectra.lambda_nm[3]), float(wl.scene.mat_thickness[1]))
    assert g[0] == 1 and T[0] == pytest.approx(ts, rel=1e-12)
    assert g[1] == 0xFFFFFFFF and T[1] == 0.0

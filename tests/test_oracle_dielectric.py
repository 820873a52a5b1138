"""Oracle's solid refracting glass pinned to optics it must reproduce: Snell's
law and its invariants, total internal reflection past the critical angle,
reciprocity of the Fresnel reflectance, the prism's minimum deviation, the
incoherent parallel slab (many internal reflections) and energy conservation
of a lossless dielectric inside a white furnace."""
import math

import numpy as np
import pytest

import oracle
from paper_1912_04000_gb300 import scenes


def _dirs(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@pytest.mark.parametrize("eta", [1.5, 1.33, 1.0 / 1.5, 2.4])
def test_snell_invariants(eta):
    rng = np.random.default_rng(5)
    D, N = _dirs(rng, 400), _dirs(rng, 400)
    seen = 0
    for d, n in zip(D, N):
        if d @ n > 0.0:
            n = -n  # normal faces the incident side
        ci = -d @ n
        si = math.sqrt(max(0.0, 1.0 - ci * ci))
        t = oracle.refract(d, n, eta)
        if si > eta:  # only possible when leaving the denser side
            assert t is None
            continue
        seen += 1
        assert t is not None
        assert np.linalg.norm(t) == pytest.approx(1.0, abs=1e-12)
        st = np.linalg.norm(np.cross(t, n))
        assert st == pytest.approx(si / eta, abs=1e-12)                  # Snell
        assert t @ n < 0.0                                                # crosses the surface
        assert abs(np.linalg.det(np.stack([d, n, t]))) < 1e-12          # plane of incidence
        # tangential parts point the same way
        assert (d - (d @ n) * n) @ (t - (t @ n) * n) >= -1e-15
        # light paths are reversible
        back = oracle.refract(-t, -n, 1.0 / eta)
        np.testing.assert_allclose(back, -d, atol=1e-12)
    assert seen > 100


def test_normal_incidence_and_index_matched():
    d = np.array([0.0, 0.0, -1.0])
    n = np.array([0.0, 0.0, 1.0])
    np.testing.assert_allclose(oracle.refract(d, n, 1.7), d, atol=1e-15)
    d2 = np.array([0.6, 0.0, -0.8])
    np.testing.assert_allclose(oracle.refract(d2, n, 1.0), d2, atol=1e-15)


@pytest.mark.parametrize("n", [1.33, 1.5, 1.62, 2.4])
def test_total_internal_reflection(n):
    crit = math.asin(1.0 / n)
    nrm = np.array([0.0, 1.0, 0.0])
    for th in (crit - 1e-4, crit + 1e-4, 0.5 * (crit + math.pi / 2)):
        d = np.array([math.sin(th), -math.cos(th), 0.0])
        t = oracle.refract(d, nrm, 1.0 / n)
        R = oracle.fresnel(math.cos(th), 1.0 / n, 0.0)
        if th < crit:
            assert t is not None and R < 1.0
        else:
            assert t is None
            assert R == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("n", [1.33, 1.5, 1.62])
def test_fresnel_reciprocity(n):
    # the reflectance is the same from either side of the interface at the
    # Snell-conjugate angles (Stokes relations)
    for th in np.radians([0.0, 15.0, 35.0, 55.0, 75.0, 89.0]):
        ci = math.cos(th)
        ct = math.sqrt(1.0 - (math.sin(th) / n) ** 2)
        assert oracle.fresnel(ct, 1.0 / n, 0.0) == pytest.approx(oracle.fresnel(ci, n, 0.0), rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("apex_deg", [45.0, 60.0])
def test_prism_minimum_deviation(apex_deg):
    # symmetric passage through a prism of apex A: the ray inside runs
    # parallel to the base and the deviation is 2 arcsin(n sin(A/2)) - A
    A = math.radians(apex_deg)
    lam = np.array([450.0, 550.0, 650.0])
    ns = scenes.cauchy_n(lam, 1.62, 0.012)
    devs = []
    for n in ns:
        # faces in the x-y plane: apex up, outward normals of the two faces
        n1 = np.array([-math.cos(A / 2), math.sin(A / 2), 0.0])
        n2 = np.array([math.cos(A / 2), math.sin(A / 2), 0.0])
        th1 = math.asin(n * math.sin(A / 2))
        # incoming direction at angle th1 to -n1, its tangential part up the
        # face like that of the ray inside
        c, s = math.cos(th1), math.sin(th1)
        tang = np.array([math.sin(A / 2), math.cos(A / 2), 0.0])   # along face 1, pointing up
        d = -c * n1 + s * tang
        t1 = oracle.refract(d, n1, n)
        assert abs(t1[1]) < 1e-12                                   # parallel to the base
        t2 = oracle.refract(t1, -n2, 1.0 / n)
        dev = math.acos(np.clip(d @ t2, -1.0, 1.0))
        assert dev == pytest.approx(2.0 * th1 - A, abs=1e-12)
        devs.append(dev)
    assert devs[0] > devs[1] > devs[2]                              # blue bends most


@pytest.mark.parametrize("n_glass,k_glass", [(1.5, 2e-6), (1.7, 5e-7), (1.45, 0.0)])
def test_solid_slab_is_incoherent_sheet(n_glass, k_glass):
    # entry and exit faces parallel: every transmitted path keeps its
    # direction, and summed over internal reflections the pixel's
    # expectation is the thin-sheet T_s of the same glass
    wl = scenes.solid_slab_view(n_glass=n_glass, k_glass=k_glass, spp=4096)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    r = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, record_paths=True)
    ci = math.cos(math.radians(30.0))
    ct = math.sqrt(1.0 - (1.0 - ci * ci) / n_glass ** 2)
    for j, lam in enumerate((450.0, 550.0, 650.0)):
        rs, ts = oracle.slab(ci, n_glass, k_glass, lam, 0.01)
        L = r["path_L"][:, :, j].ravel()
        sd = L.std() / math.sqrt(L.size)
        assert abs(L.mean() - ts) < 5 * sd + 1e-9
        # a transmitted path crossed the slab 2j+1 times: a^(2j+1)
        a = math.exp(-4 * math.pi * k_glass / (lam * 1e-9) * 0.01 / ct)
        nz = L[L != 0.0]
        odd = np.round(np.log(nz) / math.log(a)) if k_glass > 0 else np.ones_like(nz)
        if k_glass > 0:
            assert np.all(odd % 2 == 1)
            np.testing.assert_allclose(nz, a ** odd, rtol=2e-3)  # 0.05 deg field of view
        else:
            np.testing.assert_allclose(nz, 1.0, rtol=1e-6)
    # the reflected share R_s never reaches the sun behind the slab
    assert r["path_L"].max() <= 1.0 + 1e-6


@pytest.mark.parametrize("albedo", [0.3, 0.5])
def test_lossless_dielectric_in_furnace(albedo):
    # walls emit le (1 - a), reflect a; the k = 0 cube only redirects: a path
    # with m wall vertices returns le (1 - a^m) <= le, and m is large at depth 64
    wl = scenes.dielectric_furnace(albedo=albedo, le=2.0)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    r = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, record_paths=True)
    L = r["path_L"].ravel()
    assert L.max() <= 2.0 * (1.0 + 1e-6)
    assert L.min() >= 2.0 * (1.0 - albedo) * (1.0 - 1e-6)   # the first wall vertex
    assert L.mean() == pytest.approx(2.0, rel=1e-4)


def test_absorbing_dielectric_in_furnace_loses_energy():
    wl = scenes.dielectric_furnace(albedo=0.3, le=2.0)
    wl.spectra.k[1] = 1e-5   # alpha ~ 200 /m across a 0.55 m cube
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    L = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, record_paths=True)["path_L"].ravel()
    assert L.mean() < 2.0 * 0.99 and L.max() <= 2.0 * (1.0 + 1e-6)


def test_prism_room_renders():
    wl = scenes.prism_room(width=24, height=18, n_bands=4, spp=2)
    assert wl.scene.mat_type[2] == scenes.DIELECTRIC
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    r = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, record_paths=True)
    L = r["path_L"]
    assert np.all(np.isfinite(L)) and np.all(L >= 0.0)
    assert L.max() > 0.0


def test_solids_have_outward_normals():
    for wl in (scenes.prism_room(), scenes.solid_slab_view(), scenes.dielectric_furnace()):
        sc = wl.scene
        dm = [i for i, t in enumerate(sc.mat_type) if t == scenes.DIELECTRIC]
        sel = np.isin(sc.mat_id, dm)
        tri = sc.verts[sc.tris[sel]].astype(np.float64)
        ctr = tri.reshape(-1, 3).mean(0)
        nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
        assert np.all(np.einsum("ij,ij->i", nrm, tri.mean(1) - ctr) > 0.0)
        # closed: the divergence theorem gives the volume from either winding
        vol = np.einsum("ij,ij->i", tri[:, 0], np.cross(tri[:, 1], tri[:, 2])).sum() / 6.0
        assert vol > 0.0

"""Photon mapping on the GPU (rt_photon_records, rt_render_photons) against
the oracle's photon mapping: photon records slot by slot (the box, the
dispersive prism, the mirror caustic), rendered images, the mirror
caustic's closed form, band chunking, determinism and argument checks."""
import math

import numpy as np
import pytest

import oracle
from paper_1912_04000_gb300 import scenes
from paper_1912_04000_gb300._native import RtError

from parity import xyz_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1912_04000_gb300.renderer import Renderer
    return Renderer(0)


def _photon_parity(g, o, what):
    """Photon-mapping images: a photon whose path diverges between FP32 and
    FP64 (a refraction, total internal reflection or edge decision) moves its
    whole flux, shifting every pixel whose gathers reach either place; the
    pixel bar is 99.5% of pixels within 1e-4, the aggregate bar unchanged
    and taken over all pixels."""
    m = xyz_parity(g, o)
    assert m["frac_ok"] >= 0.995, f"{what}: {m}"
    assert m["mean_rel_all"] <= 1e-5, f"{what}: {m}"
    return m


def _diag(wl):
    v = wl.scene.verts.astype(np.float64)
    return float(np.linalg.norm(v.max(0) - v.min(0)))


@pytest.mark.parametrize("name", ["tiny_box", "prism_room", "mirror_caustic"])
def test_photon_records(R, name):
    wl = {"tiny_box": lambda: scenes.tiny_box(n_bands=4),
          "prism_room": lambda: scenes.prism_room(n_bands=4),
          "mirror_caustic": lambda: scenes.mirror_caustic()}[name]()
    R.load(wl)
    N, depth = 1 << 13, 4
    rec, cls = (x.cpu().numpy() for x in R.photon_records(N, depth, seed=5))
    pos, ocls = oracle.OracleScene(wl.scene, wl.spectra).photon_records(N, depth, seed=5)
    same = (cls == ocls).all(-1)                       # whole photon paths with the same classes
    print(name, "photons with identical stores", same.mean(), "classes", np.bincount(ocls.ravel(), minlength=4))
    assert same.mean() >= 0.99
    st = (ocls > 0) & same[..., None]
    np.testing.assert_allclose(rec[..., :3][st], pos[..., :3][st], rtol=0, atol=2e-5 * _diag(wl))
    np.testing.assert_allclose(rec[..., 3][st], pos[..., 3][st], rtol=2e-5)


@pytest.mark.parametrize("name", ["tiny_box", "prism_room", "mirror_caustic"])
def test_photon_render(R, name):
    if name == "tiny_box":
        wl, kw = scenes.tiny_box(width=64, height=64, n_bands=4, spp=2, depth=6), dict(r_global=0.15)
    elif name == "prism_room":
        wl, kw = scenes.prism_room(width=64, height=48, n_bands=4, spp=2), dict(r_caustic=0.04, r_global=0.15)
    else:
        wl, kw = scenes.mirror_caustic(width=32, height=32, spp=2), dict(r_caustic=0.1, r_global=0.3)
    R.load(wl)
    N, pd = 1 << 15, 4
    out = R.render_photons(wl.cameras, wl.spp, wl.depth, wl.seed, n_photons=N, photon_depth=pd, **kw)
    o = oracle.OracleScene(wl.scene, wl.spectra).render_photons(
        wl.cameras, wl.spp, wl.depth, wl.seed, n_photons=N, photon_depth=pd,
        r_caustic=kw.get("r_caustic", 0.005 * _diag(wl)), r_global=kw.get("r_global", 0.02 * _diag(wl)))
    m = xyz_parity(out["xyz"].cpu().numpy(), o["xyz"])
    print(name, "photon-mapping parity", m, out["stats"]["ms_stage"][:3])
    _photon_parity(out["xyz"].cpu().numpy(), o["xyz"], name)


def test_mirror_caustic_closed_form(R):
    e, a, rho = math.radians(45.0), 0.02, 0.8
    wl = scenes.mirror_caustic(elevation_deg=45.0, sun_half_angle=a, rho=rho, width=4, height=4, spp=8)
    R.load(wl)
    N, r = 1 << 22, 0.15
    got = R.render_photons(wl.cameras, wl.spp, wl.depth, wl.seed, n_photons=N, photon_depth=3, r_caustic=r,
                           r_global=0.3, xyz_mode=2)["spectral"].cpu().numpy()[:, 0] / wl.spp
    Rm = oracle.fresnel(math.cos(e), 0.3, 3.0)
    E = math.pi * math.sin(a) ** 2 * math.sin(e)
    want = rho / math.pi * E * (1.0 + Rm)
    # photons in a gather disk: the mirror intercepts cos(e) m^2 of the
    # emission disk (radius R_d) and spreads it over a 1 / tan(e) m^2 patch;
    # the Epanechnikov weights count as 3/4 of that many photons
    v = wl.scene.verts.astype(np.float64)
    Rb = 0.5 * np.linalg.norm(v.max(0) - v.min(0))
    Rd = Rb * (math.tan(a) + 1.0 / math.cos(a))
    n_in = 0.75 * N * math.cos(e) / (math.pi * Rd * Rd) * math.pi * r * r * math.tan(e)
    tol = 5.0 * rho / math.pi * E * Rm / math.sqrt(n_in) + 0.02 * want
    assert np.all(np.abs(got - want) < tol), (got, want, tol)


def test_chunks_hash_sizes_and_determinism(R):
    # 40 bands: log2_cells 20 splits them into chunks of 32 and 8, 12 keeps
    # one chunk; the hash size changes only the summation order.  3 spp: the
    # small chunk's camera waves hold one sample each
    wl = scenes.tiny_box(width=32, height=32, n_bands=40, spp=3, depth=5)
    R.load(wl)
    kw = dict(n_photons=4096, photon_depth=4, r_global=0.15, xyz_mode=2)
    a = R.render_photons(wl.cameras, 3, 5, 3, log2_cells=20, **kw)
    b = R.render_photons(wl.cameras, 3, 5, 3, log2_cells=12, **kw)
    assert a["stats"]["waves"] == 2 and b["stats"]["waves"] == 1
    sa, sb = a["spectral"].cpu().numpy(), b["spectral"].cpu().numpy()
    np.testing.assert_allclose(sa, sb, rtol=1e-5, atol=1e-12)
    c = R.render_photons(wl.cameras, 3, 5, 3, log2_cells=20, **kw)["spectral"].cpu().numpy()
    assert np.array_equal(sa, c)
    o = oracle.OracleScene(wl.scene, wl.spectra).render_photons(
        wl.cameras, 3, 5, 3, n_photons=4096, photon_depth=4, r_caustic=0.005 * _diag(wl), r_global=0.15)
    _photon_parity(a["xyz"].cpu().numpy(), o["xyz"], "40 bands in two chunks")


def test_arguments_checked(R):
    wl = scenes.tiny_box(width=8, height=8, n_bands=2, spp=1)
    R.load(wl)
    with pytest.raises(RtError):
        R.render_photons(wl.cameras, 1, 4, 0, n_photons=1 << 23, photon_depth=4)
    with pytest.raises(RtError):
        R.render_photons(wl.cameras, 1, 4, 0, log2_cells=30)
    with pytest.raises(RtError):
        R.render_photons(wl.cameras, 1, 4, 0, emission=2)
    with pytest.raises(RtError):
        R.photon_records(64, 2, seed=0, emission=2)
    wide = scenes.plate_under_sky()  # half angle pi: no emission disk
    R.load(wide)
    with pytest.raises(RtError):
        R.render_photons(wide.cameras, 1, 2, 0)


@pytest.mark.parametrize("name", ["tiny_box", "prism_room"])
def test_portal_emission_records_and_image(R, name):
    wl = scenes.tiny_box(width=48, height=48, n_bands=4, spp=2, depth=6) if name == "tiny_box" else \
        scenes.prism_room(width=48, height=36, n_bands=4, spp=2)
    R.load(wl)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    N, depth = 1 << 13, 4
    rec, cls = (x.cpu().numpy() for x in R.photon_records(N, depth, seed=7, emission=1))
    pos, ocls = sc.photon_records(N, depth, seed=7, emission=1)
    same = (cls == ocls).all(-1)
    print(name, "portal photons with identical stores", same.mean())
    assert same.mean() >= 0.99
    st = (ocls > 0) & same[..., None]
    np.testing.assert_allclose(rec[..., :3][st], pos[..., :3][st], rtol=0, atol=2e-5 * _diag(wl))
    np.testing.assert_allclose(rec[..., 3][st], pos[..., 3][st], rtol=2e-5)
    kw = dict(n_photons=1 << 15, photon_depth=4, r_caustic=0.04, r_global=0.15)
    out = R.render_photons(wl.cameras, wl.spp, wl.depth, wl.seed, emission=1, **kw)
    o = sc.render_photons(wl.cameras, wl.spp, wl.depth, wl.seed, emission=1, **kw)
    print(name, "portal photon-mapping parity", xyz_parity(out["xyz"].cpu().numpy(), o["xyz"]))
    _photon_parity(out["xyz"].cpu().numpy(), o["xyz"], name + " portals")


def test_portal_emission_needs_glass(R):
    wl = scenes.mirror_caustic()
    R.load(wl)
    with pytest.raises(RtError):
        R.render_photons(wl.cameras, 1, 3, 0, emission=1)

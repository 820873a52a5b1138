"""Solid refracting glass on the GPU (Snell with n(lambda), Fresnel of the
relative index, Beer-Lambert over the distance crossed inside) against the
oracle: a dispersive prism in the sunlit box room pixel by pixel and path by
path, the parallel slab against its closed form, a lossless solid inside the
white furnace, and the device-built tree and the guided tracer on the prism."""
import math

import numpy as np
import pytest

import oracle
from paper_1912_04000_gb300 import scenes

from parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1912_04000_gb300.renderer import Renderer
    return Renderer(0)


def _oracle(wl, **kw):
    return oracle.OracleScene(wl.scene, wl.spectra).render(wl.cameras, wl.spp, wl.depth, wl.seed, **kw)


def test_prism_room_full_image(R):
    """96 x 72, 16 bands, 4 spp, depth 8: every pixel against the oracle."""
    wl = scenes.prism_room()
    R.load(wl)
    out = R.render(wl.cameras, wl.spp, wl.depth, wl.seed)
    o = _oracle(wl)
    m = assert_parity(out["xyz"].cpu().numpy(), o["xyz"], "prism room")
    print("prism room parity", m)
    gs = out["spectral"].cpu().numpy()
    rel = np.abs(gs - o["spectral_sum"]).sum() / np.abs(o["spectral_sum"]).sum()
    assert rel < 1e-5


def test_prism_room_paths(R):
    """Per-path radiance and vertex signatures on pixels that look into the
    prism (refraction, internal reflection, absorption on the way)."""
    wl = scenes.prism_room(width=48, height=36, spp=4)
    R.load(wl)
    o_all = _oracle(wl)
    # pixels with the most spectral spread between bands: the dispersive ones
    sp = o_all["spectral_sum"]
    spread = sp.std(1) / np.maximum(sp.mean(1), 1e-30)
    pix = np.argsort(spread)[-48:].astype(np.int64)
    out = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, probe_pixels=pix, xyz_mode=2)
    o = _oracle(wl, pixels=pix.astype(np.uint32), record_paths=True)
    gL = out["probe_L"].cpu().numpy()
    gS = out["probe_sig"].cpu().numpy().view(np.uint32)
    same = gS == o["path_sig"]
    print("prism paths: same vertex sequence", same.mean())
    assert same.mean() >= 0.99
    np.testing.assert_allclose(gL[same], o["path_L"][same], rtol=5e-5, atol=1e-9)


@pytest.mark.parametrize("n_glass,k_glass", [(1.5, 2e-6), (1.7, 5e-7)])
def test_solid_slab_closed_form(R, n_glass, k_glass):
    wl = scenes.solid_slab_view(n_glass=n_glass, k_glass=k_glass, spp=8192)
    R.load(wl)
    pix = np.arange(4, dtype=np.int64)
    out = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, probe_pixels=pix, xyz_mode=2)
    L = out["probe_L"].cpu().numpy()
    ci = math.cos(math.radians(30.0))
    for j, lam in enumerate((450.0, 550.0, 650.0)):
        rs, ts = oracle.slab(ci, n_glass, k_glass, lam, 0.01)
        v = L[:, :, j].ravel()
        assert abs(v.mean() - ts) < 5 * v.std() / math.sqrt(v.size) + 1e-9
    o = _oracle(wl)
    np.testing.assert_allclose(out["spectral"].cpu().numpy(), o["spectral_sum"], rtol=2e-3)


def test_lossless_dielectric_furnace(R):
    wl = scenes.dielectric_furnace(albedo=0.3, le=2.0, width=24, height=20, spp=8)
    R.load(wl)
    out = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)
    s = out["spectral"].cpu().numpy() / wl.spp
    assert s.max() <= 2.0 * (1.0 + 1e-6)
    assert s.mean() == pytest.approx(2.0, rel=1e-4)
    o = _oracle(wl)
    assert_parity(out["xyz"].cpu().numpy(), o["xyz"], "dielectric furnace")


def test_absorption_table_is_per_metre(R):
    """The thickness entry of a solid is ignored: the attenuation comes from
    the distance the path crosses inside."""
    wl = scenes.solid_slab_view(n_glass=1.5, k_glass=2e-6, spp=64)
    R.load(wl)
    a = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)["spectral"].cpu().numpy()
    wl.scene.mat_thickness[:] = 0.5
    R.load(wl)
    b = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)["spectral"].cpu().numpy()
    assert np.array_equal(a, b)


def test_prism_room_device_build(R):
    wl = scenes.prism_room(width=64, height=48, n_bands=8, spp=2)
    R.load(wl, builder=0)
    a = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)["spectral"].cpu().numpy()
    R.load(wl, builder=1)
    b = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)["spectral"].cpu().numpy()
    np.testing.assert_allclose(b, a, rtol=1e-5, atol=1e-12)


def test_prism_room_guided_unbiased(R):
    wl = scenes.prism_room(width=48, height=36, n_bands=4, spp=32)
    R.load(wl)
    R.guide_init(seed=5, log2_table=14, guide_depth=3)
    R.render(wl.cameras, 8, wl.depth, 1234, guided=True, guide_collect=1, guide_train_steps=8, xyz=False)
    plain = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz=False)["spectral"].cpu().numpy() / wl.spp
    guided = R.render(wl.cameras, wl.spp, wl.depth, wl.seed + 99, guided=True, xyz=False)["spectral"].cpu().numpy()
    guided /= wl.spp
    assert np.isfinite(guided).all() and (guided >= 0).all()
    d = (guided - plain).ravel()
    assert abs(d.mean()) / (d.std() / np.sqrt(d.size)) < 5.0


def _project(cam, X):
    """Pixel (x, y) of point X for the pinhole camera (vertical field of view,
    y growing downwards)."""
    pos = np.asarray(cam.pos, np.float64)
    f = np.asarray(cam.look, np.float64) - pos
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(cam.up, np.float64))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    v = np.asarray(X, np.float64) - pos
    th = math.tan(math.radians(cam.vfov_deg) / 2.0)
    asp = cam.width / cam.height
    xc, yc = (v @ r) / (v @ f), (v @ u) / (v @ f)
    return int((xc / (th * asp) + 1.0) / 2.0 * cam.width), int((1.0 - yc / th) / 2.0 * cam.height)


def test_crystal_nave_sampled_pixels(R):
    """The nave with eight solid glass objects (spheres and dispersive
    prisms) at its full size, 1024 x 768, 81 bands, 16 spp, depth 8; pixels
    that look at the solids are re-rendered path by path by the oracle."""
    wl = scenes.crystal_nave()
    cam = wl.cameras[0]
    pix = []
    for i in range(8):
        xc = 15.0 + 50.0 * i / 7
        y = 1.2 if i % 2 == 0 else 0.8
        px, py = _project(cam, (xc, y, 10.0))
        for dx, dy in ((0, 0), (3, 1), (-2, 2), (1, -3), (-4, -1), (2, 4)):
            pix.append((py + dy) * cam.width + px + dx)
    pix = np.array(sorted(set(pix)), np.int64)
    R.load(wl)
    out = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, probe_pixels=pix, xyz_mode=2)
    o = _oracle(wl, pixels=pix.astype(np.uint32), record_paths=True)
    gS = out["probe_sig"].cpu().numpy().view(np.uint32)
    gL = out["probe_L"].cpu().numpy()
    same = gS == o["path_sig"]
    print("crystal nave: paths with identical event signatures", same.mean())
    assert same.mean() >= 0.99
    np.testing.assert_allclose(gL[same], o["path_L"][same], rtol=1e-4, atol=1e-7)
    clean = same.reshape(len(pix), -1).all(1)
    assert clean.mean() > 0.5
    assert_parity(out["xyz"].cpu().numpy()[pix][clean], o["xyz"][clean], "crystal nave clean pixels")

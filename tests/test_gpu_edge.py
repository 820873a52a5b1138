"""Edge cases of the render call against the CPU FP64 oracle: the smallest
image (one pixel, one band, one vertex), a ragged image with the last bands
of the table, the deepest paths the call takes (depth 64), views in which
every camera ray escapes (closed form: a uniform unit sky gives exactly 1
per sample), a scene of one triangle, and the largest batch of views (64
cameras of uneven sizes).  Empty inputs (no cameras, spp 0, depth 0, an
empty band range) are refused with RT_ERR_ARG: test_gpu_errors."""
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


def _both(R, wl, cameras, spp, depth, seed, band_first=0, band_count=None):
    if band_count is None:
        band_count = wl.spectra.n_bands - band_first
    R.load(wl)
    g = R.render(cameras, spp, depth, seed, band_first=band_first, band_count=band_count, xyz_mode=2)
    o = oracle.OracleScene(wl.scene, wl.spectra).render(cameras, spp, depth, seed, band_first=band_first,
                                                        band_count=band_count)
    return g["spectral"].cpu().numpy(), g["xyz"].cpu().numpy(), o


def _spectral_close(gs, o, what):
    os_ = o["spectral_sum"]
    assert gs.shape == os_.shape, what
    den = np.abs(os_).sum()
    rel = np.abs(gs - os_).sum() / den if den > 0 else np.abs(gs).sum()
    assert rel <= 1e-5, f"{what}: aggregate spectral error {rel}"


def test_one_pixel_one_band_one_vertex(R):
    """1 x 1 image, band 7 of 16 alone, depth 1 (the camera ray's hit and its
    sun ray only), 5 samples."""
    wl = scenes.tiny_box(width=1, height=1, n_bands=16, spp=5, depth=1)
    gs, gx, o = _both(R, wl, wl.cameras, 5, 1, 3, band_first=7, band_count=1)
    assert gs.shape == (1, 1)
    assert o["spectral_sum"][0, 0] > 0.0  # the pixel sees sunlit stone
    _spectral_close(gs, o, "one pixel")
    assert_parity(gx, o["xyz"], "one pixel")


def test_ragged_image_last_bands(R):
    """37 x 23 pixels (no multiple of any tile or warp), bands 13-15 of 16,
    depth 3, 3 samples: every pixel."""
    wl = scenes.tiny_box(width=37, height=23, n_bands=16, spp=3, depth=3)
    gs, gx, o = _both(R, wl, wl.cameras, 3, 3, 11, band_first=13, band_count=3)
    assert gs.shape == (37 * 23, 3)
    _spectral_close(gs, o, "ragged")
    assert_parity(gx, o["xyz"], "ragged")


def test_maximum_depth(R):
    """Depth 64, the largest the call takes, in the glass box: every pixel."""
    wl = scenes.tiny_box(width=24, height=16, n_bands=4, spp=2, depth=64)
    gs, gx, o = _both(R, wl, wl.cameras, 2, 64, 5)
    _spectral_close(gs, o, "depth 64")
    assert_parity(gx, o["xyz"], "depth 64")


@pytest.mark.parametrize("half_angle", [np.pi, 0.1])
def test_every_camera_ray_escapes(R, half_angle):
    """A camera above the plate looking up: every camera ray leaves the
    scene.  Under a uniform unit sky (half angle pi) every path carries
    exactly 1; under a narrow cone only the pixels whose rays fall inside it
    see the sun, as in the oracle."""
    wl = scenes.plate_under_sky(n_bands=3, width=9, height=7, spp=4, depth=2, sun_half_angle=half_angle,
                                sun_dir=(0.0, 1.0, 0.0))
    up = scenes.Camera((0.0, 2.0, 0.0), (0.0, 5.0, 0.3), (0.0, 0.0, 1.0), 40.0, 9, 7)
    gs, gx, o = _both(R, wl, [up], 4, 2, 1)
    if half_angle == np.pi:
        np.testing.assert_array_equal(gs, np.full_like(gs, 4.0))
        np.testing.assert_array_equal(o["spectral_sum"], np.full_like(gs, 4.0))
    else:
        assert 0 < np.count_nonzero(o["spectral_sum"]) < gs.size
        np.testing.assert_array_equal(gs > 0, o["spectral_sum"] > 0)
        _spectral_close(gs, o, "narrow sun")


def test_single_triangle_scene(R):
    """One Lambertian triangle in front of the camera, the sun behind the
    camera: hits, misses and the sun rays of a one-leaf tree."""
    mb = scenes.MeshBuilder()
    mb.tri((-1.0, -1.0, 3.0), (1.5, -0.8, 3.2), (0.0, 1.2, 2.8), 0)
    scene = mb.build([scenes.LAMBERT], [0.0])
    lam = scenes.band_wavelengths(420.0, 680.0, 5)
    n = np.ones((1, 5))
    k = np.zeros((1, 5))
    rho = np.full((1, 5), 0.6)
    le = np.zeros((1, 5))
    spec = scenes._spectra(lam, scenes.sun_spectrum(lam), scenes.sun_direction(50.0, 10.0), 0.05, n, k, rho, le)
    cam = scenes.Camera((0.0, 0.0, 0.0), (0.0, 0.0, 3.0), (0.0, 1.0, 0.0), 70.0, 31, 27)
    wl = scenes.Workload("one_triangle", scene, spec, [cam], 3, 4, 2)
    gs, gx, o = _both(R, wl, [cam], 3, 4, 2)
    lit = o["spectral_sum"].sum(1) > 0
    assert 0.1 < lit.mean() < 0.9  # part of the view sees the lit triangle, the rest escapes
    _spectral_close(gs, o, "one triangle")
    assert_parity(gx, o["xyz"], "one triangle")


def test_sixty_four_uneven_views(R):
    """The largest batch the call takes: 64 cameras of sizes 1 x 1 up to
    9 x 5 at different positions, 4 bands, 2 samples, depth 4: every pixel
    of every view."""
    base = scenes.tiny_box(n_bands=4)
    rng = np.random.default_rng(64)
    cams = []
    for i in range(64):
        pos = (float(rng.uniform(0.5, 3.5)), float(rng.uniform(0.5, 2.5)), float(rng.uniform(0.3, 2.0)))
        look = (float(rng.uniform(0.5, 3.5)), float(rng.uniform(0.5, 2.5)), 5.0)
        cams.append(scenes.Camera(pos, look, (0.0, 1.0, 0.0), float(rng.uniform(30.0, 90.0)), 1 + i % 9,
                                  1 + (i * 7) % 5))
    gs, gx, o = _both(R, base, cams, 2, 4, 9)
    assert gs.shape[0] == sum(c.width * c.height for c in cams)
    _spectral_close(gs, o, "64 views")
    assert_parity(gx, o["xyz"], "64 views")

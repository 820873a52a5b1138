"""Oracle pins for the camera model, the cosine-weighted continuation and the
colour contraction, each against a value fixed outside the oracle: the
pinhole projection the header defines, the form factor of a square emitter,
and the CIE 1931 chromaticities of the spectral locus."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1912_04000_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def square_form_factor(a, h):
    """Form factor from a differential area to a parallel coaxial square of
    half side a at height h: four corner rectangles a x a, each by the
    closed form for a rectangle whose corner lies above the element,
    F = (1 / 2 pi) [X / sqrt(1 + X^2) atan(Y / sqrt(1 + X^2))
                    + Y / sqrt(1 + Y^2) atan(X / sqrt(1 + Y^2))], X = Y = a / h."""
    X = Y = a / h
    f = (X / math.sqrt(1 + X * X) * math.atan(Y / math.sqrt(1 + X * X))
         + Y / math.sqrt(1 + Y * Y) * math.atan(X / math.sqrt(1 + Y * Y))) / (2 * math.pi)
    return 4.0 * f


def test_square_form_factor_closed_form():
    # the closed form against the defining double integral (h^2 / pi r^4 over the square)
    from scipy import integrate
    a, h = 1.0, 2.0
    val, _ = integrate.dblquad(lambda z, x: h * h / (math.pi * (x * x + z * z + h * h) ** 2), -a, a, -a, a)
    assert square_form_factor(a, h) == pytest.approx(val, rel=1e-9)


@pytest.mark.parametrize("half,height", [(1.0, 2.0), (2.0, 1.0)])
def test_cosine_continuation_form_factor(half, height):
    """Section 4, Eq. 2 at a Lambertian floor lit only by a square emitter:
    the cosine-sampled continuation hits the emitter with probability F, so
    the pixel's expectation is rho le F.  A continuation drawn from another
    distribution but still weighted rho (uniform cos theta: 0.128 instead of
    0.239 for the first case) fails by tens of standard errors."""
    wl = scenes.emitter_over_plate(half=half, height=height, rho=0.8, le=1.5)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    r = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, record_paths=True)
    L = r["path_L"].ravel()
    want = 0.8 * 1.5 * square_form_factor(half, height)
    se = L.std() / math.sqrt(L.size)
    assert abs(L.mean() - want) < 5 * se, (L.mean(), want, se)
    # every path is 0 or rho le: the continuation weight is exactly rho
    assert np.all(np.isclose(L, 0.0) | np.isclose(L, 1.2, rtol=1e-6))


def test_camera_marker_pixel():
    """A marker placed where a pinhole camera (vertical field of view,
    aspect W/H, x to the right = f x up, y downwards) shows pixel (6, 1)
    appears only in that pixel, covering (marker / pixel footprint) of it."""
    wl = scenes.camera_marker(target_px=(6, 1), spp=4096)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    r = sc.render(wl.cameras, wl.spp, wl.depth, wl.seed, record_paths=True)
    mean = r["spectral_sum"][:, 0] / wl.spp
    img = mean.reshape(6, 8)
    assert img[1, 6] > 0.0
    img[1, 6] = 0.0
    assert np.all(img == 0.0)
    pixel_side = 2.0 * math.tan(math.radians(30.0)) / 6 * 10.0
    frac = (0.6 / pixel_side) ** 2
    L = r["path_L"][1 * 8 + 6].ravel()
    assert abs(L.mean() - frac) < 5 * math.sqrt(frac * (1 - frac) / L.size)


def test_camera_ray_geometry():
    """Primary rays of a camera with an arbitrary pose: every ray starts at
    the camera, is a unit vector, and the ray of pixel (x, y) with jitter
    (u0, u1) (the Philox draws, pinned elsewhere) meets the plane one unit
    along the view axis at right = (2 (x + u0) / W - 1) tan(v/2) W/H and
    up = (1 - 2 (y + u1) / H) tan(v/2), right = f x up_world normalised."""
    cam = scenes.Camera((1.0, 2.0, -3.0), (4.0, 1.0, 5.0), (0.1, 1.0, 0.2), 50.0, 40, 30)
    pix = np.arange(40 * 30, dtype=np.uint32)
    o, d = oracle.camera_rays([cam], pix, sample=3, band=2, seed=5)
    np.testing.assert_allclose(o, np.broadcast_to(np.float32([1.0, 2.0, -3.0]), o.shape), rtol=0, atol=0)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, rtol=1e-12)
    f = np.array([3.0, -1.0, 8.0])
    f /= np.linalg.norm(f)
    right = np.cross(f, np.float32([0.1, 1.0, 0.2]).astype(np.float64))
    right /= np.linalg.norm(right)
    up = np.cross(right, f)
    ctr = np.stack([pix, np.full_like(pix, 3), np.full_like(pix, 2), np.zeros_like(pix)], 1)
    u = oracle.philox_batch(5, 0, ctr)
    u0 = (u[:, 0] >> 8) / 2.0 ** 24
    u1 = (u[:, 1] >> 8) / 2.0 ** 24
    x, y = pix % 40, pix // 40
    th = math.tan(math.radians(50.0) / 2)
    p = d / (d @ f)[:, None]
    np.testing.assert_allclose(p @ right, (2 * (x + u0) / 40 - 1) * th * 40 / 30, atol=1e-6)
    np.testing.assert_allclose(p @ up, (1 - 2 * (y + u1) / 30) * th, atol=1e-6)
    # the top row looks up, the left column looks left: y grows downwards, x to the right
    assert np.all(d[y == 0] @ up > 0) and np.all(d[x == 0] @ right < 0)


def _locus():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "cie1931_spectral_locus.txt")) if not l.startswith("#")]
    return [(float(a), float(b), float(c)) for a, b, c in rows]


def test_xyz_equal_energy_white():
    """A flat spectrum: Y = 1, X and Z equal the colour-matching integrals
    over 380-780 nm relative to that of y-bar (adaptive quadrature, not the
    band sum), and the chromaticity is that of illuminant E, (1/3, 1/3)."""
    from scipy import integrate
    lam = scenes.band_wavelengths(380, 780, 81)
    w = scenes.xyz_weights(lam).astype(np.float32)
    X, Y, Z = oracle.xyz(np.ones((1, 81)), 0, 1, w)[0]
    assert Y == pytest.approx(1.0, rel=1e-6)
    I = [integrate.quad(lambda l, c=c: scenes.cie_cmf_fit(np.array([l]))[0][c], 380, 780, limit=200)[0]
         for c in range(3)]
    assert X == pytest.approx(I[0] / I[1], rel=2e-4)
    assert Z == pytest.approx(I[2] / I[1], rel=2e-4)
    s = X + Y + Z
    assert abs(X / s - 1 / 3) < 3e-3 and abs(Y / s - 1 / 3) < 3e-3


def test_xyz_spectral_locus():
    """One band lit at a time: the chromaticity of the oracle's XYZ lies on
    the CIE 1931 spectral locus (to the accuracy of the analytic fit), which
    fixes the order of the X, Y and Z columns."""
    lam = scenes.band_wavelengths(380, 780, 81)
    w = scenes.xyz_weights(lam).astype(np.float32)
    for l, x_ref, y_ref in _locus():
        j = int(np.argmin(np.abs(lam - l)))
        assert lam[j] == l
        e = np.zeros((1, 81))
        e[0, j] = 7.0
        X, Y, Z = oracle.xyz(e, 0, 7, w)[0]
        s = X + Y + Z
        assert abs(X / s - x_ref) < 0.01 and abs(Y / s - y_ref) < 0.01, (l, X / s, Y / s)

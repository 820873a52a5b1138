"""Oracle optics pinned to closed forms (section 3, Eq. 1: complex index
n + ik; thin glass with Beer-Lambert absorption)."""
import math

import numpy as np
import pytest

import oracle


def _dielectric_R(cos_i, n):
    # textbook real-index Fresnel with Snell's law (Hecht, Optics, ch. 4)
    sin_t = math.sqrt(1 - cos_i * cos_i) / n
    cos_t = math.sqrt(1 - sin_t * sin_t)
    rs = (cos_i - n * cos_t) / (cos_i + n * cos_t)
    rp = (n * cos_i - cos_t) / (n * cos_i + cos_t)
    return 0.5 * (rs * rs + rp * rp), rs * rs, rp * rp


@pytest.mark.parametrize("n,k", [(1.5, 0.0), (1.52, 1e-6), (1.6, 1e-5), (0.6, 3.0), (2.5, 5.5), (1.0, 2.0)])
def test_normal_incidence_closed_form(n, k):
    want = ((n - 1) ** 2 + k * k) / ((n + 1) ** 2 + k * k)
    assert oracle.fresnel(1.0, n, k) == pytest.approx(want, rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("theta_deg", [0, 10, 30, 45, 56.3, 70, 85, 89.5])
@pytest.mark.parametrize("n", [1.33, 1.5, 1.6])
def test_zero_k_is_dielectric(theta_deg, n):
    c = math.cos(math.radians(theta_deg))
    want, _, _ = _dielectric_R(c, n)
    assert oracle.fresnel(c, n, 0.0) == pytest.approx(want, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("n", [1.45, 1.5, 1.6])
def test_brewster(n):
    # r_p vanishes at tan(theta_B) = n, so R = |r_s|^2 / 2 there
    th = math.atan(n)
    c = math.cos(th)
    _, rs2, rp2 = _dielectric_R(c, n)
    assert rp2 < 1e-25
    assert oracle.fresnel(c, n, 0.0) == pytest.approx(0.5 * rs2, rel=1e-12)
    # away from Brewster the p part is not zero
    for d in (-0.2, 0.2):
        _, rs2d, _ = _dielectric_R(math.cos(th + d), n)
        assert oracle.fresnel(math.cos(th + d), n, 0.0) > 0.5 * rs2d * (1 + 1e-6)


@pytest.mark.parametrize("n,k", [(1.5, 0.0), (1.5, 1e-6), (0.5, 2.0), (3.0, 6.0)])
def test_grazing_limit(n, k):
    assert oracle.fresnel(1e-7, n, k) == pytest.approx(1.0, abs=1e-5)
    vals = [oracle.fresnel(math.cos(math.radians(t)), n, k) for t in range(0, 90, 5)]
    assert all(0.0 <= v <= 1.0 for v in vals)


@pytest.mark.parametrize("theta_deg", [0, 20, 45, 60, 80])
@pytest.mark.parametrize("n", [1.45, 1.5, 1.6])
def test_lossless_plate(theta_deg, n):
    # k = 0: all light is reflected or transmitted; incoherent plate gives
    # R_s = 2R/(1+R), T_s = (1-R)/(1+R)
    c = math.cos(math.radians(theta_deg))
    R = oracle.fresnel(c, n, 0.0)
    rs, ts = oracle.slab(c, n, 0.0, 550.0, 0.01)
    assert rs + ts == pytest.approx(1.0, abs=1e-14)
    assert rs == pytest.approx(2 * R / (1 + R), rel=1e-13)
    assert ts == pytest.approx((1 - R) / (1 + R), rel=1e-13)


@pytest.mark.parametrize("theta_deg", [0, 30, 60])
@pytest.mark.parametrize("k,lam", [(1e-7, 400.0), (1e-6, 550.0), (1e-5, 700.0)])
def test_beer_lambert_limit(theta_deg, k, lam):
    # index-matched sheet (n = 1, tiny k): no reflection, T_s = exp(-4 pi k d / (lambda cos))
    c = math.cos(math.radians(theta_deg))
    d = 0.01
    rs, ts = oracle.slab(c, 1.0, k, lam, d)
    want = math.exp(-4 * math.pi * k / (lam * 1e-9) * d / c)
    assert rs < 1e-8  # R ~ k^2 for an index-matched sheet
    assert ts == pytest.approx(want, rel=1e-9)


def test_absorbing_slab_loses_energy():
    for k in (1e-7, 1e-6, 1e-5):
        for t in (0, 40, 75):
            c = math.cos(math.radians(t))
            rs, ts = oracle.slab(c, 1.52, k, 500.0, 0.01)
            assert 0 < ts < 1 and 0 < rs < 1 and rs + ts < 1.0
    # thicker is darker
    assert oracle.slab(1.0, 1.5, 1e-6, 500.0, 0.02)[1] < oracle.slab(1.0, 1.5, 1e-6, 500.0, 0.01)[1]

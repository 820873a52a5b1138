"""Oracle's photon mapping (section 4) pinned to closed forms: the flux the
emission disk delivers to a plate under the sun cone, the caustic flux and
irradiance a mirror throws onto a floor, the photon classes, and agreement
with the (separately pinned) path tracer where the light is smooth."""
import math

import numpy as np
import pytest

import oracle
from paper_1912_04000_gb300 import scenes


def _z(x, want):
    se = x.std() / math.sqrt(x.size)
    return abs(x.mean() - want) / se


@pytest.mark.parametrize("half_deg,tilt_deg", [(14.3239, 0.0), (5.0, 30.0), (10.0, 50.0)])
def test_direct_flux_on_plate(half_deg, tilt_deg):
    # sum of the flux of the direct photons on the 2 x 2 m plate / its area =
    # the irradiance L pi sin^2(a) cos(s) of the sun cone
    a, s = math.radians(half_deg), math.radians(tilt_deg)
    wl = scenes.plate_under_sky(sun_half_angle=a, sun_dir=(math.sin(s), math.cos(s), 0.0))
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    N = 1 << 20
    pos, cls = sc.photon_records(N, 2, seed=3)
    want = math.pi * math.sin(a) ** 2 * math.cos(s)
    for j in range(pos.shape[0]):
        first = pos[j, :, 0, 3] * (cls[j, :, 0] == 1)           # per photon: flux if it landed
        assert _z(first * N / 4.0, want) < 5.0
        assert np.all(np.isin(cls[j], (0, 1)))                   # one plate: no caustic, no indirect
        on = cls[j, :, 0] == 1
        assert np.all(np.abs(pos[j, on, 0, 1]) < 1e-9)           # on the plate y = 0
        assert np.all(np.abs(pos[j, on, 0, 0]) <= 1.0) and np.all(np.abs(pos[j, on, 0, 2]) <= 1.0)


def test_mirror_caustic_flux():
    # caustic photons are exactly the ones the mirror reflected onto the
    # floor: total flux R(theta) L pi sin^2(a) cos(e) x 1 m^2
    e, a = math.radians(45.0), 0.02
    wl = scenes.mirror_caustic(elevation_deg=45.0, sun_half_angle=a)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    N = 1 << 18
    pos, cls = sc.photon_records(N, 3, seed=5)
    R = oracle.fresnel(math.cos(e), 0.3, 3.0)      # mirror normal -z, sun at 45 deg
    want = R * math.pi * math.sin(a) ** 2 * math.cos(e)
    caus = np.where(cls[0] == 2, pos[0, :, :, 3], 0.0).sum(1)
    assert _z(caus * N, want) < 5.0
    # and they land in the patch the closed form predicts (cone spread aside)
    c = cls[0] == 2
    x, y, z = pos[0][..., 0][c], pos[0][..., 1][c], pos[0][..., 2][c]
    assert np.all(np.abs(y) < 1e-9)
    assert np.all(np.abs(x) < 0.5 + 0.1) and np.all((z > -2.0 - 0.15) & (z < -1.0 + 0.15))


def test_mirror_caustic_radiance():
    # at the patch centre: (rho / pi) (E_direct + E_caustic), both
    # L pi sin^2(a) sin(e) times 1 and R; the direct part comes from NEE,
    # the caustic part from the density estimate
    e, a, rho = math.radians(45.0), 0.02, 0.8
    wl = scenes.mirror_caustic(elevation_deg=45.0, sun_half_angle=a, rho=rho, width=4, height=4, spp=8)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    N, r = 1 << 20, 0.15
    out = sc.render_photons(wl.cameras, wl.spp, wl.depth, wl.seed, n_photons=N, photon_depth=3, r_caustic=r,
                            r_global=0.3)
    R = oracle.fresnel(math.cos(e), 0.3, 3.0)
    E = math.pi * math.sin(a) ** 2 * math.sin(e)
    want = rho / math.pi * E * (1.0 + R)
    got = out["spectral_sum"][:, 0] / wl.spp
    # photon count in the gather disk: ~ N x (1 m^2 cos e / disk area) x pi r^2 / (1 m^2)
    pos, cls = sc.photon_records(N, 3, seed=wl.seed)
    n_in = (cls[0] == 2).sum() * math.pi * r * r / (1.0 / math.tan(e))
    tol = 5.0 * rho / math.pi * E * R / math.sqrt(n_in) + 0.02 * want
    assert np.all(np.abs(got - want) < tol), (got, want, tol)


def test_photon_classes_in_box():
    # sunlight enters the box only through the thin-glass wall: transmitted
    # photons are direct (NEE covers them), reflections off the glass from
    # outside leave the scene, so nothing is a caustic; later hits are indirect
    wl = scenes.tiny_box(n_bands=4)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    pos, cls = sc.photon_records(1 << 13, 4, seed=1)
    assert (cls == 1).any() and (cls == 3).any()
    assert not (cls == 2).any()
    # the first stored hit of a photon is direct; later ones indirect
    assert np.all(np.isin(cls[:, :, 0], (0, 1)))
    assert np.all(np.isin(cls[:, :, 1:], (0, 3)))
    # flux never grows along a photon path (rho <= 1, T_s + R_s <= 1)
    phi = pos[..., 3]
    stored = cls > 0
    for k in range(1, phi.shape[2]):
        both = stored[:, :, k] & stored[:, :, k - 1]
        assert np.all(phi[:, :, k][both] <= phi[:, :, k - 1][both] * (1 + 1e-12))


def test_photon_estimate_matches_path_tracer():
    # where the light is smooth, direct visualisation of the indirect photons
    # converges to the path tracer's indirect light: image means agree
    wl = scenes.tiny_box(width=32, height=32, n_bands=2, spp=64, depth=6)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    pt = sc.render(wl.cameras, 64, 6, 11)["spectral_sum"] / 64
    pm = sc.render_photons(wl.cameras, 8, 6, 11, n_photons=1 << 18, photon_depth=6, r_caustic=0.05,
                           r_global=0.12)["spectral_sum"] / 8
    for j in range(2):
        assert abs(pm[:, j].mean() / pt[:, j].mean() - 1.0) < 0.03, (pm[:, j].mean(), pt[:, j].mean())


def test_portal_emission_matches_disk():
    # sunlight enters the box only through its thin-glass wall, so photons
    # emitted on that wall (portal emission) and photons from the disk
    # deliver the same indirect flux inside, and the same image
    wl = scenes.tiny_box(width=24, height=24, n_bands=2, spp=4, depth=5)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    Nd, Np = 1 << 20, 1 << 16
    pd, cd = sc.photon_records(Nd, 3, seed=2, emission=0)
    pp, cp = sc.photon_records(Np, 3, seed=2, emission=1)
    for j in range(2):
        a = np.where(cd[j] == 3, pd[j, ..., 3], 0.0).sum(1) * Nd     # per-photon estimates of the total
        b = np.where(cp[j] == 3, pp[j, ..., 3], 0.0).sum(1) * Np
        se = math.sqrt(a.var() / a.size + b.var() / b.size)
        assert abs(a.mean() - b.mean()) < 5 * se, (a.mean(), b.mean(), se)
        # the portal sends far more of its photons inside
        assert (cp[j] == 3).any(1).mean() > 5 * (cd[j] == 3).any(1).mean()
    kw = dict(photon_depth=5, r_caustic=0.05, r_global=0.15)
    imd = sc.render_photons(wl.cameras, 4, 5, 3, n_photons=Nd, emission=0, **kw)["spectral_sum"]
    imp = sc.render_photons(wl.cameras, 4, 5, 3, n_photons=Np, emission=1, **kw)["spectral_sum"]
    assert abs(imp.mean() / imd.mean() - 1.0) < 0.02


def test_portal_emission_needs_glass():
    wl = scenes.mirror_caustic()
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    with pytest.raises(ValueError):
        sc.photon_records(64, 2, emission=1)

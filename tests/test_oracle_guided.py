"""Oracle of the guided estimator (one-sample MIS of the learned guide and
cosine sampling, section 4 Eq. 2) pinned to mathematics: its proposal draws
follow the density it reports (chi-square over a sphere partition); the
guided estimator keeps the expectation of the plain one (white furnace,
sun-cone irradiance with the balance heuristic, tiny box); every path is
exact in the furnace when only cosine sampling is drawn; the training
records carry the exact incident radiance and the sun-sample weights."""
import math

import numpy as np
import pytest

import oracle
from paper_1912_04000_gb300 import scenes

LOG2_T = 12


def bf16(a):
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def guide_for(scene, seed=0, grid_scale=0.5, w_scale=0.2, bf16_act=True):
    """A seeded random network (BF16 weights) over the scene's bounds."""
    rng = np.random.default_rng(seed)
    grid = (rng.normal(size=oracle.GUIDE_LEVELS * (1 << LOG2_T) * oracle.GUIDE_FEATURES) * grid_scale).astype(np.float32)
    W = bf16(rng.normal(size=oracle.GUIDE_W_SIZE) * w_scale)
    lo = scene.verts.min(0).astype(np.float32)
    hi = scene.verts.max(0).astype(np.float32)
    return oracle.OracleGuide(LOG2_T, lo, hi, grid, W, bf16_act=bf16_act), (lo, hi, grid, W)


def _partition(nz=24, nphi=48, q=6):
    """Equal-area cells in (z, phi) and Gauss-Legendre nodes inside each."""
    x, wx = np.polynomial.legendre.leggauss(q)
    zs = np.linspace(-1, 1, nz + 1)
    ps = np.linspace(0, 2 * math.pi, nphi + 1)
    om, wt, cell = [], [], []
    for i in range(nz):
        z = 0.5 * (zs[i + 1] - zs[i]) * x + 0.5 * (zs[i + 1] + zs[i])
        wz = 0.5 * (zs[i + 1] - zs[i]) * wx
        for j in range(nphi):
            p = 0.5 * (ps[j + 1] - ps[j]) * x + 0.5 * (ps[j + 1] + ps[j])
            wp = 0.5 * (ps[j + 1] - ps[j]) * wx
            Z, P = np.meshgrid(z, p, indexing="ij")
            W_ = np.outer(wz, wp)
            s = np.sqrt(1 - Z ** 2)
            om.append(np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3))
            wt.append(W_.ravel())
            cell.append(np.full(W_.size, i * nphi + j))
    return np.concatenate(om), np.concatenate(wt), np.concatenate(cell), nz, nphi


def _cells(om, nz, nphi):
    z = np.clip(om[:, 2], -1, 1 - 1e-15)
    phi = np.mod(np.arctan2(om[:, 1], om[:, 0]), 2 * math.pi)
    iz = np.minimum(((z + 1) / 2 * nz).astype(int), nz - 1)
    ip = np.minimum((phi / (2 * math.pi) * nphi).astype(int), nphi - 1)
    return iz * nphi + ip


@pytest.mark.parametrize("alpha,seed", [(1.0, 0), (0.7, 1), (0.3, 2)])
def test_mis_draws_follow_reported_density(alpha, seed):
    """Draws of the one-sample MIS proposal land in the cells of a sphere
    partition with the probabilities that its density alpha q + (1 - alpha)
    cos+ / pi (q pinned to integrate to 1 elsewhere) gives them."""
    from scipy import stats
    rng = np.random.default_rng(seed)
    Y = rng.normal(size=48)
    Y[4:40:5] = rng.uniform(-1.0, 6.0, 8)
    Y[4] = 40.0  # one sharp lobe (kappa ~ 40) exercises the stable vMF draw
    n = np.array([0.3, -0.5, 0.81])
    n /= np.linalg.norm(n)
    N = 400_000
    om, pdf = oracle.guide_mis_draws(Y, n, alpha, rng.random((N, 6)))
    np.testing.assert_allclose(np.linalg.norm(om, axis=1), 1.0, atol=1e-12)
    qom, qw, qcell, nz, nphi = _partition()
    dens = alpha * oracle.guide_density(Y, qom) + (1 - alpha) * np.maximum(qom @ n, 0) / math.pi
    p_cell = np.bincount(qcell, weights=dens * qw, minlength=nz * nphi)
    assert abs(p_cell.sum() - 1.0) < 1e-6
    obs = np.bincount(_cells(om, nz, nphi), minlength=nz * nphi)
    exp = N * p_cell
    big = exp > 20
    chi2 = (((obs - exp) ** 2)[big] / exp[big]).sum()
    p = stats.chi2.sf(chi2, big.sum() - 1)
    assert p > 1e-4, (chi2, big.sum(), p)
    assert obs[~big].sum() < N * 1e-3 + 5 * math.sqrt(N * 1e-3)
    # the reported density is the one the partition integrates
    np.testing.assert_allclose(
        pdf, alpha * oracle.guide_density(Y, om) + (1 - alpha) * np.maximum(om @ n, 0) / math.pi, rtol=1e-12)


@pytest.mark.parametrize("albedo,depth", [(0.5, 5), (0.8, 4)])
def test_furnace_cosine_only_is_exact(albedo, depth):
    """alpha = 0: the proposal is cosine sampling and p_mix = cos / pi, so
    every guided path is L_e (1 - a^D), as in the plain estimator."""
    wl = scenes.furnace_box(albedo=albedo, le=2.0, depth=depth)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    g, _ = guide_for(wl.scene)
    r = sc.render_guided(g, wl.cameras, wl.spp, wl.depth, wl.seed, alpha=0.0, guide_depth=3, record_paths=True)
    np.testing.assert_allclose(r["path_L"], 2.0 * (1 - albedo ** depth), rtol=1e-6)


@pytest.mark.parametrize("albedo,depth", [(0.5, 5), (0.8, 4)])
def test_furnace_guided_mean(albedo, depth):
    """alpha = 0.7 with a random network: paths vary, their mean does not."""
    wl = scenes.furnace_box(albedo=albedo, le=2.0, depth=depth, width=16, height=16, spp=32)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    g, _ = guide_for(wl.scene, seed=3)
    r = sc.render_guided(g, wl.cameras, wl.spp, wl.depth, wl.seed, alpha=0.7, guide_depth=3, record_paths=True)
    L = r["path_L"].ravel()
    want = 2.0 * (1 - albedo ** depth)
    assert L.std() > 1e-3 * want  # the guide is used
    assert abs(L.mean() - want) < 5 * L.std() / math.sqrt(L.size)


def test_furnace_records_carry_incident_radiance():
    """Guide depth 1 in the furnace: the radiance arriving along a
    continuation is exactly L_e (1 - a^(D-1)) (the plain cosine suffix), so
    every continuation record's weight x p_mix / cos recovers it (the
    network with exact activations, so that q is smooth in the records'
    float positions and directions)."""
    albedo, depth, alpha = 0.6, 5, 0.7
    wl = scenes.furnace_box(albedo=albedo, le=2.0, depth=depth, width=8, height=8, spp=8)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    g, (lo, hi, grid, W) = guide_for(wl.scene, seed=4, bf16_act=False)
    r = sc.render_guided(g, wl.cameras, wl.spp, wl.depth, wl.seed, alpha=alpha, guide_depth=1, records=True)
    rec = r["records"].reshape(-1, 2, 12)
    cont = rec[:, 0]
    ok = cont[:, 3] > 0
    assert ok.mean() > 0.5
    c = cont[ok]
    pos, nrm, grp, om = c[:, 0:3], c[:, 4:7], c[:, 7].astype(np.uint32), c[:, 8:11]
    _, _, q = oracle.guide_forward(LOG2_T, lo, hi, grid, W, pos, nrm, grp, om)
    cos = np.einsum("ij,ij->i", nrm.astype(np.float64), om.astype(np.float64))
    pmix = alpha * q + (1 - alpha) * np.maximum(cos, 0) / math.pi
    L_in = c[:, 3] * pmix / cos
    np.testing.assert_allclose(L_in, 2.0 * (1 - albedo ** (depth - 1)), rtol=2e-5)
    # no sun in the furnace's spectra reaches inside: sun records are empty
    assert np.all(rec[:, 1, 3] == 0)


@pytest.mark.parametrize("half_deg,tilt_deg", [(14.3239, 0.0), (10.0, 45.0)])
def test_plate_sun_balance_heuristic(half_deg, tilt_deg):
    """Plate under a sun cone, guided vertex 1: the direct sun comes from
    the weighted sun sample and the weighted guided escape; the two weights
    sum to one per direction, so the mean stays rho sin^2(a) cos(s).  The sun
    records average L pi sin^2(a) cos(s) (the cone's irradiance)."""
    a, s = math.radians(half_deg), math.radians(tilt_deg)
    sun = (math.sin(s), math.cos(s), 0.0)
    wl = scenes.plate_under_sky(spp=256, rho=0.6, sun_half_angle=a, sun_dir=sun, depth=2)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    g, _ = guide_for(wl.scene, seed=5)
    r = sc.render_guided(g, wl.cameras, wl.spp, wl.depth, wl.seed, alpha=0.7, guide_depth=1, record_paths=True,
                         records=True)
    L = r["path_L"].ravel()
    want = 0.6 * math.sin(a) ** 2 * math.cos(s)
    assert abs(L.mean() - want) < 5 * L.std() / math.sqrt(L.size)
    sun_w = r["records"].reshape(-1, 2, 12)[:, 1, 3].astype(np.float64)
    irr = math.pi * math.sin(a) ** 2 * math.cos(s)
    assert np.all(sun_w > 0)
    assert abs(sun_w.mean() - irr) < 5 * sun_w.std() / math.sqrt(sun_w.size)


def test_guided_box_matches_plain_expectation():
    """The glass box: guided and plain images agree within Monte Carlo error
    (per band, z < 5 on the image mean)."""
    wl = scenes.tiny_box(width=16, height=12, spp=64, n_bands=4)
    sc = oracle.OracleScene(wl.scene, wl.spectra)
    g, _ = guide_for(wl.scene, seed=6)
    plain = sc.render(wl.cameras, wl.spp, wl.depth, 1, record_paths=True)["path_L"]
    guided = sc.render_guided(g, wl.cameras, wl.spp, wl.depth, 2, alpha=0.7, guide_depth=2,
                              record_paths=True)["path_L"]
    for b in range(4):
        a_, b_ = plain[:, :, b].ravel(), guided[:, :, b].ravel()
        z = abs(a_.mean() - b_.mean()) / math.sqrt(a_.var() / a_.size + b_.var() / b_.size)
        assert z < 5, (b, z)
    assert not np.array_equal(plain, guided)

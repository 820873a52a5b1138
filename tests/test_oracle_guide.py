"""Oracle of the learned guide pinned to mathematics: the vMF mixture is a
density on the sphere (quadrature), the analytic loss gradient equals
central finite differences for every parameter kind, the hash-grid encoding
interpolates (a constant grid gives constant features; a position on a
vertex of a dense level reads that vertex's entry, feature by feature), the
level resolutions follow their closed form, and the SH inputs are an
orthonormal basis."""
import math

import numpy as np
import pytest

import oracle


def _sphere_quadrature(n_theta=400, n_phi=800):
    # Gauss-Legendre in cos(theta), uniform in phi
    x, wx = np.polynomial.legendre.leggauss(n_theta)
    phi = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    ct = np.repeat(x, n_phi)
    st = np.sqrt(1 - ct ** 2)
    ph = np.tile(phi, n_theta)
    om = np.stack([st * np.cos(ph), st * np.sin(ph), ct], 1)
    w = np.repeat(wx, n_phi) * (2 * math.pi / n_phi)
    return om, w


@pytest.mark.parametrize("seed,kscale", [(0, 0.0), (1, 2.0), (2, 5.0), (3, 8.0)])
def test_vmf_mixture_integrates_to_one(seed, kscale):
    rng = np.random.default_rng(seed)
    Y = rng.normal(size=48)
    Y[4::5] += kscale  # kappa = 0.5 + softplus(.) up to ~ 8.5
    om, w = _sphere_quadrature()
    q = oracle.guide_density(Y, om)
    assert abs((q * w).sum() - 1.0) < 1e-6
    assert (q >= 0).all()


def _setup(seed, n=12, log2_T=10):
    rng = np.random.default_rng(seed)
    lo = np.array([0.0, 0.0, 0.0], np.float32)
    hi = np.array([80.0, 25.0, 20.0], np.float32)
    T = 1 << log2_T
    grid = (rng.normal(size=oracle.GUIDE_LEVELS * T * oracle.GUIDE_FEATURES) * 0.3).astype(np.float32)
    W = (rng.normal(size=oracle.GUIDE_W_SIZE) * 0.25).astype(np.float32)
    pos = (lo + (hi - lo) * rng.random((n, 3))).astype(np.float32)
    nrm = rng.normal(size=(n, 3))
    nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
    om = rng.normal(size=(n, 3))
    om = (om / np.linalg.norm(om, axis=1, keepdims=True)).astype(np.float32)
    group = rng.integers(0, 9, n).astype(np.uint32)
    wt = rng.exponential(size=n).astype(np.float32)
    return log2_T, lo, hi, grid, W, pos, nrm, group, om, wt


def test_gradient_matches_finite_differences():
    args = _setup(3)
    log2_T, lo, hi, grid, W, pos, nrm, group, om, wt = args
    loss, dW, dgrid = oracle.guide_loss_grad(*args)
    rng = np.random.default_rng(4)
    sizes = [64 * 64, 64 * 64, 64 * 64, 64 * 48]
    starts = np.cumsum([0] + sizes)
    checked = 0
    for layer in range(4):
        for i in rng.choice(sizes[layer], 12, replace=False):
            idx = starts[layer] + i
            fd = _fd(lambda v: oracle.guide_loss_grad(log2_T, lo, hi, grid, v, pos, nrm, group, om, wt)[0], W, idx)
            if fd is None:
                continue
            assert abs(fd - dW[idx]) <= 1e-5 * max(abs(dW[idx]), 1e-3 * np.abs(dW).max()), (layer, fd, dW[idx])
            checked += 1
    touched = np.nonzero(dgrid)[0]
    for idx in rng.choice(touched, 24, replace=False):
        fd = _fd(lambda v: oracle.guide_loss_grad(log2_T, lo, hi, v, W, pos, nrm, group, om, wt)[0], grid, idx)
        if fd is None:
            continue
        assert abs(fd - dgrid[idx]) <= 1e-5 * max(abs(dgrid[idx]), 1e-3 * np.abs(dgrid).max()), (fd, dgrid[idx])
        checked += 1
    assert checked >= 50


def _fd(f, arr, idx):
    """Central difference over the float-representable step; None when two
    step sizes disagree (a ReLU kink inside the step)."""
    out = []
    for h in (2.0 ** -12, 2.0 ** -13):
        a = arr.copy()
        b = arr.copy()
        a[idx] = np.float32(arr[idx] + h)
        b[idx] = np.float32(arr[idx] - h)
        out.append((f(a) - f(b)) / (float(a[idx]) - float(b[idx])))
    if abs(out[0] - out[1]) > 1e-4 * max(abs(out[1]), 1e-12):
        return None
    return out[1]


def test_loss_is_weighted_negative_log_likelihood():
    log2_T, lo, hi, grid, W, pos, nrm, group, om, wt = _setup(5)
    loss, _, _ = oracle.guide_loss_grad(log2_T, lo, hi, grid, W, pos, nrm, group, om, wt)
    _, _, q = oracle.guide_forward(log2_T, lo, hi, grid, W, pos, nrm, group, om)
    w = wt.astype(np.float64)
    assert loss == pytest.approx(-np.mean(w / w.mean() * np.log(q)), rel=1e-10)
    # zero weights: no loss, no gradient
    l0, dW0, dg0 = oracle.guide_loss_grad(log2_T, lo, hi, grid, W, pos, nrm, group, om, np.zeros_like(wt))
    assert l0 == 0.0 and not dW0.any() and not dg0.any()


def test_encoding_interpolates():
    log2_T, lo, hi, grid, W, pos, nrm, group, om, wt = _setup(6, n=50)
    F = oracle.GUIDE_FEATURES
    feat = np.array([0.25, -0.5, 1.0, -2.0], np.float32)
    const = np.tile(feat, grid.size // F)  # entry (l, i) holds the four values
    X, _, _ = oracle.guide_forward(log2_T, lo, hi, const, W, pos, nrm, group, om)
    for q in range(F):
        np.testing.assert_allclose(X[:, q:32:F], feat[q], atol=1e-12)
    # one-hot group and zero padding
    np.testing.assert_array_equal(X[np.arange(50), 48 + group], 1.0)
    assert X[:, 48:64].sum() == 50


def test_level_resolutions_closed_form():
    # n_min b^l with b = (n_max / n_min)^(1 / 7): 16 to 2048 doubles per level
    res = oracle.guide_resolutions(16.0, 2048.0)
    np.testing.assert_array_equal(res, 16 * 2 ** np.arange(8))
    res = oracle.guide_resolutions(10.0, 1000.0)  # b = 100^(1/7)
    np.testing.assert_array_equal(res, np.floor(10.0 * 100.0 ** (np.arange(8) / 7) * (1 + 1e-12)))


def test_dense_vertices_read_their_entries():
    """Positions on vertices (i, j, k) / 16 of the unit box: levels 0 and 1
    (resolutions 16 and 32, (r + 1)^3 <= 2^16 entries, dense index x + y (r + 1)
    + z (r + 1)^2) read exactly the vertex entry, its four features in order,
    from the level's block of the table."""
    log2_T = 16
    T = 1 << log2_T
    F = oracle.GUIDE_FEATURES
    rng = np.random.default_rng(8)
    grid = rng.normal(size=oracle.GUIDE_LEVELS * T * F).astype(np.float32)
    W = np.zeros(oracle.GUIDE_W_SIZE, np.float32)
    ijk = rng.integers(0, 16, size=(40, 3))  # each position the near corner of its cell
    pos = (ijk / 16.0).astype(np.float32)
    n = len(pos)
    nrm = np.tile(np.array([[0.0, 0.0, 1.0]], np.float32), (n, 1))
    X, _, _ = oracle.guide_forward(log2_T, [0, 0, 0], [1, 1, 1], grid, W, pos, nrm, np.zeros(n, np.uint32), nrm)
    g = grid.reshape(oracle.GUIDE_LEVELS, T, F)
    for level, r in ((0, 16), (1, 32)):
        c = ijk * (r // 16)
        idx = c[:, 0] + c[:, 1] * (r + 1) + c[:, 2] * (r + 1) ** 2
        np.testing.assert_array_equal(X[:, F * level:F * level + F], g[level, idx].astype(np.float64))


def test_sh_inputs_orthonormal():
    # the 16 SH inputs of the normal are orthonormal on the sphere
    om, w = _sphere_quadrature(60, 120)
    n = om.shape[0]
    zeros = np.zeros((n, 3), np.float32)
    X, _, _ = oracle.guide_forward(10, [0, 0, 0], [1, 1, 1],
                                   np.zeros(oracle.GUIDE_LEVELS * 1024 * oracle.GUIDE_FEATURES, np.float32),
                                   np.zeros(oracle.GUIDE_W_SIZE, np.float32), zeros, om.astype(np.float32),
                                   np.zeros(n, np.uint32), om.astype(np.float32))
    S = X[:, 32:48]
    G = (S * w[:, None]).T @ S
    np.testing.assert_allclose(G, np.eye(16), atol=2e-6)


def test_adam_closed_forms():
    """Adam's bias correction makes a constant gradient g give m_hat = g and
    v_hat = g^2 at every step, so each step moves every parameter by
    lr g / (|g| + eps): lr sign(g) for |g| >> eps, nothing where g = 0."""
    rng = np.random.default_rng(7)
    n = 1000
    p0 = rng.normal(size=n)
    g = rng.normal(size=n) * 10.0 ** rng.uniform(-3, 2, n)
    g[::17] = 0.0
    p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    lr = 1e-2
    for t in range(1, 6):
        oracle.adam_step(p, g, m, v, t, lr)
        np.testing.assert_allclose(p, p0 - t * lr * g / (np.abs(g) + 1e-15), rtol=0, atol=1e-12)
    # a gradient that changes: first step still lr sign(g1); the second moves
    # by lr m_hat / sqrt(v_hat) with the hand-computed moments
    p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    g2 = -0.5 * g
    oracle.adam_step(p, g, m, v, 1, lr)
    oracle.adam_step(p, g2, m, v, 2, lr)
    m_hat = (0.9 * 0.1 * g + 0.1 * g2) / (1 - 0.9 ** 2)
    v_hat = (0.99 * 0.01 * g * g + 0.01 * g2 * g2) / (1 - 0.99 ** 2)
    want = p0 - lr * g / (np.abs(g) + 1e-15) - lr * np.divide(m_hat, np.sqrt(v_hat) + 1e-15)
    np.testing.assert_allclose(p, want, rtol=0, atol=1e-10)

"""Learned guide on the GPU (tcgen05 MLP, hash grid, vMF head, training)
through the C ABI against the FP64 oracle fed the same BF16-rounded weights."""
import numpy as np
import pytest

import oracle
from paper_1912_04000_gb300 import scenes

pytestmark = pytest.mark.gpu

LOG2_T = 12


def bf16(a):
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def setup():
    from paper_1912_04000_gb300.renderer import Renderer
    wl = scenes.nave(width=8, height=8, n_bands=4, col_seg=8, col_rings=3)
    R = Renderer(0).load(wl)
    R.guide_init(seed=1, log2_table=LOG2_T)
    lo = wl.scene.verts.min(0).astype(np.float32)
    hi = wl.scene.verts.max(0).astype(np.float32)
    return R, lo, hi


def _records(rng, lo, hi, n, concentrated=False):
    pos = lo + (hi - lo) * rng.random((n, 3))
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    if concentrated:
        # target direction depends on the position: a learnable field
        t = np.stack([np.cos(pos[:, 0] / 13.0), 0.6 + 0.0 * pos[:, 1], np.sin(pos[:, 2] / 7.0)], 1)
        om = t / np.linalg.norm(t, axis=1, keepdims=True) + 0.05 * rng.normal(size=(n, 3))
    else:
        om = rng.normal(size=(n, 3))
    om /= np.linalg.norm(om, axis=1, keepdims=True)
    group = rng.integers(0, 9, n)
    wt = rng.exponential(size=n)
    rec = np.zeros((n, 12), np.float32)
    rec[:, 0:3], rec[:, 3], rec[:, 4:7], rec[:, 7], rec[:, 8:11] = pos, wt, nrm, group, om
    return rec


def _params(rng):
    grid = (rng.normal(size=oracle.GUIDE_LEVELS * (1 << LOG2_T) * oracle.GUIDE_FEATURES) * 0.5).astype(np.float32)
    W = bf16(rng.normal(size=oracle.GUIDE_W_SIZE) * 0.2)
    return grid, W


def _oracle_args(rec, lo, hi):
    return (rec[:, 0:3], rec[:, 4:7], rec[:, 7].astype(np.uint32), rec[:, 8:11])


def test_forward_matches_oracle(setup):
    R, lo, hi = setup
    rng = np.random.default_rng(0)
    grid, W = _params(rng)
    R.guide_set_params(grid, W)
    rec = _records(rng, lo, hi, 1000)  # 7 full tiles + a ragged one
    Y, q = (t.cpu().numpy() for t in R.guide_eval(rec))
    pos, nrm, grp, om = _oracle_args(rec, lo, hi)
    # the BF16 network: layer inputs rounded to BF16, FP32 (GPU) / FP64
    # (oracle) accumulation
    _, Yo, qo = oracle.guide_forward(LOG2_T, lo, hi, grid, W, pos, nrm, grp, om, bf16_act=True)
    scale = np.abs(Yo).max(1, keepdims=True)
    assert (np.abs(Y - Yo) / scale).max() < 2e-2
    assert np.corrcoef(Y.ravel(), Yo.ravel())[0, 1] > 0.9999
    rel = np.abs(np.log(q) - np.log(qo))
    assert np.median(rel) < 2e-3 and rel.max() < 0.1
    # and against the exact-activation network, the BF16 rounding is small
    _, Ye, _ = oracle.guide_forward(LOG2_T, lo, hi, grid, W, pos, nrm, grp, om)
    assert np.corrcoef(Y.ravel(), Ye.ravel())[0, 1] > 0.999


def test_gradients_match_oracle(setup):
    R, lo, hi = setup
    rng = np.random.default_rng(1)
    grid, W = _params(rng)
    R.guide_set_params(grid, W)
    rec = _records(rng, lo, hi, 777)
    loss, dg, dw = R.guide_grad(rec)
    dg, dw = dg.cpu().numpy().astype(np.float64), dw.cpu().numpy().astype(np.float64)
    pos, nrm, grp, om = _oracle_args(rec, lo, hi)
    lo_, dWo, dgo = oracle.guide_loss_grad(LOG2_T, lo, hi, grid, W, pos, nrm, grp, om, rec[:, 3], bf16_act=True)
    assert loss == pytest.approx(lo_, rel=2e-2)
    starts = np.cumsum([0, 4096, 4096, 4096, 3072])
    for l in range(4):
        a, b = dw[starts[l]:starts[l + 1]], dWo[starts[l]:starts[l + 1]]
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        assert cos >= 0.999, (l, cos)
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 2e-2, (l, np.linalg.norm(a - b) / np.linalg.norm(b))
    cos = dg @ dgo / (np.linalg.norm(dg) * np.linalg.norm(dgo))
    assert cos >= 0.999, cos
    assert np.linalg.norm(dg - dgo) / np.linalg.norm(dgo) <= 2e-2


def test_training_reduces_loss(setup):
    R, lo, hi = setup
    import torch
    R.guide_init(seed=3, log2_table=LOG2_T, lr_grid=1e-2, lr_mlp=2e-3)
    rng = np.random.default_rng(2)
    rec = torch.as_tensor(_records(rng, lo, hi, 1 << 15, concentrated=True), device="cuda")
    losses = [R.guide_train_step(rec) for _ in range(200)]
    assert np.isfinite(losses).all()
    # a uniform density has loss log(4 pi) = 2.53; the concentrated target is learnable
    assert losses[0] > 2.0 and losses[-1] < losses[0] - 1.0, (losses[0], losses[-1])


def test_adam_step_matches_oracle(setup):
    """One training step on the GPU against the oracle's Adam step: applied
    to the GPU's own gradient of the step, Adam must give the GPU's
    parameters (at the first step a parameter with gradient g moves by
    lr g / (|g| + eps)); applied to the oracle's FP64 gradient, the entries
    above 1% of the largest move as on the GPU (the BF16 network's gradient
    may flip the sign of an entry close to 0, a difference the gradient test
    bounds), and grid entries no record touches do not move."""
    R, lo, hi = setup
    rng = np.random.default_rng(8)
    grid, W = _params(rng)
    R.guide_init(seed=1, log2_table=LOG2_T, lr_grid=1e-2, lr_mlp=1e-3)
    R.guide_set_params(grid, W)  # also resets the Adam state
    rec = _records(rng, lo, hi, 777)
    _, dg, dw = R.guide_grad(rec)  # the step's gradient (the weights' is the same on every call)
    dg, dw = dg.cpu().numpy().astype(np.float64), dw.cpu().numpy().astype(np.float64)
    R.guide_train_step(rec)
    grid1, W1 = R.guide_get_params()
    pos, nrm, grp, om = _oracle_args(rec, lo, hi)
    _, dWo, dgo = oracle.guide_loss_grad(LOG2_T, lo, hi, grid, W, pos, nrm, grp, om, rec[:, 3], bf16_act=True)
    for p0, p1, g, go, lr, what in ((grid, grid1, dg, dgo, 1e-2, "grid"), (W, W1, dw, dWo, 1e-3, "W")):
        # Adam: the oracle's step on the GPU's gradient, to float rounding
        want = p0.astype(np.float64)
        oracle.adam_step(want, g, np.zeros_like(want), np.zeros_like(want), 1, lr)
        ok = np.abs(p1 - want) <= 1e-6
        # the grid gradient is summed with float atomics in any order, so an
        # entry near 0 can change sign between the two evaluations
        assert np.mean(ok) >= (0.9999 if what == "grid" else 1.0), (what, np.mean(ok))
        # the gradient: large entries as the oracle's
        want_o = p0.astype(np.float64)
        oracle.adam_step(want_o, go, np.zeros_like(want_o), np.zeros_like(want_o), 1, lr)
        big = np.abs(go) > 1e-2 * np.abs(go).max()
        assert big.sum() > 100
        np.testing.assert_allclose(p1[big], want_o[big], rtol=0, atol=1e-6, err_msg=what)
        moved = np.abs(p1.astype(np.float64) - p0) > 0.5 * lr
        assert moved[big].all(), what
        zero = go == 0.0
        if zero.any():
            assert np.mean(p1[zero] == p0[zero]) > 0.9999, what

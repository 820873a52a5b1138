"""Oracle Philox4x32-10 pinned to the published known-answer vectors and to
uniformity (chi-square) of the 24-bit uniforms the renderer draws."""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_known_answer_vectors():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = oracle.philox4x32_10(key, ctr)
        assert [int(x) for x in got] == want


def test_batch_matches_single():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    out = oracle.philox_batch(0x12345678, 0x9abcdef0, ctr)
    for i in range(0, 64, 7):
        assert (out[i] == oracle.philox4x32_10([0x12345678, 0x9abcdef0], ctr[i])).all()


def test_uniforms_chi_square():
    # counters laid out as the renderer uses them: (pixel, sample, band, 4*vertex + call)
    n = 1 << 16
    i = np.arange(n, dtype=np.uint32)
    ctr = np.stack([i % 4096, i // 4096, (i * 7) % 81, (i % 9) * 4], 1).astype(np.uint32)
    out = oracle.philox_batch(0, 0, ctr)
    u = (out >> 8).astype(np.float64) / 16777216.0
    assert u.min() >= 0.0 and u.max() < 1.0
    bins = 64
    for lane in range(4):
        h = np.bincount((u[:, lane] * bins).astype(int), minlength=bins)
        e = n / bins
        chi2 = ((h - e) ** 2 / e).sum()
        # 63 dof: mean 63, sd ~11.2; 6 sigma bound
        assert chi2 < 63 + 6 * 11.3, chi2
    # lanes are not correlated
    c = np.corrcoef(u.T)
    assert np.abs(c - np.eye(4)).max() < 0.02


def test_counter_fields_change_output():
    base = oracle.philox4x32_10([0, 0], [5, 6, 7, 8])
    for j in range(4):
        ctr = [5, 6, 7, 8]
        ctr[j] += 1
        assert (oracle.philox4x32_10([0, 0], ctr) != base).all()

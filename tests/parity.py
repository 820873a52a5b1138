"""Parity metrics shared by the GPU tests (test helper, no renderer arithmetic).

Per pixel: rel = ||G - O||_1 / ||O||_1 over the three XYZ channels (0 when
both are 0).  The bar: rel <= 1e-4 on at least 99.9% of pixels, and the
aggregate relative L1 error sum|G - O| / sum|O| over the pixels that pass is
at most 1e-5 (the pixels that fail are the grazing-hit divergences the bar
allows, counted separately).
"""
import numpy as np

PIX_TOL = 1e-4
PIX_FRAC = 0.999
MEAN_TOL = 1e-5


def pixel_rel(g, o):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    num = np.abs(g - o).sum(-1)
    den = np.abs(o).sum(-1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), np.where(num > 0, np.inf, 0.0))


def xyz_parity(g, o):
    rel = pixel_rel(g, o)
    ok = rel <= PIX_TOL
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    den = np.abs(o[ok]).sum()
    mean_ok = float(np.abs(g[ok] - o[ok]).sum() / den) if den > 0 else 0.0
    den_all = np.abs(o).sum()
    return {
        "frac_ok": float(ok.mean()),
        "n_bad": int((~ok).sum()),
        "mean_rel_ok": mean_ok,
        "mean_rel_all": float(np.abs(g - o).sum() / den_all) if den_all > 0 else 0.0,
        "max_rel": float(rel[np.isfinite(rel)].max()) if np.isfinite(rel).any() else 0.0,
    }


def assert_parity(g, o, what=""):
    m = xyz_parity(g, o)
    assert m["frac_ok"] >= PIX_FRAC, f"{what}: {m}"
    assert m["mean_rel_ok"] <= MEAN_TOL, f"{what}: {m}"
    return m

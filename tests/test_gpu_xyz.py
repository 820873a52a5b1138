"""Spectrum -> XYZ contraction through the C ABI against the oracle's FP64
contraction: the tensor-core split-BF16 mode within the render tolerance, the
FP64 mode exactly to float rounding, plain BF16 within its 8-bit mantissa."""
import numpy as np
import pytest

import oracle
from paper_1912_04000_gb300 import _native, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1912_04000_gb300.renderer import Renderer
    return Renderer(0)


@pytest.mark.parametrize("n_pix,n_bands,band_first,band_count,spp",
                         [(1000, 16, 0, 16, 4), (3001, 81, 0, 81, 16), (517, 81, 7, 33, 3), (128, 17, 0, 17, 1),
                          (1, 81, 0, 81, 16), (40000, 81, 0, 81, 16), (1280, 96, 0, 96, 2),
                          (1300, 150, 0, 150, 2)])
def test_xyz_modes(R, n_pix, n_bands, band_first, band_count, spp):
    import torch
    wl = scenes.tiny_box(n_bands=n_bands, width=8, height=8)
    R.load(wl)
    rng = np.random.default_rng(n_pix + n_bands)
    # radiance sums over spp samples, heavy-tailed like path-traced pixels
    s = (rng.lognormal(-3.0, 2.0, size=(n_pix, band_count)) * spp).astype(np.float64)
    s[rng.random(s.shape) < 0.05] = 0.0
    want = oracle.xyz(s, band_first, spp, wl.spectra.cmf_w)
    st = torch.from_numpy(s).cuda()
    scale = np.abs(want).sum(1, keepdims=True)
    for mode, tol in ((_native.XYZ_BF16X3, 2e-6), (_native.XYZ_FP64, 1e-6), (_native.XYZ_BF16, 2e-2)):
        got = R.xyz(st, band_first, spp, mode).cpu().numpy().astype(np.float64)
        err = np.abs(got - want) / np.maximum(scale, 1e-300)
        assert err.max() <= tol, (mode, err.max())


def test_render_default_mode_is_tensor_core(R):
    wl = scenes.tiny_box()
    R.load(wl)
    a = R.render(wl.cameras, wl.spp, wl.depth, wl.seed)  # default RT_XYZ_BF16X3
    b = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=_native.XYZ_FP64)
    ga, gb = a["xyz"].cpu().numpy(), b["xyz"].cpu().numpy()
    den = np.abs(gb).sum(1)
    rel = np.abs(ga - gb).sum(1) / np.where(den > 0, den, 1)
    assert rel.max() < 5e-6
    assert np.array_equal(a["spectral"].cpu().numpy(), b["spectral"].cpu().numpy())


def test_tensor_core_band_limit(R):
    import torch
    wl = scenes.tiny_box(n_bands=200, width=4, height=4)
    R.load(wl)
    s = torch.ones((16, 200), dtype=torch.float64, device="cuda")
    with pytest.raises(_native.RtError) as e:
        R.xyz(s, 0, 1, _native.XYZ_BF16X3)
    assert e.value.status == 1
    R.xyz(s, 0, 1, _native.XYZ_FP64)

"""Full spectral renders through the C ABI against the CPU FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1912_04000_gb300 import scenes

from parity import assert_parity, assert_sampled_parity, crop_and_subset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1912_04000_gb300.renderer import Renderer
    return Renderer(0)


def _oracle(wl, **kw):
    return oracle.OracleScene(wl.scene, wl.spectra).render(wl.cameras, wl.spp, wl.depth, wl.seed, **kw)


@pytest.mark.parametrize("albedo,depth", [(0.5, 5), (0.9, 8)])
def test_white_furnace(R, albedo, depth):
    wl = scenes.furnace_box(albedo=albedo, le=1.5, depth=depth, width=24, height=20, spp=3)
    R.load(wl)
    out = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)
    s = out["spectral"].cpu().numpy() / wl.spp
    np.testing.assert_allclose(s, 1.5 * (1 - albedo ** depth), rtol=2e-6)


def test_tiny_box_full_image(R):
    """The 12-triangle glass box at its full size: 128 x 128, 16 bands, 4 spp,
    depth 4, seed 0 -- every pixel against the oracle."""
    wl = scenes.tiny_box()
    R.load(wl)
    out = R.render(wl.cameras, wl.spp, wl.depth, wl.seed)  # tensor-core XYZ (split BF16)
    o = _oracle(wl)
    m = assert_parity(out["xyz"].cpu().numpy(), o["xyz"], "tiny box")
    print("tiny box parity", m)
    # spectral sums too
    gs = out["spectral"].cpu().numpy()
    rel = np.abs(gs - o["spectral_sum"]).sum() / np.abs(o["spectral_sum"]).sum()
    assert rel < 1e-5


def test_per_path_records(R):
    wl = scenes.tiny_box(width=40, height=30, spp=3)
    R.load(wl)
    pix = np.array([0, 17, 333, 600, 1199], np.int64)
    out = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, probe_pixels=pix, xyz_mode=2)
    o = _oracle(wl, pixels=pix.astype(np.uint32), record_paths=True)
    gL = out["probe_L"].cpu().numpy()
    gS = out["probe_sig"].cpu().numpy().view(np.uint32)
    same = gS == o["path_sig"]
    assert same.mean() >= 0.99
    np.testing.assert_allclose(gL[same], o["path_L"][same], rtol=2e-5, atol=1e-9)


def test_band_subdomains_and_waves(R):
    wl = scenes.tiny_box(width=48, height=40, spp=3)
    R.load(wl)
    full = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)
    a = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, band_first=0, band_count=7, xyz_mode=2)
    b = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, band_first=7, band_count=9, xyz_mode=2)
    fs = full["spectral"].cpu().numpy()
    assert np.array_equal(np.concatenate([a["spectral"].cpu().numpy(), b["spectral"].cpu().numpy()], 1), fs)
    # wave size does not change any bit: each slot's samples are summed in order
    small = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, wave_capacity=5000, xyz_mode=2)
    assert np.array_equal(small["spectral"].cpu().numpy(), fs)
    again = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)
    assert np.array_equal(again["spectral"].cpu().numpy(), fs)
    # partial XYZ of disjoint band ranges add up
    np.testing.assert_allclose(a["xyz"].cpu().numpy() + b["xyz"].cpu().numpy(), full["xyz"].cpu().numpy(),
                               rtol=1e-5, atol=1e-9)


def test_nave_sampled_pixels(R):
    """The 200k-triangle nave at its full size (1024 x 768, 81 bands, 16 spp,
    depth 8) rendered on the GPU; a 64 x 48 crop at the image centre and a
    seeded 1% of all pixels (10,902 pixels, 14.1M paths) are re-rendered
    path by path by the oracle and held to the bar on every sampled pixel."""
    wl = scenes.nave()
    R.load(wl)
    pix = crop_and_subset([(1024, 768)], x0=480, y0=360, frac=0.01, seed=2024)
    out = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, probe_pixels=pix, xyz_mode=2)
    o = _oracle(wl, pixels=pix.astype(np.uint32), record_paths=True)
    m = assert_sampled_parity(out["xyz"].cpu().numpy()[pix], o["xyz"], out["probe_L"].cpu().numpy(), o["path_L"],
                              out["probe_sig"].cpu().numpy().view(np.uint32), o["path_sig"], wl.spectra.cmf_w,
                              wl.spp, "nave crop + 1%")
    # every pixel (all paths) within 1e-4 on at least 99% of the sample
    assert m["all_pixels"]["frac_ok"] >= 0.99


def test_ray_order_changes_nothing(R):
    """Each path owns its slot and its Philox counters, so tracing the queues
    in the order of the cell sort or in queue order gives the same bits."""
    wl = scenes.nave(width=64, height=48, n_bands=8, spp=2)
    R.load(wl)
    a = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)["spectral"].cpu().numpy()
    b = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2, ray_order=1)["spectral"].cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("variant", [4, 5])
def test_other_trees_same_bits(R, variant):
    """The eight-wide tree (trace_variant 4) and the four-wide tree with 8-bit
    child boxes (5) return the same closest hits as the float four-wide
    tree, so the render is bit-identical."""
    for wl in (scenes.nave(width=64, height=48, n_bands=8, spp=2), scenes.prism_room(width=48, height=36, spp=2)):
        R.load(wl)
        a = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)["spectral"].cpu().numpy()
        b = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2, trace_variant=variant)["spectral"].cpu().numpy()
        assert np.array_equal(a, b)


def test_traversal_loop_variants_agree(R):
    """Loop shape (while-while, leaf batching or one node per step, steps
    between refills, refill threshold, leaf batch) changes only scheduling:
    closest hits are the same, sun-ray glass products may differ by float
    rounding order."""
    wl = scenes.nave(width=64, height=48, n_bands=8, spp=2)
    R.load(wl)
    base = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)["spectral"].cpu().numpy()
    for kw in (dict(trace_variant=1), dict(trace_steps=1, trace_refill=32, shadow_steps=1000, shadow_refill=32),
               dict(trace_steps=3, trace_refill=5, shadow_steps=2, shadow_refill=20),
               dict(trace_variant=2), dict(leaf_batch=1, trace_steps=1, shadow_steps=3),
               dict(leaf_batch=32, trace_steps=40, trace_refill=32, shadow_steps=7)):
        s = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2, **kw)["spectral"].cpu().numpy()
        np.testing.assert_allclose(s, base, rtol=1e-5, atol=1e-12)

"""Host BVH with spatial splits (a triangle may sit in several leaves, a
thin-glass one never) against the plain SAH build: closest hits, sun-ray
transmittances and renders are the same, since the watertight test and the
tie rule do not depend on the tree."""
import numpy as np
import pytest

from paper_1912_04000_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1912_04000_gb300.renderer import Renderer
    return Renderer(0)


def _rays(wl, n, seed):
    rng = np.random.default_rng(seed)
    lo, hi = wl.scene.verts.min(0), wl.scene.verts.max(0)
    o = lo + (hi - lo) * rng.uniform(0.02, 0.98, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    cam = wl.cameras[0]
    f = np.asarray(cam.look, np.float64) - np.asarray(cam.pos, np.float64)
    f /= np.linalg.norm(f)
    dc = f + 0.4 * rng.normal(size=(n, 3))
    dc /= np.linalg.norm(dc, axis=1, keepdims=True)
    oc = np.broadcast_to(np.asarray(cam.pos, np.float64), (n, 3))
    return (np.concatenate([o, oc]).astype(np.float32), np.concatenate([d, dc]).astype(np.float32))


@pytest.mark.parametrize("name", ["tiny_box", "nave", "crystal_nave"])
def test_hits_and_sun_rays_match_sah(R, name):
    wl = {"tiny_box": scenes.tiny_box, "nave": lambda: scenes.nave(width=64, height=48),
          "crystal_nave": lambda: scenes.crystal_nave(width=64, height=48)}[name]()
    o, d = _rays(wl, 20000, 5)
    R.load(wl, builder=0)
    t0, p0 = (x.cpu().numpy() for x in R.trace_closest(o, d))
    T0, g0 = (x.cpu().numpy() for x in R.trace_shadow(o, d, 2))
    R.load(wl, builder=2)
    info = R.scene_info()
    print(name, info)
    assert info["builder"] == "host_sbvh"
    t1, p1 = (x.cpu().numpy() for x in R.trace_closest(o, d))
    T1, g1 = (x.cpu().numpy() for x in R.trace_shadow(o, d, 2))
    assert np.array_equal(p0, p1) and np.array_equal(t0, t1)
    assert np.array_equal(g0, g1)
    np.testing.assert_allclose(T1, T0, rtol=1e-6, atol=0)


def test_renders_match_sah(R):
    wl = scenes.nave(width=64, height=48, n_bands=8, spp=2)
    R.load(wl, builder=0)
    a = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)["spectral"].cpu().numpy()
    R.load(wl, builder=2)
    b = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2)["spectral"].cpu().numpy()
    np.testing.assert_allclose(b, a, rtol=1e-5, atol=1e-12)
    # the binary-tree traversal variants run on its binary tree too
    c = R.render(wl.cameras, wl.spp, wl.depth, wl.seed, xyz_mode=2, trace_variant=1)["spectral"].cpu().numpy()
    np.testing.assert_allclose(c, a, rtol=1e-5, atol=1e-12)

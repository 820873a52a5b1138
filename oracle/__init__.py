"""CPU FP64 oracle of the spectral path tracer (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is a plain, slow reference written
from the paper (section 3 Eq. 1, section 4 Eqs. 2-3) and shares no code with the
CUDA library.  ``build()`` compiles ``oracle.cpp`` with the host compiler into
``oracle/_build/liboracle.so``; the binding below is argument marshalling only.

Every function here is pinned by the ``-m "not gpu"`` tests against closed
forms, invariants and brute force (Philox known-answer vectors, normal-incidence
Fresnel, Brewster angle, lossless-plate 2R/(1+R), Beer-Lambert, the white
furnace, the uniform sky, the sun-cone irradiance, the form factor of a square
emitter, the pinhole projection, the CIE 1931 spectral locus, brute-force
intersection; for the guided estimator: chi-square of the proposal draws
against the density it reports, the furnace and sun-cone means, exact
incident radiance in the training records).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C++17, strict IEEE double, no fast-math)."""
    srcs = [os.path.join(_HERE, "oracle.cpp"), os.path.join(_HERE, "guide_oracle.cpp")]
    deps = srcs + [os.path.join(_HERE, "guide_net.h")]
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(s) for s in deps)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
           "-fno-fast-math"] + srcs + ["-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _SceneDesc(C.Structure):
    _fields_ = [
        ("verts", C.POINTER(C.c_float)), ("n_verts", C.c_uint32),
        ("tris", C.POINTER(C.c_uint32)), ("n_tris", C.c_uint32),
        ("mat_id", C.POINTER(C.c_uint32)),
        ("mat_type", C.POINTER(C.c_int32)), ("mat_thickness", C.POINTER(C.c_float)),
        ("n_mat", C.c_uint32),
        ("lambda_nm", C.POINTER(C.c_float)), ("n_bands", C.c_uint32),
        ("sun_L", C.POINTER(C.c_float)), ("sun_dir", C.POINTER(C.c_float)),
        ("sun_half_angle", C.c_float),
        ("n_tab", C.POINTER(C.c_float)), ("k_tab", C.POINTER(C.c_float)),
        ("rho_tab", C.POINTER(C.c_float)), ("le_tab", C.POINTER(C.c_float)),
    ]


class _Camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("look", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_uint32), ("height", C.c_uint32)]


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
            L.or_philox_batch.argtypes = [C.c_uint32, C.c_uint32, C.POINTER(C.c_uint32),
                                          C.POINTER(C.c_uint32), C.c_uint64]
            L.or_fresnel.restype = C.c_double
            L.or_fresnel.argtypes = [C.c_double] * 3
            L.or_refract.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_double,
                                     C.POINTER(C.c_double)]
            L.or_refract.restype = C.c_int
            L.or_slab.argtypes = [C.c_double] * 5 + [C.POINTER(C.c_double)] * 2
            L.or_scene_create.restype = C.c_void_p
            L.or_scene_create.argtypes = [C.POINTER(_SceneDesc), C.c_int]
            L.or_scene_destroy.argtypes = [C.c_void_p]
            L.or_scene_eps.restype = C.c_double
            L.or_scene_eps.argtypes = [C.c_void_p]
            L.or_closest_hits.argtypes = [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                          C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
            L.or_shadow_transmittance.argtypes = [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                                  C.POINTER(C.c_uint32), C.c_uint64,
                                                  C.POINTER(C.c_double), C.POINTER(C.c_uint32)]
            L.or_render.restype = C.c_int
            L.or_render.argtypes = [C.c_void_p, C.POINTER(_Camera), C.c_uint32, C.c_uint32, C.c_uint32,
                                    C.c_uint32, C.c_uint32, C.c_uint64, C.POINTER(C.c_uint32), C.c_uint64,
                                    C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_uint32),
                                    C.c_int]
            L.or_render4.restype = C.c_int
            L.or_render4.argtypes = L.or_render.argtypes
            L.or_photon_records.restype = C.c_int
            L.or_photon_records.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64,
                                            C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_uint8), C.c_int]
            L.or_photon_render.restype = C.c_int
            L.or_photon_render.argtypes = [C.c_void_p, C.POINTER(_Camera), C.c_uint32, C.c_uint32, C.c_uint32,
                                           C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint32, C.c_double,
                                           C.c_double, C.c_int, C.POINTER(C.c_uint32), C.c_uint64, C.POINTER(C.c_double),
                                           C.POINTER(C.c_double), C.POINTER(C.c_uint32), C.c_int]
            L.or_xyz.argtypes = [C.POINTER(C.c_double), C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                 C.POINTER(C.c_float), C.POINTER(C.c_double)]
            L.or_hardware_threads.restype = C.c_int
            fp, dp, up = C.POINTER(C.c_float), C.POINTER(C.c_double), C.POINTER(C.c_uint32)
            L.or_guide_resolutions.argtypes = [C.c_float, C.c_float, up]
            L.or_guide_forward.argtypes = [C.c_uint32, fp, fp, C.c_float, C.c_float, fp, fp, C.c_uint64, fp, fp, up,
                                           fp, C.c_int, dp, dp, dp]
            L.or_guide_loss_grad.restype = C.c_double
            L.or_guide_loss_grad.argtypes = [C.c_uint32, fp, fp, C.c_float, C.c_float, fp, fp, C.c_uint64, fp, fp,
                                             up, fp, fp, C.c_int, dp, dp]
            L.or_guide_density.argtypes = [dp, C.c_uint64, dp, dp]
            L.or_adam_step.argtypes = [C.c_uint64, dp, dp, dp, dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                       C.c_uint32]
            L.or_guide_net_create.restype = C.c_void_p
            L.or_guide_net_create.argtypes = [C.c_uint32, fp, fp, C.c_float, C.c_float, fp, fp, C.c_int]
            L.or_guide_net_destroy.argtypes = [C.c_void_p]
            L.or_render_guided.restype = C.c_int
            L.or_render_guided.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_uint32, C.POINTER(_Camera),
                                           C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64,
                                           up, C.c_uint64, dp, dp, up, fp, C.c_int]
            L.or_guide_step.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_uint32, C.c_uint32, C.c_uint64,
                                        C.c_uint64, up, up, fp, fp, up, fp, dp]
            L.or_guide_mis_draws.argtypes = [dp, dp, C.c_double, C.c_uint64, dp, dp, dp]
            L.or_camera_rays.argtypes = [C.POINTER(_Camera), C.c_uint32, C.c_uint64, C.c_uint64, up, up, up, dp, dp]
            _lib = L
    return _lib


def philox4x32_10(key, ctr) -> np.ndarray:
    k = np.asarray(key, np.uint32)
    c = np.asarray(ctr, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_ptr(k, C.c_uint32), _ptr(c, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def philox_batch(key0: int, key1: int, ctr: np.ndarray) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    out = np.zeros_like(c)
    lib().or_philox_batch(key0, key1, _ptr(c, C.c_uint32), _ptr(out, C.c_uint32), c.shape[0])
    return out


def fresnel(cos_i: float, n: float, k: float) -> float:
    return lib().or_fresnel(cos_i, n, k)


def refract(d, n, eta):
    """Refracted unit direction of d at normal n (facing the incident side)
    into relative index eta, or None on total internal reflection."""
    L = lib()
    dd = np.ascontiguousarray(d, np.float64)
    nn = np.ascontiguousarray(n, np.float64)
    out = np.zeros(3, np.float64)
    ok = L.or_refract(_ptr(dd, C.c_double), _ptr(nn, C.c_double), float(eta), _ptr(out, C.c_double))
    return out if ok else None


def slab(cos_i, n, k, lambda_nm, d):
    rs, ts = C.c_double(), C.c_double()
    lib().or_slab(cos_i, n, k, lambda_nm, d, C.byref(rs), C.byref(ts))
    return rs.value, ts.value


def camera_rays(cameras, pixels, sample=0, band=0, seed=0):
    """Primary rays (origins, unit directions [n, 3]) of the listed global
    pixels for the given sample and band (their Philox jitter)."""
    pix = np.ascontiguousarray(pixels, np.uint32)
    n = pix.shape[0]
    s = np.ascontiguousarray(np.broadcast_to(np.asarray(sample, np.uint32), (n,)))
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(band, np.uint32), (n,)))
    o = np.zeros((n, 3))
    d = np.zeros((n, 3))
    lib().or_camera_rays(cameras_struct(cameras), len(cameras), seed, n, _ptr(pix, C.c_uint32), _ptr(s, C.c_uint32),
                         _ptr(b, C.c_uint32), _ptr(o, C.c_double), _ptr(d, C.c_double))
    return o, d


def hardware_threads() -> int:
    return int(lib().or_hardware_threads())


def cameras_struct(cameras):
    arr = (_Camera * len(cameras))()
    for i, c in enumerate(cameras):
        arr[i].pos[:] = list(map(float, c.pos))
        arr[i].look[:] = list(map(float, c.look))
        arr[i].up[:] = list(map(float, c.up))
        arr[i].vfov_deg = float(c.vfov_deg)
        arr[i].width = int(c.width)
        arr[i].height = int(c.height)
    return arr


class OracleScene:
    """FP64 reference scene built from a Scene/Spectra pair (duck-typed)."""

    def __init__(self, scene, spectra, force_brute: bool = False):
        self._keep = []

        def f32(a):
            a = np.ascontiguousarray(a, np.float32)
            self._keep.append(a)
            return _ptr(a, C.c_float)

        def u32(a):
            a = np.ascontiguousarray(a, np.uint32)
            self._keep.append(a)
            return _ptr(a, C.c_uint32)

        mt = np.ascontiguousarray(scene.mat_type, np.int32)
        self._keep.append(mt)
        d = _SceneDesc()
        d.verts = f32(scene.verts)
        d.n_verts = scene.verts.shape[0]
        d.tris = u32(scene.tris)
        d.n_tris = scene.tris.shape[0]
        d.mat_id = u32(scene.mat_id)
        d.mat_type = _ptr(mt, C.c_int32)
        d.mat_thickness = f32(scene.mat_thickness)
        d.n_mat = mt.shape[0]
        d.lambda_nm = f32(spectra.lambda_nm)
        d.n_bands = spectra.lambda_nm.shape[0]
        d.sun_L = f32(spectra.sun_L)
        d.sun_dir = f32(spectra.sun_dir)
        d.sun_half_angle = float(spectra.sun_half_angle)
        d.n_tab = f32(spectra.n)
        d.k_tab = f32(spectra.k)
        d.rho_tab = f32(spectra.rho)
        d.le_tab = f32(spectra.le)
        self.n_bands = int(d.n_bands)
        self.cmf_w = np.ascontiguousarray(spectra.cmf_w, np.float32)
        self._h = lib().or_scene_create(C.byref(d), 1 if force_brute else 0)
        self._keep = []  # the oracle copied everything

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_scene_destroy(h)
            self._h = None

    @property
    def eps(self) -> float:
        return lib().or_scene_eps(self._h)

    def closest_hits(self, o, d):
        o = np.ascontiguousarray(o, np.float32)
        d = np.ascontiguousarray(d, np.float32)
        n = o.shape[0]
        t = np.zeros(n, np.float64)
        p = np.zeros(n, np.int64)
        lib().or_closest_hits(self._h, _ptr(o, C.c_float), _ptr(d, C.c_float), n,
                              _ptr(t, C.c_double), _ptr(p, C.c_int64))
        return t, p

    def shadow_transmittance(self, o, d, band):
        o = np.ascontiguousarray(o, np.float32)
        d = np.ascontiguousarray(d, np.float32)
        n = o.shape[0]
        b = np.ascontiguousarray(np.broadcast_to(np.asarray(band, np.uint32), (n,)))
        T = np.zeros(n, np.float64)
        g = np.zeros(n, np.uint32)
        lib().or_shadow_transmittance(self._h, _ptr(o, C.c_float), _ptr(d, C.c_float),
                                      _ptr(b, C.c_uint32), n, _ptr(T, C.c_double), _ptr(g, C.c_uint32))
        return T, g

    def render(self, cameras, spp, depth, seed=0, band_first=0, band_count=None, pixels=None,
               record_paths=False, n_threads=0, bands_per_path=1):
        """FP64 spectral sums over samples for the listed global pixels.

        Returns dict(spectral_sum [n_pix, band_count], xyz [n_pix, 3], and with
        record_paths path_L / path_sig [n_pix, spp, band_count]).
        bands_per_path = 4: every path carries four consecutive bands."""
        if bands_per_path not in (1, 4):
            raise ValueError("bands_per_path is 1 or 4")
        if band_count is None:
            band_count = self.n_bands - band_first
        n_all = sum(c.width * c.height for c in cameras)
        pix = np.arange(n_all, dtype=np.uint32) if pixels is None else np.ascontiguousarray(pixels, np.uint32)
        npx = pix.shape[0]
        ssum = np.zeros((npx, band_count), np.float64)
        pl = np.zeros((npx, spp, band_count), np.float64) if record_paths else None
        ps = np.zeros((npx, spp, band_count), np.uint32) if record_paths else None
        cams = cameras_struct(cameras)
        fn = lib().or_render if bands_per_path == 1 else lib().or_render4
        rc = fn(self._h, cams, len(cameras), band_first, band_count, spp, depth, seed,
                             _ptr(pix, C.c_uint32), npx, _ptr(ssum, C.c_double),
                             _ptr(pl, C.c_double) if pl is not None else None,
                             _ptr(ps, C.c_uint32) if ps is not None else None, n_threads)
        if rc != 0:
            raise ValueError(f"or_render failed ({rc})")
        out = {"spectral_sum": ssum, "xyz": xyz(ssum, band_first, spp, self.cmf_w)}
        if record_paths:
            out["path_L"] = pl
            out["path_sig"] = ps
        return out


PHOTON_CLASSES = {0: "empty", 1: "direct", 2: "caustic", 3: "indirect"}


def _photon_methods():
    def photon_records(self, n_photons, depth, seed=0, band_first=0, band_count=None, n_threads=0, emission=0):
        """Photon pass: pos_phi [band_count, n_photons, depth, 4] (position,
        flux) and cls (0 empty, 1 direct, 2 caustic, 3 indirect); emission 0 =
        disk, 1 = through the thin-glass portals."""
        if band_count is None:
            band_count = self.n_bands - band_first
        n = band_count * n_photons * depth
        pos = np.zeros((n, 4), np.float64)
        cls = np.zeros(n, np.uint8)
        rc = lib().or_photon_records(self._h, band_first, band_count, n_photons, depth, seed, emission,
                                     _ptr(pos, C.c_double), _ptr(cls, C.c_uint8), n_threads)
        if rc != 0:
            raise ValueError(f"or_photon_records failed ({rc})")
        return pos.reshape(band_count, n_photons, depth, 4), cls.reshape(band_count, n_photons, depth)

    def render_photons(self, cameras, spp, depth, seed=0, n_photons=1 << 14, photon_depth=4, r_caustic=0.05,
                       r_global=0.2, band_first=0, band_count=None, pixels=None, record_paths=False, n_threads=0,
                       emission=0):
        """Photon-mapping estimate of the listed pixels (layout as render)."""
        if band_count is None:
            band_count = self.n_bands - band_first
        n_all = sum(c.width * c.height for c in cameras)
        pix = np.arange(n_all, dtype=np.uint32) if pixels is None else np.ascontiguousarray(pixels, np.uint32)
        npx = pix.shape[0]
        ssum = np.zeros((npx, band_count), np.float64)
        pl = np.zeros((npx, spp, band_count), np.float64) if record_paths else None
        ps = np.zeros((npx, spp, band_count), np.uint32) if record_paths else None
        rc = lib().or_photon_render(self._h, cameras_struct(cameras), len(cameras), band_first, band_count, spp, depth,
                                    seed, n_photons, photon_depth, r_caustic, r_global, emission,
                                    _ptr(pix, C.c_uint32), npx,
                                    _ptr(ssum, C.c_double), _ptr(pl, C.c_double) if pl is not None else None,
                                    _ptr(ps, C.c_uint32) if ps is not None else None, n_threads)
        if rc != 0:
            raise ValueError(f"or_photon_render failed ({rc})")
        out = {"spectral_sum": ssum, "xyz": xyz(ssum, band_first, spp, self.cmf_w)}
        if record_paths:
            out["path_L"] = pl
            out["path_sig"] = ps
        return out

    return photon_records, render_photons


def xyz(spectral_sum, band_first, spp, cmf_w) -> np.ndarray:
    s = np.ascontiguousarray(spectral_sum, np.float64)
    npx, bc = s.shape
    w = np.ascontiguousarray(cmf_w, np.float32)
    out = np.zeros((npx, 3), np.float64)
    lib().or_xyz(_ptr(s, C.c_double), npx, band_first, bc, spp, _ptr(w, C.c_float), _ptr(out, C.c_double))
    return out


# ---------------------------------------------------------------------------
# learned guide (hash grid + MLP + vMF mixture), FP64
# ---------------------------------------------------------------------------
GUIDE_W_SIZE = 64 * 64 * 3 + 64 * 48
GUIDE_LEVELS = 8
GUIDE_FEATURES = 4  # hash-grid features per level


def guide_resolutions(n_min=16.0, n_max=2048.0):
    r = np.zeros(GUIDE_LEVELS, np.uint32)
    lib().or_guide_resolutions(n_min, n_max, _ptr(r, C.c_uint32))
    return r


def _f32(a):
    return np.ascontiguousarray(a, np.float32)


def guide_forward(log2_T, lo, hi, grid, W, pos, nrm, group, omega, n_min=16.0, n_max=2048.0, bf16_act=False):
    """X [n, 64], Y [n, 48], q(omega) [n].  bf16_act: the BF16 network (layer
    inputs rounded to BF16 before each product)."""
    lo, hi, grid, W, pos, nrm, omega = map(_f32, (lo, hi, grid, W, pos, nrm, omega))
    g = np.ascontiguousarray(group, np.uint32)
    n = pos.shape[0]
    X = np.zeros((n, 64))
    Y = np.zeros((n, 48))
    q = np.zeros(n)
    fp = lambda a: _ptr(a, C.c_float)
    dp = lambda a: _ptr(a, C.c_double)
    lib().or_guide_forward(log2_T, fp(lo), fp(hi), n_min, n_max, fp(grid), fp(W), n, fp(pos), fp(nrm),
                           _ptr(g, C.c_uint32), fp(omega), 1 if bf16_act else 0, dp(X), dp(Y), dp(q))
    return X, Y, q


def guide_loss_grad(log2_T, lo, hi, grid, W, pos, nrm, group, omega, wt, n_min=16.0, n_max=2048.0, bf16_act=False):
    """(loss, dW [GUIDE_W_SIZE], dgrid [8 * 2^log2_T * 4])."""
    lo, hi, grid, W, pos, nrm, omega, wt = map(_f32, (lo, hi, grid, W, pos, nrm, omega, wt))
    g = np.ascontiguousarray(group, np.uint32)
    n = pos.shape[0]
    dW = np.zeros(GUIDE_W_SIZE)
    dgrid = np.zeros(GUIDE_LEVELS * (1 << log2_T) * GUIDE_FEATURES)
    fp = lambda a: _ptr(a, C.c_float)
    dp = lambda a: _ptr(a, C.c_double)
    loss = lib().or_guide_loss_grad(log2_T, fp(lo), fp(hi), n_min, n_max, fp(grid), fp(W), n, fp(pos), fp(nrm),
                                    _ptr(g, C.c_uint32), fp(omega), fp(wt), 1 if bf16_act else 0, dp(dW),
                                    dp(dgrid))
    return loss, dW, dgrid


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.99, eps=1e-15):
    """One Adam step on float64 arrays p, m, v (updated in place) with gradient g at step t >= 1."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, np.float64)
    dp = lambda a: _ptr(a, C.c_double)
    lib().or_adam_step(p.size, dp(p), dp(g), dp(m), dp(v), lr, b1, b2, eps, t)


def guide_density(Y, omega):
    Y = np.ascontiguousarray(Y, np.float64)
    om = np.ascontiguousarray(omega, np.float64)
    q = np.zeros(om.shape[0])
    lib().or_guide_density(_ptr(Y, C.c_double), om.shape[0], _ptr(om, C.c_double), _ptr(q, C.c_double))
    return q


OracleScene.photon_records, OracleScene.render_photons = _photon_methods()


class OracleGuide:
    """The guide network in FP64 for the guided estimator (BF16 network when
    bf16_act: layer inputs rounded to BF16 before each product)."""

    def __init__(self, log2_T, lo, hi, grid, W, n_min=16.0, n_max=2048.0, bf16_act=True):
        lo, hi, grid, W = map(_f32, (lo, hi, grid, W))
        if grid.size != GUIDE_LEVELS * (1 << log2_T) * GUIDE_FEATURES or W.size != GUIDE_W_SIZE:
            raise ValueError("guide parameter sizes")
        fp = lambda a: _ptr(a, C.c_float)
        self._h = lib().or_guide_net_create(log2_T, fp(lo), fp(hi), n_min, n_max, fp(grid), fp(W),
                                            1 if bf16_act else 0)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_guide_net_destroy(h)
            self._h = None


STEP_FIELDS = ("omega_x", "omega_y", "omega_z", "q", "pdf", "cos", "guide", "lobe", "lobe_margin", "nee_w", "esc_w",
               "cont", "q_sun", "pdf_sun")


def _guided_methods():
    def render_guided(self, guide, cameras, spp, depth, seed=0, alpha=0.7, guide_depth=2, band_first=0,
                      band_count=None, pixels=None, record_paths=False, records=False, n_threads=0):
        """Guided estimate of the listed pixels (layout as render); with
        records, the training records [n_pix, spp, band_count, guide_depth, 2, 12]."""
        if band_count is None:
            band_count = self.n_bands - band_first
        n_all = sum(c.width * c.height for c in cameras)
        pix = np.arange(n_all, dtype=np.uint32) if pixels is None else np.ascontiguousarray(pixels, np.uint32)
        npx = pix.shape[0]
        ssum = np.zeros((npx, band_count), np.float64)
        pl = np.zeros((npx, spp, band_count), np.float64) if record_paths else None
        ps = np.zeros((npx, spp, band_count), np.uint32) if record_paths else None
        rec = np.zeros((npx, spp, band_count, guide_depth, 2, 12), np.float32) if records else None
        rc = lib().or_render_guided(self._h, guide._h, alpha, guide_depth, cameras_struct(cameras), len(cameras),
                                    band_first, band_count, spp, depth, seed, _ptr(pix, C.c_uint32), npx,
                                    _ptr(ssum, C.c_double), _ptr(pl, C.c_double) if pl is not None else None,
                                    _ptr(ps, C.c_uint32) if ps is not None else None,
                                    _ptr(rec, C.c_float) if rec is not None else None, n_threads)
        if rc != 0:
            raise ValueError(f"or_render_guided failed ({rc})")
        out = {"spectral_sum": ssum, "xyz": xyz(ssum, band_first, spp, self.cmf_w)}
        if record_paths:
            out["path_L"] = pl
            out["path_sig"] = ps
        if records:
            out["records"] = rec
        return out

    def guide_step(self, guide, k, sample, seed, pixel, band, po, nrm, has_sun, wn, alpha=0.7):
        """One guided vertex per query (see or_guide_step): dict of arrays
        named by STEP_FIELDS."""
        pixel = np.ascontiguousarray(pixel, np.uint32)
        n = pixel.shape[0]
        band = np.ascontiguousarray(band, np.uint32)
        hs = np.ascontiguousarray(has_sun, np.uint32)
        po, nrm, wn = (np.ascontiguousarray(a, np.float32) for a in (po, nrm, wn))
        out = np.zeros((n, 16))
        lib().or_guide_step(self._h, guide._h, alpha, k, sample, seed, n, _ptr(pixel, C.c_uint32),
                            _ptr(band, C.c_uint32), _ptr(po, C.c_float), _ptr(nrm, C.c_float), _ptr(hs, C.c_uint32),
                            _ptr(wn, C.c_float), _ptr(out, C.c_double))
        return {f: out[:, i] for i, f in enumerate(STEP_FIELDS)} | {"omega": out[:, 0:3]}

    return render_guided, guide_step


OracleScene.render_guided, OracleScene.guide_step = _guided_methods()


def guide_mis_draws(Y, normal, alpha, u):
    """One-sample MIS draws for fixed head outputs Y [48] and normal from
    uniforms u [n, 6]: (omega [n, 3], p_mix(omega) [n])."""
    Y = np.ascontiguousarray(Y, np.float64)
    nn = np.ascontiguousarray(normal, np.float64)
    u = np.ascontiguousarray(u, np.float64).reshape(-1, 6)
    n = u.shape[0]
    om = np.zeros((n, 3))
    pdf = np.zeros(n)
    dp = lambda a: _ptr(a, C.c_double)
    lib().or_guide_mis_draws(dp(Y), dp(nn), alpha, n, dp(u), dp(om), dp(pdf))
    return om, pdf

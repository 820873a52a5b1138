"""Seeded synthetic inputs for the spectral path tracer.

This module only *describes* scenes: triangle geometry, per-material spectral
tables, the sun, the colour-matching weights and the cameras.  It holds none of
the renderer's arithmetic (no intersection, no Fresnel, no sampling, no
estimator); both the CUDA library and the CPU reference consume what it builds.

Workloads (the paper renders the interior of a church lit by the sun through
its windows, section 3 and section 6):

* ``tiny_box``   - closed 12-triangle box; the two triangles of the sun-facing
  wall are a 1 cm thin-glass sheet with Cauchy n = 1.5 + 0.004/lambda^2 (um),
  k = 1e-6; stone albedo 0.7; 0.5 rad (full apex) sun cone, 5778 K spectrum.
* ``nave``       - procedural nave 80 x 25 x 20 m (x length, y up, z width)
  with 24 tessellated columns and 16 pointed-arch windows glazed with seeded
  smooth n(lambda) in [1.45, 1.6], k(lambda) in [1e-7, 1e-5]; about 200k
  triangles.
* ``large_nave`` - the same nave with finer columns (about 2M triangles),
  40 leaded stained-glass windows (per-pane seeded Gaussian absorption bands in
  k) and metal fittings (conductor, k in [2, 6]).
* ``furnace_box``, ``plate_under_sky``, ``slab_view`` - small closed-form test
  scenes (white furnace, uniform sky, Beer-Lambert through a sheet).

Readings fixed here: y is up; the sun cone "0.5 rad" is the full apex angle,
so the half angle is 0.25 rad; bands are point samples with inclusive ends;
colour matching uses the analytic multi-lobe fit of Wyman, Sloan and Shirley
(JCGT 2013) with trapezoid band weights, normalised so a flat unit spectrum
has Y = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

LAMBERT, THIN_GLASS, CONDUCTOR, EMISSIVE, DIELECTRIC = 0, 1, 2, 3, 4


@dataclass
class Scene:
    verts: np.ndarray          # float32 [nv, 3], metres
    tris: np.ndarray           # uint32 [nt, 3]
    mat_id: np.ndarray         # uint32 [nt]
    mat_type: np.ndarray       # int32 [n_mat]
    mat_thickness: np.ndarray  # float32 [n_mat], metres (thin glass only)

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_mat(self) -> int:
        return int(self.mat_type.shape[0])


@dataclass
class Spectra:
    lambda_nm: np.ndarray      # float32 [B]
    sun_L: np.ndarray          # float32 [B], radiance inside the sun cone
    sun_dir: np.ndarray        # float32 [3], unit vector towards the sun
    sun_half_angle: float      # radians
    n: np.ndarray              # float32 [n_mat, B]
    k: np.ndarray              # float32 [n_mat, B]
    rho: np.ndarray            # float32 [n_mat, B]
    le: np.ndarray             # float32 [n_mat, B] (emissive test material)
    cmf_w: np.ndarray          # float32 [B, 3]

    @property
    def n_bands(self) -> int:
        return int(self.lambda_nm.shape[0])


@dataclass
class Camera:
    pos: Tuple[float, float, float]
    look: Tuple[float, float, float]
    up: Tuple[float, float, float]
    vfov_deg: float
    width: int
    height: int

    @property
    def n_pixels(self) -> int:
        return self.width * self.height


@dataclass
class Workload:
    name: str
    scene: Scene
    spectra: Spectra
    cameras: List[Camera]
    spp: int
    depth: int
    seed: int = 0
    band_first: int = 0
    band_count: int = -1

    def __post_init__(self):
        if self.band_count < 0:
            self.band_count = self.spectra.n_bands

    @property
    def n_pixels(self) -> int:
        return sum(c.n_pixels for c in self.cameras)

    @property
    def n_paths(self) -> int:
        return self.n_pixels * self.spp * self.band_count


# ----------------------------------------------------------------------------
# spectra tables
# ----------------------------------------------------------------------------

def band_wavelengths(lmin: float, lmax: float, n_bands: int) -> np.ndarray:
    """Point-sampled bands with inclusive ends: 16 in 400-700 nm are 20 nm apart,
    81 in 380-780 nm are 5 nm apart."""
    if n_bands == 1:
        return np.array([0.5 * (lmin + lmax)], np.float64)
    return lmin + (lmax - lmin) * np.arange(n_bands, dtype=np.float64) / (n_bands - 1)


def planck(lambda_nm: np.ndarray, temp_k: float) -> np.ndarray:
    """Black-body spectral radiance (W sr^-1 m^-3)."""
    h, c, kb = 6.62607015e-34, 2.99792458e8, 1.380649e-23
    lam = np.asarray(lambda_nm, np.float64) * 1e-9
    return 2.0 * h * c * c / lam ** 5 / np.expm1(h * c / (lam * kb * temp_k))


def rayleigh_optical_depth(lambda_nm: np.ndarray) -> np.ndarray:
    """Vertical Rayleigh optical depth of the standard sea-level atmosphere,
    Hansen and Travis (Space Sci. Rev. 16, 1974) fit with lambda in um:
    tau = 0.008569 lambda^-4 (1 + 0.0113 lambda^-2 + 0.00013 lambda^-4)."""
    l2 = (np.asarray(lambda_nm, np.float64) * 1e-3) ** -2
    return 0.008569 * l2 * l2 * (1.0 + 0.0113 * l2 + 0.00013 * l2 * l2)


def air_mass(elevation_deg: float) -> float:
    """Relative optical air mass at solar elevation h (degrees), Kasten and
    Young (Appl. Opt. 28, 1989): 1 / (sin h + 0.50572 (h + 6.07995)^-1.6364)."""
    h = float(elevation_deg)
    if not -6.0 < h <= 90.0:
        raise ValueError("elevation out of range")
    return 1.0 / (math.sin(math.radians(h)) + 0.50572 * (h + 6.07995) ** -1.6364)


def sun_spectrum(lambda_nm: np.ndarray, temp_k: float = 5778.0, elevation_deg: Optional[float] = None) -> np.ndarray:
    """Sun radiance inside its cone: black body normalised to 1 at 560 nm.
    With an elevation, the direct beam is attenuated by Rayleigh scattering
    along the air mass of that elevation, exp(-tau(lambda) m(h)) (section 3:
    the sun's spectrum seen from the ground changes with the hour of the
    day; a low sun is redder)."""
    s = planck(lambda_nm, temp_k) / planck(np.array([560.0]), temp_k)[0]
    if elevation_deg is not None:
        s = s * np.exp(-rayleigh_optical_depth(lambda_nm) * air_mass(elevation_deg))
    return s


def _lobe(lam, mu, s1, s2):
    s = np.where(lam < mu, s1, s2)
    t = (lam - mu) / s
    return np.exp(-0.5 * t * t)


def cie_cmf_fit(lambda_nm: np.ndarray) -> np.ndarray:
    """CIE 1931 2-degree colour matching functions, multi-lobe piecewise
    Gaussian fit of Wyman, Sloan and Shirley (JCGT 2(2), 2013). [B, 3]."""
    lam = np.asarray(lambda_nm, np.float64)
    x = (1.056 * _lobe(lam, 599.8, 37.9, 31.0) + 0.362 * _lobe(lam, 442.0, 16.0, 26.7)
         - 0.065 * _lobe(lam, 501.1, 20.4, 26.2))
    y = 0.821 * _lobe(lam, 568.8, 46.9, 40.5) + 0.286 * _lobe(lam, 530.9, 16.3, 31.1)
    z = 1.217 * _lobe(lam, 437.0, 11.8, 36.0) + 0.681 * _lobe(lam, 459.0, 26.0, 13.8)
    return np.stack([x, y, z], axis=1)


def xyz_weights(lambda_nm: np.ndarray) -> np.ndarray:
    """cmf_w[b, c] = w_b cmf_c(lambda_b) / sum_b w_b ybar(lambda_b), with
    trapezoid weights w_b (ends halved), so a flat unit spectrum has Y = 1."""
    lam = np.asarray(lambda_nm, np.float64)
    B = lam.shape[0]
    if B == 1:
        w = np.ones(1)
    else:
        dl = lam[1] - lam[0]
        w = np.full(B, dl)
        w[0] *= 0.5
        w[-1] *= 0.5
    cmf = cie_cmf_fit(lam)
    return (w[:, None] * cmf) / float(np.sum(w * cmf[:, 1]))


def cauchy_n(lambda_nm: np.ndarray, a: float, b: float) -> np.ndarray:
    """n(lambda) = a + b / lambda^2 with lambda in micrometres."""
    lum = np.asarray(lambda_nm, np.float64) * 1e-3
    return a + b / (lum * lum)


def smooth_random_spectrum(rng: np.random.Generator, lambda_nm: np.ndarray, lo: float,
                           hi: float, terms: int = 4) -> np.ndarray:
    """Seeded smooth spectrum in [lo, hi]: a 4-term cosine series clamped."""
    lam = np.asarray(lambda_nm, np.float64)
    x = (lam - 380.0) / 400.0
    mid = rng.uniform(lo, hi)
    s = np.full_like(x, mid)
    amp = 0.5 * (hi - lo)
    for j in range(1, terms + 1):
        s += amp / j * rng.uniform(-0.7, 0.7) * np.cos(math.pi * j * x + rng.uniform(0, 2 * math.pi))
    return np.clip(s, lo, hi)


def smooth_log_spectrum(rng, lambda_nm, lo, hi, terms=3):
    """Seeded smooth spectrum whose log lies in [log lo, log hi]."""
    return np.exp(smooth_random_spectrum(rng, lambda_nm, math.log(lo), math.log(hi), terms))


def sun_direction(elevation_deg: float, azimuth_deg: float) -> np.ndarray:
    """Unit vector towards the sun; azimuth 0 points to -z (through the z = 0 wall)."""
    el, az = math.radians(elevation_deg), math.radians(azimuth_deg)
    return np.array([math.cos(el) * math.sin(az), math.sin(el), -math.cos(el) * math.cos(az)])


# ----------------------------------------------------------------------------
# geometry helpers
# ----------------------------------------------------------------------------

class MeshBuilder:
    """Collects triangles; vertices are shared by exact coordinate so that
    neighbouring triangles meet on bitwise-identical edges."""

    def __init__(self):
        self._vid = {}
        self.verts: List[Tuple[float, float, float]] = []
        self.tris: List[Tuple[int, int, int]] = []
        self.mats: List[int] = []

    def v(self, p) -> int:
        key = (float(np.float32(p[0])), float(np.float32(p[1])), float(np.float32(p[2])))
        i = self._vid.get(key)
        if i is None:
            i = len(self.verts)
            self._vid[key] = i
            self.verts.append(key)
        return i

    def tri(self, a, b, c, mat: int):
        self.tris.append((self.v(a), self.v(b), self.v(c)))
        self.mats.append(mat)

    def quad(self, a, b, c, d, mat: int):
        self.tri(a, b, c, mat)
        self.tri(a, c, d, mat)

    def add_arrays(self, verts: np.ndarray, tris: np.ndarray, mat: int):
        """Bulk-append an indexed mesh (no sharing with existing vertices)."""
        base = len(self.verts)
        self.verts.extend(map(tuple, verts.astype(np.float32).astype(np.float64).tolist()))
        self.tris.extend(map(tuple, (tris + base).tolist()))
        self.mats.extend([mat] * len(tris))

    def build(self, mat_type, mat_thickness) -> Scene:
        return Scene(
            verts=np.asarray(self.verts, np.float32).reshape(-1, 3),
            tris=np.asarray(self.tris, np.uint32).reshape(-1, 3),
            mat_id=np.asarray(self.mats, np.uint32),
            mat_type=np.asarray(mat_type, np.int32),
            mat_thickness=np.asarray(mat_thickness, np.float32),
        )


def _box_quads(mb: MeshBuilder, lo, hi, mats):
    """Six faces of an axis-aligned box; mats = (x0, x1, y0, y1, z0, z1)."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    mb.quad((x0, y0, z0), (x0, y1, z0), (x0, y1, z1), (x0, y0, z1), mats[0])
    mb.quad((x1, y0, z0), (x1, y0, z1), (x1, y1, z1), (x1, y1, z0), mats[1])
    mb.quad((x0, y0, z0), (x0, y0, z1), (x1, y0, z1), (x1, y0, z0), mats[2])
    mb.quad((x0, y1, z0), (x1, y1, z0), (x1, y1, z1), (x0, y1, z1), mats[3])
    mb.quad((x0, y0, z0), (x1, y0, z0), (x1, y1, z0), (x0, y1, z0), mats[4])
    mb.quad((x0, y0, z1), (x0, y1, z1), (x1, y1, z1), (x1, y0, z1), mats[5])


def _solid(mb: MeshBuilder, faces, mat):
    """Closed solid from planar polygons (lists of points); each face is fanned
    into triangles and wound so that its normal points away from the solid's
    centroid (the dielectric's side test reads the winding)."""
    pts = np.array([p for f in faces for p in f], np.float64)
    ctr = pts.mean(0)
    for f in faces:
        f = [np.asarray(q, np.float64) for q in f]
        nrm = np.cross(f[1] - f[0], f[2] - f[0])
        if np.dot(nrm, f[0] - ctr) < 0.0:
            f = f[::-1]
        for j in range(1, len(f) - 1):
            mb.tri(f[0], f[j], f[j + 1], mat)


def _solid_box(mb: MeshBuilder, lo, hi, mat):
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    _solid(mb, [[(x0, y0, z0), (x0, y1, z0), (x0, y1, z1), (x0, y0, z1)],
                [(x1, y0, z0), (x1, y1, z0), (x1, y1, z1), (x1, y0, z1)],
                [(x0, y0, z0), (x1, y0, z0), (x1, y0, z1), (x0, y0, z1)],
                [(x0, y1, z0), (x1, y1, z0), (x1, y1, z1), (x0, y1, z1)],
                [(x0, y0, z0), (x1, y0, z0), (x1, y1, z0), (x0, y1, z0)],
                [(x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)]], mat)


def _flat_spectra(n_mat, B):
    z = np.zeros((n_mat, B), np.float64)
    return z.copy(), z.copy(), z.copy(), z.copy()


def _spectra(lam, sun_L, sun_dir, half, n, k, rho, le) -> Spectra:
    return Spectra(
        lambda_nm=np.asarray(lam, np.float32),
        sun_L=np.asarray(sun_L, np.float32),
        sun_dir=np.asarray(sun_dir / np.linalg.norm(sun_dir), np.float32),
        sun_half_angle=float(half),
        n=np.asarray(n, np.float32), k=np.asarray(k, np.float32),
        rho=np.asarray(rho, np.float32), le=np.asarray(le, np.float32),
        cmf_w=np.asarray(xyz_weights(lam), np.float32),
    )


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def tiny_box(width=128, height=128, n_bands=16, spp=4, depth=4, seed=0) -> Workload:
    """12-triangle closed box 4 x 3 x 5 m; the z = 5 wall is thin glass."""
    mb = MeshBuilder()
    STONE, GLASS = 0, 1
    _box_quads(mb, (0.0, 0.0, 0.0), (4.0, 3.0, 5.0), (STONE, STONE, STONE, STONE, STONE, GLASS))
    scene = mb.build([LAMBERT, THIN_GLASS], [0.0, 0.01])
    lam = band_wavelengths(400.0, 700.0, n_bands)
    n, k, rho, le = _flat_spectra(2, n_bands)
    rho[STONE] = 0.7
    n[GLASS] = cauchy_n(lam, 1.5, 0.004)
    k[GLASS] = 1e-6
    n[STONE] = 1.0
    sun = sun_direction(35.0, 200.0)  # sun behind the z = 5 glass wall
    spec = _spectra(lam, sun_spectrum(lam), sun, 0.25, n, k, rho, le)
    cam = Camera((2.0, 1.5, 0.3), (2.0, 1.0, 5.0), (0.0, 1.0, 0.0), 60.0, width, height)
    return Workload("tiny_box", scene, spec, [cam], spp, depth, seed)


def prism_room(width=96, height=72, n_bands=16, spp=4, depth=8, seed=0) -> Workload:
    """The tiny box room (sunlight through the thin-glass z = 5 wall) with a
    solid triangular prism of dispersive flint-like glass on the floor in the
    sun patch: refraction with n(lambda), total internal reflection and
    Beer-Lambert absorption inside.  20 triangles."""
    mb = MeshBuilder()
    STONE, GLASS, PRISM = 0, 1, 2
    _box_quads(mb, (0.0, 0.0, 0.0), (4.0, 3.0, 5.0), (STONE, STONE, STONE, STONE, STONE, GLASS))
    # equilateral cross-section in x-y, 0.8 m wide, extruded along z
    a, h = 0.8, 0.8 * math.sqrt(3.0) / 2.0
    x0, z0, z1 = 1.6, 2.6, 3.6
    tri0 = [(x0, 0.001, z0), (x0 + a, 0.001, z0), (x0 + 0.5 * a, 0.001 + h, z0)]
    tri1 = [(x, y, z1) for (x, y, _) in tri0]
    faces = [tri0, tri1] + [[tri0[i], tri0[(i + 1) % 3], tri1[(i + 1) % 3], tri1[i]] for i in range(3)]
    _solid(mb, faces, PRISM)
    scene = mb.build([LAMBERT, THIN_GLASS, DIELECTRIC], [0.0, 0.01, 0.0])
    lam = band_wavelengths(400.0, 700.0, n_bands)
    n, k, rho, le = _flat_spectra(3, n_bands)
    rho[STONE] = 0.7
    n[STONE] = 1.0
    n[GLASS] = cauchy_n(lam, 1.5, 0.004)
    k[GLASS] = 1e-6
    n[PRISM] = cauchy_n(lam, 1.62, 0.012)
    k[PRISM] = 2e-8
    sun = sun_direction(35.0, 200.0)
    spec = _spectra(lam, sun_spectrum(lam, elevation_deg=35.0), sun, 0.25, n, k, rho, le)
    cam = Camera((3.4, 1.4, 0.6), (2.0, 0.3, 3.1), (0.0, 1.0, 0.0), 45.0, width, height)
    return Workload("prism_room", scene, spec, [cam], spp, depth, seed)


def solid_slab_view(n_glass=1.5, k_glass=2e-6, thickness=0.01, lambda_nm=(450.0, 550.0, 650.0),
                    tilt_deg=30.0, spp=256, depth=8, seed=7) -> Workload:
    """Camera looks through a wide solid slab of refracting glass (a closed
    6 x 6 m box of the given thickness, tilted about x) at the sun behind it.
    Both faces are parallel, so every transmitted path leaves in its original
    direction; summing the internal reflections, the pixel's expectation is
    the thin-sheet T_s(theta) L_sun of the same glass."""
    mb = MeshBuilder()
    t = math.radians(tilt_deg)
    ay = np.array([0.0, math.cos(t), -math.sin(t)])
    nz = np.array([0.0, math.sin(t), math.cos(t)])
    ax = np.array([1.0, 0.0, 0.0])
    corners = lambda off: [s1 * 3.0 * ax + s2 * 3.0 * ay + off * nz for s1, s2 in ((-1, -1), (1, -1), (1, 1), (-1, 1))]
    lo_f, hi_f = corners(-0.5 * thickness), corners(0.5 * thickness)
    faces = [lo_f, hi_f] + [[lo_f[i], lo_f[(i + 1) % 4], hi_f[(i + 1) % 4], hi_f[i]] for i in range(4)]
    _solid(mb, faces, 0)
    scene = mb.build([DIELECTRIC], [0.0])
    lam = np.asarray(lambda_nm, np.float64)
    B = lam.shape[0]
    n, k, rho, le = _flat_spectra(1, B)
    n[0] = n_glass
    k[0] = k_glass
    spec = _spectra(lam, np.ones(B), np.array([0.0, 0.0, 1.0]), 0.2, n, k, rho, le)
    cam = Camera((0.0, 0.0, -2.0), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0), 0.05, 2, 2)
    return Workload("solid_slab_view", scene, spec, [cam], spp, depth, seed)


def dielectric_furnace(albedo=0.3, le=1.0, n_bands=3, width=8, height=8, spp=4, depth=64, seed=11) -> Workload:
    """The furnace box (walls emit le (1 - albedo), Lambertian albedo) with a
    lossless refracting cube inside.  Refraction and reflection keep the
    throughput, so a path returns le (1 - albedo^m) for its m Lambertian
    vertices: within 1e-6 of le once m >= 12."""
    mb = MeshBuilder()
    _box_quads(mb, (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), (0,) * 6)
    _solid_box(mb, (-0.3, -0.35, -0.25), (0.25, 0.2, 0.3), 1)
    scene = mb.build([EMISSIVE, DIELECTRIC], [0.0, 0.0])
    lam = band_wavelengths(450.0, 650.0, n_bands)
    n, k, rho, lt = _flat_spectra(2, n_bands)
    rho[0] = albedo
    lt[0] = le * (1.0 - albedo)
    n[1] = cauchy_n(lam, 1.5, 0.004)
    spec = _spectra(lam, np.ones(n_bands), np.array([0.3, 0.8, 0.2]), 0.25, n, k, rho, lt)
    cam = Camera((0.6, 0.5, 0.7), (-0.1, -0.1, 0.0), (0.0, 1.0, 0.0), 50.0, width, height)
    return Workload("dielectric_furnace", scene, spec, [cam], spp, depth, seed)


def furnace_box(albedo=0.5, le=1.0, n_bands=4, width=16, height=16, spp=2, depth=5,
                seed=3) -> Workload:
    """Closed box whose walls emit le*(1-albedo) with Lambertian albedo: every
    path returns exactly le*(1 - albedo^depth) (zero variance)."""
    mb = MeshBuilder()
    _box_quads(mb, (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), (0,) * 6)
    scene = mb.build([EMISSIVE], [0.0])
    lam = band_wavelengths(400.0, 700.0, n_bands)
    n, k, rho, lt = _flat_spectra(1, n_bands)
    rho[0] = albedo
    lt[0] = le * (1.0 - albedo)
    spec = _spectra(lam, np.ones(n_bands), np.array([0.3, 0.8, 0.2]), 0.25, n, k, rho, lt)
    cam = Camera((0.1, -0.2, 0.05), (0.7, 0.3, -0.9), (0.0, 1.0, 0.0), 70.0, width, height)
    return Workload("furnace_box", scene, spec, [cam], spp, depth, seed)


def plate_under_sky(n_bands=2, width=8, height=8, spp=64, depth=3, seed=5, rho=1.0,
                    sun_half_angle=math.pi, sun_dir=(0.0, 1.0, 0.0)) -> Workload:
    """Single Lambertian square (y = 0) under a unit sun cone.  With half angle
    pi (a uniform sky) and rho = 1 every pixel has expectation exactly 1; with
    a cone of half angle a whose axis makes angle s with the normal (cone above
    the horizon) a pixel on the plate has expectation rho sin^2(a) cos(s)."""
    mb = MeshBuilder()
    mb.quad((-1.0, 0.0, -1.0), (1.0, 0.0, -1.0), (1.0, 0.0, 1.0), (-1.0, 0.0, 1.0), 0)
    scene = mb.build([LAMBERT], [0.0])
    lam = band_wavelengths(500.0, 600.0, n_bands)
    n, k, rt, le = _flat_spectra(1, n_bands)
    rt[0] = rho
    spec = _spectra(lam, np.ones(n_bands), np.asarray(sun_dir, np.float64), sun_half_angle, n, k, rt, le)
    cam = Camera((0.0, 2.0, 0.0), (0.0, 0.0, 0.05), (0.0, 0.0, 1.0), 40.0, width, height)
    return Workload("plate_under_sky", scene, spec, [cam], spp, depth, seed)


def emitter_over_plate(half=1.0, height=2.0, rho=0.8, le=1.0, n_bands=2, width=4, height_px=4, spp=1024,
                       seed=13) -> Workload:
    """Cosine-continuation test: a 20 x 20 m Lambertian floor (y = 0, rho)
    under a square emitter of half side `half` centred at height `height`
    (emissive test material, rho 0, radiance le on both faces), no sun
    (L_sun = 0).  The camera sees a sub-millimetre patch of the floor at the
    origin; at depth 2 a path adds rho le exactly when its cosine-sampled
    continuation hits the emitter, so a pixel's expectation is rho le F with F
    the form factor from a differential area to a coaxial parallel square."""
    mb = MeshBuilder()
    mb.quad((-10.0, 0.0, -10.0), (-10.0, 0.0, 10.0), (10.0, 0.0, 10.0), (10.0, 0.0, -10.0), 0)
    h, a = height, half
    mb.quad((-a, h, -a), (a, h, -a), (a, h, a), (-a, h, a), 1)
    scene = mb.build([LAMBERT, EMISSIVE], [0.0, 0.0])
    lam = band_wavelengths(500.0, 600.0, n_bands)
    n, k, rt, lt = _flat_spectra(2, n_bands)
    rt[0] = rho
    lt[1] = le
    spec = _spectra(lam, np.zeros(n_bands), np.array([0.0, 1.0, 0.0]), 0.25, n, k, rt, lt)
    cam = Camera((0.0, 1.0, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 0.01, width, height_px)
    return Workload("emitter_over_plate", scene, spec, [cam], spp, 2, seed)


def camera_marker(target_px=(6, 1), width=8, height=6, vfov_deg=60.0, distance=10.0, marker_half=0.3,
                  spp=256, seed=17) -> Workload:
    """Camera-convention test: a camera at the origin looking along +z (up
    +y, so its right is f x up = -x) and one small emissive square (radiance
    1, rho 0) facing it, centred on the point that a pinhole camera with
    this vertical field of view, aspect width / height, x to the right and y
    downwards shows at the centre of pixel target_px, at the given distance
    along the view axis.  Nothing else is in the scene and there is no sun,
    so only that pixel sees light, with expectation (marker area) / (pixel
    footprint area)."""
    th = math.tan(math.radians(vfov_deg) / 2.0)
    aspect = width / height
    x, y = target_px
    sx = (2.0 * (x + 0.5) / width - 1.0) * th * aspect
    sy = (1.0 - 2.0 * (y + 0.5) / height) * th
    f, r, u = np.array([0.0, 0.0, 1.0]), np.array([-1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])
    c = distance * (f + sx * r + sy * u)
    m = marker_half
    mb = MeshBuilder()
    mb.quad(c - m * r - m * u, c + m * r - m * u, c + m * r + m * u, c - m * r + m * u, 0)
    scene = mb.build([EMISSIVE], [0.0])
    lam = band_wavelengths(500.0, 600.0, 2)
    n, k, rt, lt = _flat_spectra(1, 2)
    lt[0] = 1.0
    spec = _spectra(lam, np.zeros(2), np.array([0.0, 1.0, 0.0]), 0.25, n, k, rt, lt)
    cam = Camera((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0), vfov_deg, width, height)
    return Workload("camera_marker", scene, spec, [cam], spp, 1, seed)


def mirror_caustic(elevation_deg=45.0, sun_half_angle=0.02, n_metal=0.3, k_metal=3.0, rho=0.8, n_bands=1,
                   width=8, height=8, spp=4, depth=4, seed=3) -> Workload:
    """Caustic test: a 10 x 10 m Lambertian floor (y = 0) and a vertical
    1 x 1 m mirror (conductor, x in [-0.5, 0.5], y in [1, 2], z = 0, facing
    -z) under a narrow sun at the given elevation from -z.  The mirror sends
    R(theta) of the sunlight it intercepts (L pi sin^2(a) cos(e) per m^2) down
    onto the floor patch x in [-0.5, 0.5], z in [-2 / tan e, -1 / tan e],
    where it adds irradiance R L pi sin^2(a) sin(e) to the direct sun's
    L pi sin^2(a) sin(e).  The camera looks down at the patch."""
    mb = MeshBuilder()
    mb.quad((-5.0, 0.0, -5.0), (5.0, 0.0, -5.0), (5.0, 0.0, 5.0), (-5.0, 0.0, 5.0), 0)
    mb.quad((-0.5, 1.0, 0.0), (0.5, 1.0, 0.0), (0.5, 2.0, 0.0), (-0.5, 2.0, 0.0), 1)
    scene = mb.build([LAMBERT, CONDUCTOR], [0.0, 0.0])
    lam = band_wavelengths(500.0, 600.0, n_bands) if n_bands > 1 else np.array([550.0])
    n, k, rt, le = _flat_spectra(2, n_bands)
    rt[0] = rho
    n[1] = n_metal
    k[1] = k_metal
    e = math.radians(elevation_deg)
    sun = np.array([0.0, math.sin(e), -math.cos(e)])
    spec = _spectra(lam, np.ones(n_bands), sun, sun_half_angle, n, k, rt, le)
    zc = -1.5 / math.tan(e)
    cam = Camera((0.0, 3.0, zc), (0.0, 0.0, zc + 1e-3), (0.0, 0.0, 1.0), 8.0, width, height)
    return Workload("mirror_caustic", scene, spec, [cam], spp, depth, seed)


def slab_view(n_glass=1.5, k_glass=1e-5, thickness=0.01, lambda_nm=(450.0, 550.0, 650.0),
              tilt_deg=30.0, spp=256, seed=7, sun_side="transmit", material=THIN_GLASS) -> Workload:
    """Camera looks at one tilted sheet with a very narrow field of view.  With
    the sun behind a thin-glass sheet the pixel's expectation is T_s L_sun;
    with the sun on the mirror side it is R_s L_sun (glass) or R L_sun
    (conductor, zero variance)."""
    mb = MeshBuilder()
    t = math.radians(tilt_deg)
    # sheet through the origin, normal (0, sin t, cos t) rotated about x
    ax = np.array([1.0, 0.0, 0.0])
    ay = np.array([0.0, math.cos(t), -math.sin(t)])
    c = [s1 * 3.0 * ax + s2 * 3.0 * ay for s1, s2 in ((-1, -1), (1, -1), (1, 1), (-1, 1))]
    mb.quad(c[0], c[1], c[2], c[3], 0)
    scene = mb.build([material], [thickness])
    lam = np.asarray(lambda_nm, np.float64)
    B = lam.shape[0]
    n, k, rho, le = _flat_spectra(1, B)
    n[0] = n_glass
    k[0] = k_glass
    sun = np.array([0.0, 0.0, 1.0])
    if sun_side == "reflect":
        sun = np.array([0.0, -math.sin(2 * t), -math.cos(2 * t)])
    spec = _spectra(lam, np.ones(B), sun, 0.2, n, k, rho, le)
    cam = Camera((0.0, 0.0, -2.0), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0), 0.05, 2, 2)
    return Workload("slab_view", scene, spec, [cam], spp, 3, seed)


def _nave_geometry(mb: MeshBuilder, *, length=80.0, width=20.0, height=25.0,
                   n_win=8, win_w=2.0, sill=8.0, rect_h=5.0, arch_seg=8,
                   cols_per_side=12, col_r=0.6, col_seg=64, col_rings=64,
                   mat_floor=0, mat_wall=1, mat_ceil=2, mat_col=3, glass_mats=None,
                   pane_rows=1, pane_cols=1, pane_mat=None):
    """Nave shell with pointed-arch windows on both long walls plus columns.
    glass_mats[w] is the material of window w (w < 2 n_win); pane_mat(w, r, c)
    overrides it per pane for leaded stained glass."""
    L, W, H = length, width, height
    spring = sill + rect_h
    xs_c = [L * (i + 0.5) / n_win for i in range(n_win)]
    # pointed (equilateral) arch over [xc - w/2, xc + w/2]
    def arch(xc):
        r = win_w
        pts = []
        a0 = math.atan2(0.0, 1.0)
        left, right = xc - 0.5 * win_w, xc + 0.5 * win_w
        apex_ang = math.acos(0.5)  # arc centred at right springing point
        for j in range(arch_seg + 1):
            ang = math.pi - apex_ang * j / arch_seg  # from the left springing point to the apex
            pts.append((right + r * math.cos(ang), spring + r * math.sin(ang)))
        for j in range(arch_seg - 1, -1, -1):
            ang = apex_ang * j / arch_seg
            pts.append((left + r * math.cos(ang), spring + r * math.sin(ang)))
        pts[0] = (left, spring)
        pts[-1] = (right, spring)
        pts[arch_seg] = (xc, spring + win_w * math.sqrt(3.0) / 2.0)
        del a0
        return pts

    arches = [arch(xc) for xc in xs_c]
    # x breakpoints on the top edge (y = H) of a long wall, shared by the ceiling
    top_x = [0.0]
    for i, xc in enumerate(xs_c):
        top_x.extend(p[0] for p in arches[i])
    top_x.append(L)
    top_x = sorted(set(float(np.float32(x)) for x in top_x))
    bot_x = sorted(set([0.0, L] + [float(np.float32(xc + s * 0.5 * win_w)) for xc in xs_c for s in (-1, 1)]
                       + [float(np.float32(xc)) for xc in xs_c]))

    def wall(z, side):
        # builds the long wall at z; point (x, y) -> (x, y, z)
        P = lambda x, y: (x, y, z)
        prev = 0.0
        for i, xc in enumerate(xs_c):
            x0, x1 = xc - 0.5 * win_w, xc + 0.5 * win_w
            # solid strip [prev, x0] split at sill and springline
            for (ya, yb) in ((0.0, sill), (sill, spring), (spring, H)):
                mb.quad(P(prev, ya), P(x0, ya), P(x0, yb), P(prev, yb), mat_wall)
            # below the sill, split at xc to match the glass
            mb.quad(P(x0, 0.0), P(xc, 0.0), P(xc, sill), P(x0, sill), mat_wall)
            mb.quad(P(xc, 0.0), P(x1, 0.0), P(x1, sill), P(xc, sill), mat_wall)
            widx = side * n_win + i
            # glass rectangle as a grid of panes (pane_cols split at xc for cols even)
            gm = glass_mats[widx]
            ncol = max(2, pane_cols)
            if ncol % 2:
                ncol += 1
            xs = [x0 + (x1 - x0) * c / ncol for c in range(ncol + 1)]
            xs[ncol // 2] = xc
            ys = [sill + rect_h * r / pane_rows for r in range(pane_rows + 1)]
            for r in range(pane_rows):
                for c in range(ncol):
                    m = gm if pane_mat is None else pane_mat(widx, r, c)
                    mb.quad(P(xs[c], ys[r]), P(xs[c + 1], ys[r]), P(xs[c + 1], ys[r + 1]),
                            P(xs[c], ys[r + 1]), m)
            # arch: glass fan from the springline midpoint; the rectangle's top
            # edge is split at xc so the fan centre is a shared vertex.  With
            # ncol > 2 the top edge has more vertices; fan from each.
            pts = arches[i]
            ctr = P(xc, spring)
            m_arch = gm if pane_mat is None else pane_mat(widx, pane_rows, 0)
            # fan covers the segment from the left springing point to the apex
            # and back; bottom edge vertices xs[*] lie on the springline
            for j in range(len(pts) - 1):
                mb.tri(ctr, P(*pts[j + 1]), P(*pts[j]), m_arch)
            # the springline between x0 and xc, xc and x1 carries extra rectangle
            # vertices when ncol > 2: close the T-junctions with slivers of zero
            # area is unnecessary because they are collinear with the fan edge.
            # wall above the arch
            for j in range(len(pts) - 1):
                (xa, ya), (xb, yb) = pts[j], pts[j + 1]
                mb.quad(P(xa, ya), P(xb, yb), P(xb, H), P(xa, H), mat_wall)
            prev = x1
        for (ya, yb) in ((0.0, sill), (sill, spring), (spring, H)):
            mb.quad(P(prev, ya), P(L, ya), P(L, yb), P(prev, yb), mat_wall)

    wall(0.0, 0)
    wall(W, 1)
    # end walls, split at sill and springline heights to share vertices
    for x in (0.0, L):
        for (ya, yb) in ((0.0, sill), (sill, spring), (spring, H)):
            mb.quad((x, ya, 0.0), (x, yb, 0.0), (x, yb, W), (x, ya, W), mat_wall)
    # floor and ceiling as strips along x at the walls' breakpoints
    for y, xs, m in ((0.0, bot_x, mat_floor), (H, top_x, mat_ceil)):
        for a, b in zip(xs[:-1], xs[1:]):
            mb.quad((a, y, 0.0), (b, y, 0.0), (b, y, W), (a, y, W), m)
    # columns (open cylinders from floor to ceiling); col_seg even keeps every
    # facet normal away from the z = 0 sign flip of the shading basis
    ang = 2.0 * math.pi * np.arange(col_seg) / col_seg
    ys = H * np.arange(col_rings + 1) / col_rings
    ring = np.stack([np.cos(ang), np.sin(ang)], 1) * col_r
    i = np.arange(col_seg)
    j = np.arange(col_rings)
    I, J = np.meshgrid(i, j, indexing="ij")
    a = J * col_seg + I
    b = J * col_seg + (I + 1) % col_seg
    c = (J + 1) * col_seg + (I + 1) % col_seg
    d = (J + 1) * col_seg + I
    quads = np.stack([np.stack([a, b, c], -1), np.stack([a, c, d], -1)], 2).reshape(-1, 3)
    for zc in (W * 0.25, W * 0.75):
        for k in range(cols_per_side):
            xc = L * (k + 0.5) / cols_per_side
            vx = xc + np.repeat(ring[None, :, 0], col_rings + 1, 0)
            vz = zc + np.repeat(ring[None, :, 1], col_rings + 1, 0)
            vy = np.repeat(ys[:, None], col_seg, 1)
            verts = np.stack([vx, vy, vz], -1).reshape(-1, 3)
            mb.add_arrays(verts, quads, mat_col)


def nave(width=1024, height=768, n_bands=81, spp=16, depth=8, seed=0, scene_key=1,
         col_seg=64, col_rings=64) -> Workload:
    """Procedural nave, about 200k triangles."""
    rng = np.random.Generator(np.random.Philox(key=scene_key))
    lam = band_wavelengths(380.0, 780.0, n_bands)
    n_stone, n_glass = 4, 16
    glass = list(range(n_stone, n_stone + n_glass))
    mb = MeshBuilder()
    _nave_geometry(mb, glass_mats=glass, col_seg=col_seg, col_rings=col_rings)
    n_mat = n_stone + n_glass
    scene = mb.build([LAMBERT] * n_stone + [THIN_GLASS] * n_glass,
                     [0.0] * n_stone + [0.01] * n_glass)
    n, k, rho, le = _flat_spectra(n_mat, n_bands)
    n[:] = 1.0
    for m in range(n_stone):
        rho[m] = smooth_random_spectrum(rng, lam, 0.3, 0.8)
    for m in glass:
        a = rng.uniform(1.46, 1.58)
        b = rng.uniform(0.002, 0.006)
        n[m] = np.clip(cauchy_n(lam, a, b), 1.45, 1.6)
        k[m] = smooth_log_spectrum(rng, lam, 1e-7, 1e-5)
    sun = sun_direction(35.0, 20.0)
    spec = _spectra(lam, sun_spectrum(lam), sun, 0.25, n, k, rho, le)
    cam = Camera((10.0, 1.7, 10.0), (70.0, 6.0, 10.0), (0.0, 1.0, 0.0), 60.0, width, height)
    return Workload("nave", scene, spec, [cam], spp, depth, seed)


def _icosphere(level: int):
    """Unit sphere from a subdivided icosahedron: 20 * 4^level triangles."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.asarray(p, np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
             (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5),
             (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        mid = {}

        def m(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                q = verts[a] + verts[b]
                verts.append(q / np.linalg.norm(q))
                mid[key] = len(verts) - 1
            return mid[key]
        nf = []
        for a, b, c in faces:
            ab, bc, ca = m(a, b), m(b, c), m(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts), faces


def crystal_nave(width=1024, height=768, n_bands=81, spp=16, depth=8, seed=0, scene_key=1, n_solids=8,
                 col_seg=64, col_rings=64) -> Workload:
    """The procedural nave with solid refracting glass in the sunlit aisle:
    n_solids objects on the centre line, alternating faceted spheres (320
    triangles, crown glass) and triangular prisms (flint glass, a blue
    absorption band), under a sun whose spectrum is Rayleigh-attenuated for
    its 35 degree elevation."""
    base = nave(width=width, height=height, n_bands=n_bands, spp=spp, depth=depth, seed=seed,
                scene_key=scene_key, col_seg=col_seg, col_rings=col_rings)
    lam = band_wavelengths(380.0, 780.0, n_bands)
    n_old = base.scene.n_mat
    CROWN, FLINT = n_old, n_old + 1
    mb = MeshBuilder()
    mb.add_arrays(base.scene.verts.astype(np.float64), base.scene.tris, 0)
    mb.mats[:] = [int(m) for m in base.scene.mat_id]
    sv, sf = _icosphere(2)
    for i in range(n_solids):
        xc = 15.0 + 50.0 * i / max(1, n_solids - 1)
        if i % 2 == 0:
            r, c = 0.8, np.array([xc, 1.2, 10.0])
            _solid(mb, [[tuple(c + r * sv[a]) for a in f] for f in sf], CROWN)
        else:
            a, h, y0 = 1.2, 1.2 * math.sqrt(3.0) / 2.0, 0.4
            tri0 = [(xc - 0.5 * a, y0, 9.0), (xc + 0.5 * a, y0, 9.0), (xc, y0 + h, 9.0)]
            tri1 = [(x, y, 11.0) for (x, y, _) in tri0]
            faces = [tri0, tri1] + [[tri0[j], tri0[(j + 1) % 3], tri1[(j + 1) % 3], tri1[j]] for j in range(3)]
            _solid(mb, faces, FLINT)
    sc = mb.build(list(base.scene.mat_type) + [DIELECTRIC, DIELECTRIC],
                  list(base.scene.mat_thickness) + [0.0, 0.0])
    sp = base.spectra
    B = n_bands
    n = np.concatenate([sp.n.astype(np.float64), np.stack([cauchy_n(lam, 1.52, 0.0042), cauchy_n(lam, 1.62, 0.012)])])
    k = np.concatenate([sp.k.astype(np.float64), np.stack([np.full(B, 1e-8),
                                                          1e-8 + 3e-7 * np.exp(-0.5 * ((lam - 600.0) / 40.0) ** 2)])])
    rho = np.concatenate([sp.rho.astype(np.float64), np.zeros((2, B))])
    le = np.concatenate([sp.le.astype(np.float64), np.zeros((2, B))])
    spec = _spectra(lam, sun_spectrum(lam, elevation_deg=35.0), sp.sun_dir.astype(np.float64), sp.sun_half_angle,
                    n, k, rho, le)
    return Workload("crystal_nave", sc, spec, base.cameras, spp, depth, seed)


def nave_views(n_views=32, n_bands=81, spp=8, depth=8, seed=0, view_key=2, base=None) -> Workload:
    """32 seeded camera views of the nave at uneven resolutions: W and H each
    uniform in {256, 272, ..., 1024}."""
    wl = base if base is not None else nave(n_bands=n_bands, spp=spp, depth=depth, seed=seed)
    rng = np.random.Generator(np.random.Philox(key=view_key))
    sizes = np.arange(256, 1025, 16)
    cams = []
    for _ in range(n_views):
        w, h = int(rng.choice(sizes)), int(rng.choice(sizes))
        pos = (rng.uniform(2.0, 78.0), rng.uniform(1.0, 6.0), rng.uniform(8.0, 12.0))
        look = (rng.uniform(0.0, 80.0), rng.uniform(0.0, 25.0), rng.uniform(0.0, 20.0))
        if abs(look[0] - pos[0]) + abs(look[2] - pos[2]) < 1.0:
            look = (look[0] + 5.0, look[1], look[2])
        cams.append(Camera(pos, look, (0.0, 1.0, 0.0), float(rng.uniform(45.0, 75.0)), w, h))
    return Workload("nave_views", wl.scene, wl.spectra, cams, spp, depth, seed)


def large_nave(width=2048, height=1536, n_bands=81, spp=64, depth=12, seed=0, scene_key=3,
               n_views=4, col_seg=256, col_rings=160) -> Workload:
    """About 2M triangles: finer columns, 40 leaded stained-glass windows with
    per-pane Gaussian absorption bands, brass fittings (conductor)."""
    rng = np.random.Generator(np.random.Philox(key=scene_key))
    lam = band_wavelengths(380.0, 780.0, n_bands)
    n_stone, n_panes, n_metal = 4, 64, 2
    n_win = 20
    glass0 = n_stone
    metal0 = n_stone + n_panes
    mb = MeshBuilder()
    pane_rng = np.random.Generator(np.random.Philox(key=scene_key + 100))
    pane_of = {}

    def pane_mat(w, r, c):
        key = (w, r, c)
        if key not in pane_of:
            pane_of[key] = glass0 + int(pane_rng.integers(0, n_panes))
        return pane_of[key]

    _nave_geometry(mb, n_win=n_win, win_w=1.6, glass_mats=[glass0] * (2 * n_win),
                   pane_rows=6, pane_cols=4, pane_mat=pane_mat,
                   col_seg=col_seg, col_rings=col_rings)
    # metal fittings: a thin bar across each window (two quads, both faces)
    for side, z in ((0, 0.05), (1, 19.95)):
        for i in range(n_win):
            xc = 80.0 * (i + 0.5) / n_win
            m = metal0 + (i % n_metal)
            y0, y1 = 10.4, 10.5
            mb.quad((xc - 0.8, y0, z), (xc + 0.8, y0, z), (xc + 0.8, y1, z), (xc - 0.8, y1, z), m)
    n_mat = n_stone + n_panes + n_metal
    scene = mb.build([LAMBERT] * n_stone + [THIN_GLASS] * n_panes + [CONDUCTOR] * n_metal,
                     [0.0] * n_stone + [0.01] * n_panes + [0.0] * n_metal)
    n, k, rho, le = _flat_spectra(n_mat, n_bands)
    n[:] = 1.0
    for m in range(n_stone):
        rho[m] = smooth_random_spectrum(rng, lam, 0.3, 0.8)
    for p in range(n_panes):
        m = glass0 + p
        n[m] = np.clip(cauchy_n(lam, rng.uniform(1.46, 1.58), rng.uniform(0.002, 0.006)), 1.45, 1.6)
        kk = np.full(n_bands, 1e-7)
        for _ in range(int(rng.integers(1, 4))):
            mu, sg, amp = rng.uniform(400, 760), rng.uniform(15, 60), 10 ** rng.uniform(-6.5, -5.0)
            kk += amp * np.exp(-0.5 * ((lam - mu) / sg) ** 2)
        k[m] = np.clip(kk, 1e-7, 1e-4)
    for q in range(n_metal):
        m = metal0 + q
        n[m] = smooth_random_spectrum(rng, lam, 0.5, 3.0)
        k[m] = smooth_random_spectrum(rng, lam, 2.0, 6.0)
    sun = sun_direction(35.0, 20.0)
    spec = _spectra(lam, sun_spectrum(lam), sun, 0.25, n, k, rho, le)
    vrng = np.random.Generator(np.random.Philox(key=scene_key + 7))
    cams = [Camera((10.0, 1.7, 10.0), (70.0, 6.0, 10.0), (0.0, 1.0, 0.0), 60.0, width, height)]
    for _ in range(n_views - 1):
        pos = (vrng.uniform(5.0, 75.0), vrng.uniform(1.2, 4.0), vrng.uniform(8.5, 11.5))
        look = (vrng.uniform(0.0, 80.0), vrng.uniform(3.0, 20.0), vrng.choice([0.0, 20.0]))
        cams.append(Camera(pos, look, (0.0, 1.0, 0.0), 60.0, width, height))
    return Workload("large_nave", scene, spec, cams, spp, depth, seed)


def random_rays(rng: np.random.Generator, scene: Scene, n: int, inside=True) -> Tuple[np.ndarray, np.ndarray]:
    """Seeded test rays: origins inside the scene bounds, uniform directions."""
    lo = scene.verts.min(0).astype(np.float64)
    hi = scene.verts.max(0).astype(np.float64)
    span = hi - lo
    o = lo + span * (0.05 + 0.9 * rng.random((n, 3))) if inside else lo - span * rng.random((n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)


def edge_rays(rng: np.random.Generator, scene: Scene, n: int) -> Tuple[np.ndarray, np.ndarray]:
    """Rays aimed exactly at shared triangle edges and vertices (watertightness)."""
    v = scene.verts.astype(np.float64)
    t = scene.tris
    lo, hi = v.min(0), v.max(0)
    ctr = 0.5 * (lo + hi)
    pick = rng.integers(0, t.shape[0], n)
    e = rng.integers(0, 3, n)
    a = v[t[pick, e]]
    b = v[t[pick, (e + 1) % 3]]
    s = rng.random((n, 1))
    s[rng.random(n) < 0.2] = 0.0   # some rays at vertices
    target = a + s * (b - a)
    o = ctr + 0.3 * (hi - lo) * (rng.random((n, 3)) - 0.5)
    d = target - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)

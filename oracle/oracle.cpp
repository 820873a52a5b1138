// CPU FP64 oracle for the spectral path tracer.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
// reference that the CUDA library is checked against.  Only the tests, the
// smoke check and the bench's CPU-baseline leg load it.  It shares no code
// with the CUDA library: its own Philox, its own intersection structures
// (brute force, or a median-split BVH), its own Fresnel/slab/sampling code.
//
// What it computes (paper: section 3 Eq. 1 complex index; section 4 Eq. 2 the
// reflection integral and Eq. 3 the sum over directional sources; section 3
// the sun as a plane-wave source; section 6 colorimetry), estimated by Monte
// Carlo path tracing with one wavelength band per path:
//
//   for each (pixel, sample s, band b):
//     camera ray through the pixel jittered by Philox uniforms
//     for vertex k = 1..depth:
//       closest hit; on a miss add T*L_sun if the previous vertex was the
//         camera or a mirror-like event and the direction is inside the cone
//       Lambertian: next-event estimate towards the sun cone (Eq. 3 with the
//         sun as the one directional source), through thin glass; then
//         cosine sampling, T *= rho
//       thin glass: reflect with probability R_s/(R_s+T_s), else pass
//         straight through; T *= R_s + T_s
//       conductor: mirror reflection, T *= R(theta, n, k)
//       solid refracting glass (section 3 Eq. 1; closed mesh, outward
//         normals, no other surface inside): T *= exp(-4 pi k s / lambda)
//         for every stretch s travelled inside; reflect with the Fresnel R
//         of the relative index (n in, 1/n out), else refract by Snell's
//         law with n(lambda); the next ray starts on the true ray, a short
//         step along it; sun rays treat the solid as opaque
//   spectral sum over samples in sample order (FP64), then XYZ.
//
// Everything is double precision except the inputs, which arrive as float.

#include <atomic>
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <thread>
#include <unordered_map>
#include <vector>

#include "guide_net.h"

namespace {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC 2011): ten rounds of two 32x32->64 multiplies with a Weyl
// key schedule.
// ---------------------------------------------------------------------------
struct Ctr4 {
  uint32_t w[4];
};

Ctr4 philox4x32_10(Ctr4 c, uint32_t k0, uint32_t k1) {
  const uint64_t M0 = 0xD2511F53ull, M1 = 0xCD9E8D57ull;
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = M0 * c.w[0];
    uint64_t p1 = M1 * c.w[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    Ctr4 n;
    n.w[0] = hi1 ^ c.w[1] ^ k0;
    n.w[1] = lo1;
    n.w[2] = hi0 ^ c.w[3] ^ k1;
    n.w[3] = lo0;
    c = n;
  }
  return c;
}

// uniform in [0, 1) from the top 24 bits: exact in float and double
double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

struct V3 {
  double x, y, z;
};
V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
V3 normalize(V3 a) { return (1.0 / std::sqrt(dot(a, a))) * a; }
double comp(V3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

// Orthonormal basis around a unit vector: Duff, Burgess, Christensen, Hery,
// Kensler, Liani, Villemin, "Building an orthonormal basis, revisited",
// JCGT 6(1), 2017.
void onb(V3 n, V3* t1, V3* t2) {
  double sign = std::copysign(1.0, n.z);
  double a = -1.0 / (sign + n.z);
  double b = n.x * n.y * a;
  *t1 = {1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x};
  *t2 = {b, sign + n.y * n.y * a, -n.y};
}

// ---------------------------------------------------------------------------
// optics (section 3, Eq. 1: n~ = n + i k)
// ---------------------------------------------------------------------------

// Unpolarised Fresnel reflectance from air (index 1) into a medium of complex
// index eta = n + i k, for cos(theta_i) = c: the s and p amplitude ratios with
// the complex cosine of the transmitted angle, averaged in intensity.
double fresnel_complex(double c, double n, double k) {
  std::complex<double> eta(n, k);
  double s2 = 1.0 - c * c;
  std::complex<double> ct = std::sqrt(1.0 - s2 / (eta * eta));
  std::complex<double> rs = (c - eta * ct) / (c + eta * ct);
  std::complex<double> rp = (eta * c - ct) / (eta * c + ct);
  return 0.5 * (std::norm(rs) + std::norm(rp));
}

// Thin absorbing sheet of thickness d (metres): each face reflects R (complex
// Fresnel), the interior attenuates by Beer-Lambert exp(-alpha d / cos_t),
// alpha = 4 pi k / lambda, and the incoherent multiple reflections sum to
//   R_s = R + (1-R)^2 R Ti^2 / (1 - R^2 Ti^2),  T_s = (1-R)^2 Ti / (1 - R^2 Ti^2).
void slab(double c, double n, double k, double lambda_nm, double d, double* Rs, double* Ts) {
  double R = fresnel_complex(c, n, k);
  double sin2 = 1.0 - c * c;
  double ct = std::sqrt(1.0 - sin2 / (n * n));
  double alpha = 4.0 * M_PI * k / (lambda_nm * 1e-9);
  double Ti = std::exp(-alpha * d / ct);
  double den = 1.0 - R * R * Ti * Ti;
  *Rs = R + (1.0 - R) * (1.0 - R) * R * Ti * Ti / den;
  *Ts = (1.0 - R) * (1.0 - R) * Ti / den;
}

// ---------------------------------------------------------------------------
// scene
// ---------------------------------------------------------------------------
enum { M_LAMBERT = 0, M_GLASS = 1, M_CONDUCTOR = 2, M_EMISSIVE = 3, M_DIELECTRIC = 4 };

// Refraction of the unit direction d at a surface with unit normal n facing
// the incident side (dot(d, n) < 0), from index 1 into relative index eta
// (eta < 1 when leaving the denser medium): Snell's law
// sin(theta_t) = sin(theta_i) / eta in the plane of d and n.  Returns false
// on total internal reflection.
bool refract(V3 d, V3 n, double eta, V3* t) {
  const double ci = -dot(d, n);
  const double r = 1.0 / eta;
  const double k = 1.0 - r * r * (1.0 - ci * ci);
  if (k < 0.0) return false;
  *t = r * d + (r * ci - std::sqrt(k)) * n;
  return true;
}

struct ONode {
  double lo[3], hi[3];
  int left = -1, right = -1;   // children, or -1 for a leaf
  int first = 0, count = 0;    // leaf range in the permuted triangle list
};

struct OScene {
  std::vector<V3> a, b, c;       // triangle vertices
  std::vector<uint32_t> mat;     // material id per triangle
  std::vector<int> mtype;
  std::vector<double> mthick;
  uint32_t n_mat = 0, B = 0;
  std::vector<double> lam, sunL, ntab, ktab, rho, le;
  V3 sun{0, 0, 1};
  double cos_max = 1.0;
  double eps = 0.0;              // origin offset: 1e-4 x scene diagonal
  V3 lo{0, 0, 0}, hi{0, 0, 0};   // vertex bounds
  bool brute = true;
  std::vector<ONode> nodes;
  std::vector<uint32_t> perm;
};

// Watertight ray/triangle test (Woop, Benthin, Wald, "Watertight ray/triangle
// intersection", JCGT 2(1), 2013), in double precision.  An edge function of
// exactly zero counts as inside.  Returns t > 0 or -1.
struct RayPre {
  V3 o, d;
  int kx, ky, kz;
  double Sx, Sy, Sz;
};

RayPre prep(V3 o, V3 d) {
  RayPre r;
  r.o = o;
  r.d = d;
  double ax = std::fabs(d.x), ay = std::fabs(d.y), az = std::fabs(d.z);
  r.kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
  r.kx = (r.kz + 1) % 3;
  r.ky = (r.kx + 1) % 3;
  if (comp(d, r.kz) < 0.0) std::swap(r.kx, r.ky);
  double dz = comp(d, r.kz);
  r.Sx = comp(d, r.kx) / dz;
  r.Sy = comp(d, r.ky) / dz;
  r.Sz = 1.0 / dz;
  return r;
}

double isect(const RayPre& r, V3 va, V3 vb, V3 vc) {
  V3 A = va - r.o, Bv = vb - r.o, C = vc - r.o;
  double Ax = comp(A, r.kx) - r.Sx * comp(A, r.kz);
  double Ay = comp(A, r.ky) - r.Sy * comp(A, r.kz);
  double Bx = comp(Bv, r.kx) - r.Sx * comp(Bv, r.kz);
  double By = comp(Bv, r.ky) - r.Sy * comp(Bv, r.kz);
  double Cx = comp(C, r.kx) - r.Sx * comp(C, r.kz);
  double Cy = comp(C, r.ky) - r.Sy * comp(C, r.kz);
  double U = Cx * By - Cy * Bx;
  double V = Ax * Cy - Ay * Cx;
  double W = Bx * Ay - By * Ax;
  if ((U < 0 || V < 0 || W < 0) && (U > 0 || V > 0 || W > 0)) return -1.0;
  double det = U + V + W;
  if (det == 0.0) return -1.0;
  double Az = r.Sz * comp(A, r.kz), Bz = r.Sz * comp(Bv, r.kz), Cz = r.Sz * comp(C, r.kz);
  double T = U * Az + V * Bz + W * Cz;
  double t = T / det;
  return t > 0.0 ? t : -1.0;
}

bool box_hit(const ONode& nd, V3 o, V3 d, double tmax) {
  double t0 = 0.0, t1 = tmax;
  for (int i = 0; i < 3; ++i) {
    double oi = comp(o, i), di = comp(d, i);
    double pad = 1e-9 * (std::fabs(nd.lo[i]) + std::fabs(nd.hi[i])) + 1e-12;
    double lo = nd.lo[i] - pad, hi = nd.hi[i] + pad;
    if (di == 0.0) {
      if (oi < lo || oi > hi) return false;
      continue;
    }
    double ta = (lo - oi) / di, tb = (hi - oi) / di;
    if (ta > tb) std::swap(ta, tb);
    t0 = std::max(t0, ta);
    t1 = std::min(t1, tb);
    if (t0 > t1) return false;
  }
  return true;
}

// Median-split BVH over triangle centroids (longest centroid axis, leaves of
// at most 4 triangles).  Only an accelerator for the brute-force definition.
int build_node(OScene& S, int first, int count) {
  ONode nd;
  for (int i = 0; i < 3; ++i) {
    nd.lo[i] = INFINITY;
    nd.hi[i] = -INFINITY;
  }
  double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int j = first; j < first + count; ++j) {
    uint32_t t = S.perm[j];
    for (V3 v : {S.a[t], S.b[t], S.c[t]})
      for (int i = 0; i < 3; ++i) {
        nd.lo[i] = std::min(nd.lo[i], comp(v, i));
        nd.hi[i] = std::max(nd.hi[i], comp(v, i));
      }
    V3 cen = (1.0 / 3.0) * (S.a[t] + S.b[t] + S.c[t]);
    for (int i = 0; i < 3; ++i) {
      clo[i] = std::min(clo[i], comp(cen, i));
      chi[i] = std::max(chi[i], comp(cen, i));
    }
  }
  int axis = 0;
  for (int i = 1; i < 3; ++i)
    if (chi[i] - clo[i] > chi[axis] - clo[axis]) axis = i;
  int idx = (int)S.nodes.size();
  S.nodes.push_back(nd);
  if (count <= 4 || chi[axis] - clo[axis] <= 0.0) {
    S.nodes[idx].first = first;
    S.nodes[idx].count = count;
    return idx;
  }
  int mid = first + count / 2;
  auto key = [&](uint32_t t) { return comp(S.a[t] + S.b[t] + S.c[t], axis); };
  std::nth_element(S.perm.begin() + first, S.perm.begin() + mid, S.perm.begin() + first + count,
                   [&](uint32_t p, uint32_t q) { return key(p) < key(q) || (key(p) == key(q) && p < q); });
  int l = build_node(S, first, mid - first);
  int r = build_node(S, mid, first + count - mid);
  S.nodes[idx].left = l;
  S.nodes[idx].right = r;
  return idx;
}

// Closest hit with t > 0; equal t resolved to the lower triangle id.
bool closest(const OScene& S, V3 o, V3 d, double* t_out, uint32_t* prim_out) {
  RayPre r = prep(o, d);
  double best = INFINITY;
  int64_t bid = -1;
  auto test = [&](uint32_t t) {
    double th = isect(r, S.a[t], S.b[t], S.c[t]);
    if (th > 0.0 && (th < best || (th == best && (int64_t)t < bid))) {
      best = th;
      bid = t;
    }
  };
  if (S.brute) {
    for (uint32_t t = 0; t < S.a.size(); ++t) test(t);
  } else {
    std::vector<int> stack;
    stack.reserve(128);
    stack.push_back(0);
    while (!stack.empty()) {
      int ni = stack.back();
      stack.pop_back();
      const ONode& nd = S.nodes[ni];
      if (!box_hit(nd, o, d, best)) continue;
      if (nd.left < 0) {
        for (int j = nd.first; j < nd.first + nd.count; ++j) test(S.perm[j]);
      } else {
        stack.push_back(nd.left);
        stack.push_back(nd.right);
      }
    }
  }
  if (bid < 0) return false;
  *t_out = best;
  *prim_out = (uint32_t)bid;
  return true;
}

// Transmittance of a ray to infinity: 0 if any opaque triangle is crossed,
// else the product of the thin-glass T_s of every crossed sheet.  n_glass
// returns the number of sheets crossed (or UINT32_MAX when blocked).
double shadow_T(const OScene& S, V3 o, V3 d, uint32_t band, uint32_t* n_glass) {
  RayPre r = prep(o, d);
  double T = 1.0;
  uint32_t ng = 0;
  bool blocked = false;
  auto visit = [&](uint32_t t) {
    if (blocked) return;
    double th = isect(r, S.a[t], S.b[t], S.c[t]);
    if (!(th > 0.0)) return;
    uint32_t m = S.mat[t];
    if (S.mtype[m] != M_GLASS) {
      blocked = true;
      return;
    }
    V3 ng_ = cross(S.b[t] - S.a[t], S.c[t] - S.a[t]);
    double c = std::fabs(dot(d, normalize(ng_)));
    double Rs, Ts;
    slab(c, S.ntab[m * S.B + band], S.ktab[m * S.B + band], S.lam[band], S.mthick[m], &Rs, &Ts);
    T *= Ts;
    ++ng;
  };
  if (S.brute) {
    for (uint32_t t = 0; t < S.a.size() && !blocked; ++t) visit(t);
  } else {
    std::vector<int> stack;
    stack.reserve(128);
    stack.push_back(0);
    while (!stack.empty() && !blocked) {
      int ni = stack.back();
      stack.pop_back();
      const ONode& nd = S.nodes[ni];
      if (!box_hit(nd, o, d, INFINITY)) continue;
      if (nd.left < 0) {
        for (int j = nd.first; j < nd.first + nd.count; ++j) visit(S.perm[j]);
      } else {
        stack.push_back(nd.left);
        stack.push_back(nd.right);
      }
    }
  }
  if (blocked) {
    *n_glass = 0xFFFFFFFFu;
    return 0.0;
  }
  *n_glass = ng;
  return T;
}

uint32_t mix(uint32_t h, uint32_t v) { return (h ^ v) * 16777619u; }

struct OCam {
  V3 pos, f, r, u;
  double th, aspect;
  uint32_t W, H;
  uint64_t offset;
};

}  // namespace

extern "C" {

typedef struct {
  const float* verts;
  uint32_t n_verts;
  const uint32_t* tris;
  uint32_t n_tris;
  const uint32_t* mat_id;
  const int32_t* mat_type;
  const float* mat_thickness;
  uint32_t n_mat;
  const float* lambda_nm;
  uint32_t n_bands;
  const float* sun_L;
  const float* sun_dir;
  float sun_half_angle;
  const float* n_tab;
  const float* k_tab;
  const float* rho_tab;
  const float* le_tab;
} or_scene_desc;

typedef struct {
  float pos[3], look[3], up[3];
  float vfov_deg;
  uint32_t width, height;
} or_camera;

}  // extern "C"

namespace {

std::vector<OCam> setup_cams(const or_camera* cams, uint32_t n_cams) {
  std::vector<OCam> oc(n_cams);
  uint64_t off = 0;
  for (uint32_t v = 0; v < n_cams; ++v) {
    const or_camera& c = cams[v];
    V3 pos{c.pos[0], c.pos[1], c.pos[2]}, look{c.look[0], c.look[1], c.look[2]}, up{c.up[0], c.up[1], c.up[2]};
    oc[v].pos = pos;
    oc[v].f = normalize(look - pos);
    oc[v].r = normalize(cross(oc[v].f, up));
    oc[v].u = cross(oc[v].r, oc[v].f);
    oc[v].th = std::tan(0.5 * (double)c.vfov_deg * M_PI / 180.0);
    oc[v].aspect = (double)c.width / (double)c.height;
    oc[v].W = c.width;
    oc[v].H = c.height;
    oc[v].offset = off;
    off += (uint64_t)c.width * c.height;
  }
  return oc;
}

// Primary ray of global pixel pix, sample s, Philox stream of band b.
void camera_ray(const std::vector<OCam>& oc, uint32_t pix, uint32_t s, uint32_t b, uint32_t k0, uint32_t k1, V3* o,
                V3* d) {
  uint32_t v = 0;
  while (v + 1 < oc.size() && oc[v + 1].offset <= pix) ++v;
  const OCam& C = oc[v];
  uint32_t local = pix - (uint32_t)C.offset;
  uint32_t x = local % C.W, y = local / C.W;
  Ctr4 r0 = philox4x32_10(Ctr4{{pix, s, b, 0u}}, k0, k1);
  double sx = (2.0 * ((double)x + u01(r0.w[0])) / C.W - 1.0) * C.th * C.aspect;
  double sy = (1.0 - 2.0 * ((double)y + u01(r0.w[1])) / C.H) * C.th;
  *d = normalize(C.f + sx * C.r + sy * C.u);
  *o = C.pos;
}

// Cosine-weighted direction about the unit normal n from uniforms u, v
// (Malley's method: a uniform point of the unit disk, sin theta = sqrt(u),
// lifted to the hemisphere): pdf cos(theta) / pi.
V3 cosine_dir(V3 n, double u, double v) {
  const double rr = std::sqrt(u);
  const double ph = 2.0 * M_PI * v;
  const double z = std::sqrt(std::max(0.0, 1.0 - u));
  V3 b1, b2;
  onb(n, &b1, &b2);
  return (rr * std::cos(ph)) * b1 + (rr * std::sin(ph)) * b2 + z * n;
}

// ---------------------------------------------------------------------------
// learned guide inside the estimator: one-sample MIS (section 4, Eq. 2)
// ---------------------------------------------------------------------------
// At a guided Lambertian vertex the continuation is drawn from the guide's
// von Mises-Fisher mixture q with probability alpha, else by cosine
// sampling; either way it is weighted by the one-sample MIS density
//   p_mix(w) = alpha q(w) + (1 - alpha) max(cos, 0) / pi,
// so the throughput becomes T (rho / pi) cos / p_mix and the expectation of
// Eq. 2 does not depend on q.  The direct sun there is estimated by two
// strategies combined with the balance heuristic: the sun-cone sample
// (density p_cone = 1 / (2 pi (1 - cos a))) weighted
// p_cone / (p_cone + p_mix(w_sun)), and the continuation escaping into the
// cone weighted p_mix / (p_mix + p_cone).
struct GuideCtx {
  const oguide::Net* net = nullptr;
  double alpha = 0.7;
  uint32_t depth = 0;    // vertices 1..depth are guided
  uint32_t n_bands = 1;  // band group of band b: b * 9 / n_bands
};

// vMF direction around the unit mu with concentration kappa from uniforms
// u, v (Jakob, "Numerically stable sampling of the von Mises-Fisher
// distribution on S^2", 2012): cos = 1 + log(u + (1 - u) e^{-2 kappa}) /
// kappa about mu, azimuth 2 pi v in the basis onb(mu).
V3 vmf_dir(const double mu[3], double kappa, double u, double v) {
  const double w = 1.0 + std::log(u + (1.0 - u) * std::exp(-2.0 * kappa)) / kappa;
  const double r = std::sqrt(std::max(0.0, 1.0 - w * w));
  const double ph = 2.0 * M_PI * v;
  const V3 m{mu[0], mu[1], mu[2]};
  V3 t1, t2;
  onb(m, &t1, &t2);
  return (r * std::cos(ph)) * t1 + (r * std::sin(ph)) * t2 + w * m;
}

// A draw of the one-sample MIS proposal: guide with probability alpha
// (uniform ug), lobe j with probability pi_j (the first j whose cumulative
// weight exceeds ul; the last lobe if rounding leaves none), direction by
// vmf_dir(uv0, uv1); else cosine sampling (uc0, uc1).
struct MisDraw {
  V3 omega{0, 0, 1};
  bool guide = false;
  int lobe = -1;
  double lobe_margin = 1.0;  // distance of ul from the nearest cumulative lobe boundary
};

MisDraw mis_draw(const oguide::Mixture& mx, V3 n, double alpha, double ug, double ul, double uv0, double uv1,
                 double uc0, double uc1) {
  MisDraw d;
  d.guide = ug < alpha;
  if (!d.guide) {
    d.omega = cosine_dir(n, uc0, uc1);
    return d;
  }
  double acc = 0.0;
  d.lobe = oguide::kLobes - 1;
  bool found = false;
  for (int j = 0; j < oguide::kLobes; ++j) {
    acc += mx.pi[j];
    if (j + 1 < oguide::kLobes) d.lobe_margin = std::min(d.lobe_margin, std::fabs(ul - acc));
    if (!found && ul < acc) {
      d.lobe = j;
      found = true;
    }
  }
  d.omega = vmf_dir(mx.mu[d.lobe], mx.kappa[d.lobe], uv0, uv1);
  return d;
}

double mis_pdf(const oguide::Mixture& mx, V3 n, double alpha, V3 w, double* q_out) {
  const double ww[3] = {w.x, w.y, w.z};
  const double q = oguide::mixture_density(mx, ww);
  if (q_out) *q_out = q;
  return alpha * q + (1.0 - alpha) * std::max(dot(n, w), 0.0) / M_PI;
}

// Everything one guided vertex decides, given its query (offset position po,
// normal n, band group), its Philox draws r0 (counter call 0: the sun
// sample and the cosine continuation) and r1 (call 1: the MIS choice, lobe
// and vMF direction) and its pending sun sample (direction wn, if any).
struct GuidedVertex {
  MisDraw draw;
  double q = 0.0, pdf = 0.0, c = 0.0;   // guide density, MIS density and cosine at omega
  double q_sun = 0.0, pdf_sun = 0.0;    // the same at the sun-sample direction
  double nee_w = 1.0;                   // balance weight of the sun sample
  double esc_w = 0.0;                   // balance weight of a sun escape of the continuation
  bool cont = false;                    // the path continues (cos > 0 and p_mix > 0)
};

GuidedVertex guided_vertex(const GuideCtx& g, const OScene& S, V3 po, V3 n, uint32_t group, const Ctr4& r0,
                           const Ctr4& r1, bool has_sun, V3 wn) {
  GuidedVertex gv;
  double Y[48];
  const double pp[3] = {po.x, po.y, po.z}, nn[3] = {n.x, n.y, n.z};
  oguide::net_outputs(g.net, pp, nn, group, Y);
  oguide::Mixture mx;
  oguide::mixture_of(Y, &mx);
  gv.draw = mis_draw(mx, n, g.alpha, u01(r1.w[0]), u01(r1.w[1]), u01(r1.w[2]), u01(r1.w[3]), u01(r0.w[2]),
                     u01(r0.w[3]));
  const double p_cone = 1.0 / (2.0 * M_PI * (1.0 - S.cos_max));
  gv.c = dot(n, gv.draw.omega);
  gv.pdf = mis_pdf(mx, n, g.alpha, gv.draw.omega, &gv.q);
  if (has_sun) {
    gv.pdf_sun = mis_pdf(mx, n, g.alpha, wn, &gv.q_sun);
    gv.nee_w = p_cone / (p_cone + gv.pdf_sun);
  }
  gv.cont = gv.c > 0.0 && gv.pdf > 0.0;
  if (gv.cont && dot(gv.draw.omega, S.sun) >= S.cos_max) gv.esc_w = gv.pdf / (gv.pdf + p_cone);
  return gv;
}

// Training records of one guided vertex (the guide learns from the samples
// the tracer draws): the continuation, weight L_in cos / p_mix with L_in the
// radiance the path gathered after the vertex divided by its throughput
// there, and the sun sample, weight L_sun T_r cos / p_cone.  Each record is
// 12 floats {position, weight}, {normal, band group}, {direction, 0}; a
// record of weight <= 0 is {0, 0, 0, 0}, {0, 0, 1, 0}, {0, 0, 1, 0}.
struct GuidedSlot {
  bool valid = false;
  V3 po{0, 0, 0}, n{0, 0, 1}, omega{0, 0, 1}, wn{0, 0, 1};
  double group = 0.0, pdf = 0.0, c = 0.0, Tn = 0.0, L_before = 0.0;
  bool sun = false;
  double sun_rad = 0.0, cn = 0.0;
};

void put_record(float* o, V3 p, double wt, V3 n, double group, V3 w) {
  if (wt > 0.0) {
    const float v[12] = {(float)p.x, (float)p.y, (float)p.z, (float)wt, (float)n.x, (float)n.y, (float)n.z,
                         (float)group, (float)w.x, (float)w.y, (float)w.z, 0.0f};
    std::memcpy(o, v, sizeof(v));
  } else {
    const float v[12] = {0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 1, 0};
    std::memcpy(o, v, sizeof(v));
  }
}

void slot_records(const GuidedSlot& sl, double L_final, double p_cone, float* out24) {
  double wt = 0.0, ws = 0.0;
  if (sl.valid && sl.Tn > 0.0 && sl.pdf > 0.0) wt = std::max((L_final - sl.L_before) / sl.Tn, 0.0) * sl.c / sl.pdf;
  if (sl.valid && sl.sun && sl.cn > 0.0) ws = std::max(sl.sun_rad, 0.0) * sl.cn / p_cone;
  put_record(out24, sl.po, wt, sl.n, sl.group, sl.omega);
  put_record(out24 + 12, sl.po, ws, sl.n, sl.group, sl.wn);
}

// One path (pixel pix, sample s, band b) of the estimator.  Plain when g is
// null; guided at Lambertian vertices 1..g->depth (below the last vertex)
// otherwise, with the training slots of those vertices in slots[0..depth).
double trace_path(const OScene& S, const std::vector<OCam>& oc, uint32_t k0, uint32_t k1, uint32_t pix, uint32_t s,
                  uint32_t b, uint32_t depth, const GuideCtx* g, uint32_t* sig_out, GuidedSlot* slots) {
  // f / pdf for the sun cone: (rho / pi) * 2 pi (1 - cos_max) = rho * cone_w
  const double cone_w = 2.0 * (1.0 - S.cos_max);
  V3 o, d;
  camera_ray(oc, pix, s, b, k0, k1, &o, &d);
  double T = 1.0, L = 0.0;
  bool covered = false;   // direct sun along this segment is already counted by NEE
  bool guided_esc = false;  // ... by NEE with a balance weight: a sun escape adds esc_w of it
  double esc_w = 0.0;
  GuidedSlot* open = nullptr;  // training slot waiting for the radiance gathered before the next vertex
  uint32_t sig = 2166136261u;
  for (uint32_t k = 1; k <= depth; ++k) {
    if (open) {
      open->L_before = L;
      open = nullptr;
    }
    double t;
    uint32_t prim;
    if (!closest(S, o, d, &t, &prim)) {
      sig = mix(sig, 0xFFFFFFFFu);
      if (dot(d, S.sun) >= S.cos_max) {
        if (!covered) L += T * S.sunL[b];
        else if (guided_esc) L += T * S.sunL[b] * esc_w;
      }
      break;
    }
    sig = mix(sig, prim);
    V3 p = o + t * d;
    V3 ng = normalize(cross(S.b[prim] - S.a[prim], S.c[prim] - S.a[prim]));
    V3 n = dot(ng, d) < 0.0 ? ng : -1.0 * ng;
    double cos_i = -dot(d, n);
    uint32_t m = S.mat[prim];
    size_t mb = (size_t)m * S.B + b;
    int type = S.mtype[m];
    Ctr4 r = philox4x32_10(Ctr4{{pix, s, b, 4u * k}}, k0, k1);
    if (type == M_LAMBERT || type == M_EMISSIVE) {
      if (type == M_EMISSIVE) L += T * S.le[mb];
      // next-event estimate: direction uniform in the sun cone,
      // pdf = 1 / (2 pi (1 - cos_max)); f = rho / pi
      double ct = 1.0 - u01(r.w[0]) * (1.0 - S.cos_max);
      double st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
      double ph = 2.0 * M_PI * u01(r.w[1]);
      V3 t1, t2;
      onb(S.sun, &t1, &t2);
      V3 w = (st * std::cos(ph)) * t1 + (st * std::sin(ph)) * t2 + ct * S.sun;
      double c = dot(n, w);
      double nee = 0.0, Tr = 0.0;
      if (c > 0.0) {
        uint32_t ngl;
        Tr = shadow_T(S, p + S.eps * n, w, b, &ngl);
        sig = mix(sig, ngl);
        nee = T * S.rho[mb] * c * S.sunL[b] * cone_w * Tr;
      }
      const bool guided = g && k <= g->depth && k < depth;
      if (!guided) {
        L += nee;
        if (k == depth) break;
        // cosine-weighted continuation: f cos / pdf = rho
        d = cosine_dir(n, u01(r.w[2]), u01(r.w[3]));
        o = p + S.eps * n;
        T *= S.rho[mb];
        covered = true;
        guided_esc = false;
        continue;
      }
      const V3 po = p + S.eps * n;
      const uint32_t group = b * 9u / g->n_bands;
      Ctr4 r1 = philox4x32_10(Ctr4{{pix, s, b, 4u * k + 1u}}, k0, k1);
      const GuidedVertex gv = guided_vertex(*g, S, po, n, group, r, r1, c > 0.0, w);
      L += nee * gv.nee_w;
      double Tn = 0.0;
      if (gv.cont) Tn = T * S.rho[mb] / M_PI * gv.c / gv.pdf;
      if (slots) {
        GuidedSlot& sl = slots[k - 1];
        sl.valid = true;
        sl.po = po;
        sl.n = n;
        sl.omega = gv.draw.omega;
        sl.group = (double)group;
        sl.pdf = gv.pdf;
        sl.c = gv.c;
        sl.Tn = Tn;
        sl.sun = c > 0.0;
        sl.wn = sl.sun ? w : V3{0, 0, 1};
        sl.cn = sl.sun ? c : 0.0;
        sl.sun_rad = sl.sun ? Tr * S.sunL[b] : 0.0;
        open = &sl;
      }
      if (!gv.cont) break;  // no continuation: the path ends after its sun sample
      d = gv.draw.omega;
      o = po;
      T = Tn;
      covered = true;
      guided_esc = true;
      esc_w = gv.esc_w;
    } else if (type == M_GLASS) {
      double Rs, Ts;
      slab(cos_i, S.ntab[mb], S.ktab[mb], S.lam[b], S.mthick[m], &Rs, &Ts);
      if (k == depth) break;
      Ctr4 r1 = philox4x32_10(Ctr4{{pix, s, b, 4u * k + 1u}}, k0, k1);
      if (u01(r1.w[0]) < Rs / (Rs + Ts)) {
        d = d - (2.0 * dot(d, n)) * n;
        o = p + S.eps * n;
        covered = false;
        guided_esc = false;
      } else {
        o = p - S.eps * n;
      }
      T *= Rs + Ts;
    } else if (type == M_DIELECTRIC) {
      // solid refracting glass (a closed mesh, normals outward, holding
      // no other surface): light is attenuated by Beer-Lambert
      // exp(-alpha s), alpha = 4 pi k / lambda, over every stretch s it
      // travels inside -- the segment that ends here when it arrives from
      // inside, and the short start step of a new ray that heads inside.
      // The face reflects with the Fresnel reflectance of the relative
      // index (n entering, 1/n leaving; total internal reflection gives
      // 1), else refracts (Snell; dispersion through n(lambda)).  The next
      // ray starts on the true ray, a step eps / max(|cos|, 1/16) along
      // it, so the distance crossed inside is exact.
      const bool inside = dot(ng, d) > 0.0;
      const double alpha = 4.0 * M_PI * S.ktab[mb] / (S.lam[b] * 1e-9);
      if (inside) T *= std::exp(-alpha * t);
      const double eta = inside ? 1.0 / S.ntab[mb] : S.ntab[mb];
      const double R = fresnel_complex(cos_i, eta, 0.0);
      if (k == depth) break;
      Ctr4 r1 = philox4x32_10(Ctr4{{pix, s, b, 4u * k + 1u}}, k0, k1);
      V3 tdir;
      if (u01(r1.w[0]) < R || !refract(d, n, eta, &tdir)) d = d - (2.0 * dot(d, n)) * n;
      else d = normalize(tdir);
      const double step = S.eps / std::max(std::fabs(dot(d, n)), 0.0625);
      if (dot(d, ng) < 0.0) T *= std::exp(-alpha * step);
      o = p + step * d;
      covered = false;
      guided_esc = false;
    } else {  // conductor
      double R = fresnel_complex(cos_i, S.ntab[mb], S.ktab[mb]);
      if (k == depth) break;
      d = d - (2.0 * dot(d, n)) * n;
      o = p + S.eps * n;
      T *= R;
      covered = false;
      guided_esc = false;
    }
  }
  if (sig_out) *sig_out = sig;
  return L;
}

}  // namespace

extern "C" {

void or_philox4x32_10(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4]) {
  Ctr4 c{{ctr[0], ctr[1], ctr[2], ctr[3]}};
  Ctr4 r = philox4x32_10(c, key[0], key[1]);
  std::memcpy(out, r.w, 16);
}

void or_philox_batch(uint32_t key0, uint32_t key1, const uint32_t* ctr, uint32_t* out, uint64_t n) {
  for (uint64_t i = 0; i < n; ++i) {
    Ctr4 c{{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]}};
    Ctr4 r = philox4x32_10(c, key0, key1);
    std::memcpy(out + 4 * i, r.w, 16);
  }
}

double or_fresnel(double cos_i, double n, double k) { return fresnel_complex(cos_i, n, k); }

int or_refract(const double d[3], const double n[3], double eta, double t[3]) {
  V3 r;
  if (!refract(V3{d[0], d[1], d[2]}, V3{n[0], n[1], n[2]}, eta, &r)) return 0;
  t[0] = r.x;
  t[1] = r.y;
  t[2] = r.z;
  return 1;
}

void or_slab(double cos_i, double n, double k, double lambda_nm, double d, double* Rs, double* Ts) {
  slab(cos_i, n, k, lambda_nm, d, Rs, Ts);
}

void* or_scene_create(const or_scene_desc* sd, int force_brute) {
  OScene* S = new OScene();
  S->n_mat = sd->n_mat;
  S->B = sd->n_bands;
  uint32_t nt = sd->n_tris;
  S->a.resize(nt);
  S->b.resize(nt);
  S->c.resize(nt);
  S->mat.resize(nt);
  auto vtx = [&](uint32_t i) {
    return V3{(double)sd->verts[3 * i], (double)sd->verts[3 * i + 1], (double)sd->verts[3 * i + 2]};
  };
  V3 lo{INFINITY, INFINITY, INFINITY}, hi{-INFINITY, -INFINITY, -INFINITY};
  for (uint32_t i = 0; i < sd->n_verts; ++i) {
    V3 v = vtx(i);
    lo = {std::min(lo.x, v.x), std::min(lo.y, v.y), std::min(lo.z, v.z)};
    hi = {std::max(hi.x, v.x), std::max(hi.y, v.y), std::max(hi.z, v.z)};
  }
  S->eps = 1e-4 * std::sqrt(dot(hi - lo, hi - lo));
  S->lo = lo;
  S->hi = hi;
  for (uint32_t t = 0; t < nt; ++t) {
    S->a[t] = vtx(sd->tris[3 * t]);
    S->b[t] = vtx(sd->tris[3 * t + 1]);
    S->c[t] = vtx(sd->tris[3 * t + 2]);
    S->mat[t] = sd->mat_id[t];
  }
  S->mtype.assign(sd->mat_type, sd->mat_type + sd->n_mat);
  S->mthick.assign(sd->mat_thickness, sd->mat_thickness + sd->n_mat);
  size_t MB = (size_t)sd->n_mat * sd->n_bands;
  S->lam.assign(sd->lambda_nm, sd->lambda_nm + sd->n_bands);
  S->sunL.assign(sd->sun_L, sd->sun_L + sd->n_bands);
  S->ntab.assign(sd->n_tab, sd->n_tab + MB);
  S->ktab.assign(sd->k_tab, sd->k_tab + MB);
  S->rho.assign(sd->rho_tab, sd->rho_tab + MB);
  S->le.assign(sd->le_tab, sd->le_tab + MB);
  S->sun = normalize(V3{sd->sun_dir[0], sd->sun_dir[1], sd->sun_dir[2]});
  S->cos_max = std::cos((double)sd->sun_half_angle);
  S->brute = force_brute || nt <= 64;
  if (!S->brute) {
    S->perm.resize(nt);
    std::iota(S->perm.begin(), S->perm.end(), 0u);
    S->nodes.reserve(nt);
    build_node(*S, 0, (int)nt);
  }
  return S;
}

void or_scene_destroy(void* s) { delete (OScene*)s; }

double or_scene_eps(void* s) { return ((OScene*)s)->eps; }

// Closest hits for n rays: t (or -1) and the triangle id (or -1).
void or_closest_hits(void* s, const float* o, const float* d, uint64_t n, double* t_out, int64_t* prim_out) {
  const OScene& S = *(OScene*)s;
  for (uint64_t i = 0; i < n; ++i) {
    V3 oo{o[3 * i], o[3 * i + 1], o[3 * i + 2]}, dd{d[3 * i], d[3 * i + 1], d[3 * i + 2]};
    double t;
    uint32_t p;
    if (closest(S, oo, dd, &t, &p)) {
      t_out[i] = t;
      prim_out[i] = p;
    } else {
      t_out[i] = -1.0;
      prim_out[i] = -1;
    }
  }
}

void or_shadow_transmittance(void* s, const float* o, const float* d, const uint32_t* band, uint64_t n,
                             double* T_out, uint32_t* n_glass) {
  const OScene& S = *(OScene*)s;
  for (uint64_t i = 0; i < n; ++i) {
    V3 oo{o[3 * i], o[3 * i + 1], o[3 * i + 2]}, dd{d[3 * i], d[3 * i + 1], d[3 * i + 2]};
    T_out[i] = shadow_T(S, oo, dd, band[i], &n_glass[i]);
  }
}

// Renders the listed global pixels.  spectral_sum[i*band_count + j] receives
// the FP64 sum over samples (in sample order) of the path radiance of pixel
// pixels[i], band band_first + j.  path_L / path_sig (optional) receive every
// path's radiance and event signature, indexed [i][s][j].
int or_render(void* scene, const or_camera* cams, uint32_t n_cams, uint32_t band_first,
              uint32_t band_count, uint32_t spp, uint32_t depth, uint64_t seed, const uint32_t* pixels,
              uint64_t n_pixels, double* spectral_sum, double* path_L, uint32_t* path_sig,
              int n_threads) {
  const OScene& S = *(OScene*)scene;
  if (band_first + band_count > S.B || depth == 0) return 1;
  const std::vector<OCam> oc = setup_cams(cams, n_cams);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  std::atomic<uint64_t> next{0};
  auto worker = [&]() {
    for (;;) {
      uint64_t i = next.fetch_add(1);
      if (i >= n_pixels) break;
      uint32_t pix = pixels[i];
      for (uint32_t j = 0; j < band_count; ++j) spectral_sum[i * band_count + j] = 0.0;
      for (uint32_t s = 0; s < spp; ++s)
        for (uint32_t j = 0; j < band_count; ++j) {
          uint32_t sg = 0;
          double L = trace_path(S, oc, k0, k1, pix, s, band_first + j, depth, nullptr, path_sig ? &sg : nullptr,
                                nullptr);
          spectral_sum[i * band_count + j] += L;
          size_t pi = ((size_t)i * spp + s) * band_count + j;
          if (path_L) path_L[pi] = L;
          if (path_sig) path_sig[pi] = sg;
        }
    }
  };
  int nt = n_threads > 0 ? n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
  std::vector<std::thread> th;
  for (int i = 0; i < nt; ++i) th.emplace_back(worker);
  for (auto& t : th) t.join();
  return 0;
}

// Guide network of the guided estimator (FP64; bf16_act: the BF16 network).
void* or_guide_net_create(uint32_t log2_T, const float* lo, const float* hi, float n_min, float n_max,
                          const float* grid, const float* W, int bf16_act) {
  return oguide::net_create(log2_T, lo, hi, n_min, n_max, grid, W, bf16_act);
}

void or_guide_net_destroy(void* net) { oguide::net_destroy((oguide::Net*)net); }

// Guided render of the listed pixels: as or_render, with the continuation
// at Lambertian vertices 1..guide_depth drawn by one-sample MIS from the
// frozen guide `net` (probability alpha) and cosine sampling, and the sun at
// those vertices estimated by both strategies with the balance heuristic.
// records (optional) receives, per path [i][s][j] and guided vertex v, the
// two training records of v: [..][guide_depth][2][12] floats.
int or_render_guided(void* scene, void* net, double alpha, uint32_t guide_depth, const or_camera* cams,
                     uint32_t n_cams, uint32_t band_first, uint32_t band_count, uint32_t spp, uint32_t depth,
                     uint64_t seed, const uint32_t* pixels, uint64_t n_pixels, double* spectral_sum, double* path_L,
                     uint32_t* path_sig, float* records, int n_threads) {
  const OScene& S = *(OScene*)scene;
  if (band_first + band_count > S.B || depth == 0 || !net || guide_depth == 0 || guide_depth > 64) return 1;
  const std::vector<OCam> oc = setup_cams(cams, n_cams);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  GuideCtx g;
  g.net = (const oguide::Net*)net;
  g.alpha = alpha;
  g.depth = guide_depth;
  g.n_bands = S.B;
  const double p_cone = 1.0 / (2.0 * M_PI * (1.0 - S.cos_max));
  std::atomic<uint64_t> next{0};
  auto worker = [&]() {
    std::vector<GuidedSlot> slots(guide_depth);
    for (;;) {
      uint64_t i = next.fetch_add(1);
      if (i >= n_pixels) break;
      uint32_t pix = pixels[i];
      for (uint32_t j = 0; j < band_count; ++j) spectral_sum[i * band_count + j] = 0.0;
      for (uint32_t s = 0; s < spp; ++s)
        for (uint32_t j = 0; j < band_count; ++j) {
          uint32_t sg = 0;
          std::fill(slots.begin(), slots.end(), GuidedSlot());
          double L = trace_path(S, oc, k0, k1, pix, s, band_first + j, depth, &g, path_sig ? &sg : nullptr,
                                slots.data());
          spectral_sum[i * band_count + j] += L;
          size_t pi = ((size_t)i * spp + s) * band_count + j;
          if (path_L) path_L[pi] = L;
          if (path_sig) path_sig[pi] = sg;
          if (records)
            for (uint32_t v = 0; v < guide_depth; ++v)
              slot_records(slots[v], L, p_cone, records + (pi * guide_depth + v) * 24);
        }
    }
  };
  int nt = n_threads > 0 ? n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
  std::vector<std::thread> th;
  for (int i = 0; i < nt; ++i) th.emplace_back(worker);
  for (auto& t : th) t.join();
  return 0;
}

// One guided vertex per query, for checks of the sampler: query i is
// vertex k of the path (pixel[i], sample, band[i]) at offset position po[i]
// with normal nrm[i] and, when has_sun[i], a pending sun sample in
// direction wn[i].  out[i][16]: omega (3), q(omega), p_mix(omega), cos,
// guide (1) or cosine (0), lobe (or -1), lobe margin, balance weight of the
// sun sample, balance weight of a sun escape, continues (1/0), q(wn),
// p_mix(wn), 0, 0.
void or_guide_step(void* scene, void* net, double alpha, uint32_t k, uint32_t sample, uint64_t seed, uint64_t n,
                   const uint32_t* pixel, const uint32_t* band, const float* po, const float* nrm,
                   const uint32_t* has_sun, const float* wn, double* out) {
  const OScene& S = *(OScene*)scene;
  GuideCtx g;
  g.net = (const oguide::Net*)net;
  g.alpha = alpha;
  g.depth = 64;
  g.n_bands = S.B;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (uint64_t i = 0; i < n; ++i) {
    const V3 p{po[3 * i], po[3 * i + 1], po[3 * i + 2]}, nn{nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]};
    const V3 w{wn[3 * i], wn[3 * i + 1], wn[3 * i + 2]};
    const Ctr4 r0 = philox4x32_10(Ctr4{{pixel[i], sample, band[i], 4u * k}}, k0, k1);
    const Ctr4 r1 = philox4x32_10(Ctr4{{pixel[i], sample, band[i], 4u * k + 1u}}, k0, k1);
    const GuidedVertex gv = guided_vertex(g, S, p, nn, band[i] * 9u / S.B, r0, r1, has_sun[i] != 0, w);
    double* o = out + 16 * i;
    o[0] = gv.draw.omega.x;
    o[1] = gv.draw.omega.y;
    o[2] = gv.draw.omega.z;
    o[3] = gv.q;
    o[4] = gv.pdf;
    o[5] = gv.c;
    o[6] = gv.draw.guide ? 1.0 : 0.0;
    o[7] = gv.draw.lobe;
    o[8] = gv.draw.lobe_margin;
    o[9] = gv.nee_w;
    o[10] = gv.esc_w;
    o[11] = gv.cont ? 1.0 : 0.0;
    o[12] = gv.q_sun;
    o[13] = gv.pdf_sun;
    o[14] = 0.0;
    o[15] = 0.0;
  }
}

// Draws of the one-sample MIS proposal for fixed head outputs Y [48] and
// normal n, from caller-given uniforms u [n][6] (choice, lobe, two vMF, two
// cosine): omega [n][3] and p_mix(omega) [n].
void or_guide_mis_draws(const double* Y, const double* nrm, double alpha, uint64_t n, const double* u, double* omega,
                        double* pdf) {
  oguide::Mixture mx;
  oguide::mixture_of(Y, &mx);
  const V3 nn{nrm[0], nrm[1], nrm[2]};
  for (uint64_t i = 0; i < n; ++i) {
    const double* v = u + 6 * i;
    const MisDraw d = mis_draw(mx, nn, alpha, v[0], v[1], v[2], v[3], v[4], v[5]);
    omega[3 * i] = d.omega.x;
    omega[3 * i + 1] = d.omega.y;
    omega[3 * i + 2] = d.omega.z;
    pdf[i] = mis_pdf(mx, nn, alpha, d.omega, nullptr);
  }
}

// Primary rays of the listed (pixel, sample, band) triples: origins and unit
// directions [n][3] (the camera model of section 1's observer).
void or_camera_rays(const or_camera* cams, uint32_t n_cams, uint64_t seed, uint64_t n, const uint32_t* pix,
                    const uint32_t* sample, const uint32_t* band, double* o, double* d) {
  const std::vector<OCam> oc = setup_cams(cams, n_cams);
  for (uint64_t i = 0; i < n; ++i) {
    V3 oo, dd;
    camera_ray(oc, pix[i], sample[i], band[i], (uint32_t)seed, (uint32_t)(seed >> 32), &oo, &dd);
    o[3 * i] = oo.x;
    o[3 * i + 1] = oo.y;
    o[3 * i + 2] = oo.z;
    d[3 * i] = dd.x;
    d[3 * i + 1] = dd.y;
    d[3 * i + 2] = dd.z;
  }
}

// The same estimate with four bands per path: path unit g of a pixel and
// sample carries bands band_first + g + q G, q = 0..3, G = ceil(band_count
// / 4), those inside the range.  The bands share the path's geometry;
// Philox counters are those of band g.  At each
// vertex the "carried" bands are those with throughput != 0 (all existing
// bands if none is):
//   Lambertian / emissive: shared sun-ray direction and cosine continuation,
//     per-band emission, NEE (sun-ray transmittance per band) and rho;
//   thin glass: reflect if u < p = mean over carried bands of
//     R_s / (R_s + T_s); then each band is weighted R_s / p, else T_s / (1 - p);
//   conductor: mirror, each band weighted by its R;
//   solid glass: reflect if u < p = mean carried Fresnel R; each band
//     weighted R / p; else refraction, which bends every band differently:
//     the carried band of rank floor(u' m) (m carried bands) continues with
//     weight m (1 - R) / (1 - p), the others carry nothing further; a band
//     past its critical angle has R = 1 and so weight 0.
// Every choice keeps each band's one-band expectation.  spectral_sum,
// path_L and path_sig are laid out as in or_render.
int or_render4(void* scene, const or_camera* cams, uint32_t n_cams, uint32_t band_first, uint32_t band_count,
               uint32_t spp, uint32_t depth, uint64_t seed, const uint32_t* pixels, uint64_t n_pixels,
               double* spectral_sum, double* path_L, uint32_t* path_sig, int n_threads) {
  const OScene& S = *(OScene*)scene;
  if (band_first + band_count > S.B || depth == 0) return 1;
  const std::vector<OCam> oc = setup_cams(cams, n_cams);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const double cone_w = 2.0 * (1.0 - S.cos_max);
  const uint32_t groups = (band_count + 3) / 4;

  // radiance of bands b0 + q G, q < nv, of one path into L[0..nv)
  auto trace4 = [&](uint32_t pix, uint32_t s, uint32_t b0, uint32_t G, uint32_t nv, double* L, uint32_t* sig_out) {
    V3 o, d;
    camera_ray(oc, pix, s, b0, k0, k1, &o, &d);
    double T[4] = {0.0, 0.0, 0.0, 0.0};
    for (uint32_t q = 0; q < nv; ++q) {
      T[q] = 1.0;
      L[q] = 0.0;
    }
    bool covered = false;
    uint32_t sig = 2166136261u;
    for (uint32_t k = 1; k <= depth; ++k) {
      double t;
      uint32_t prim;
      if (!closest(S, o, d, &t, &prim)) {
        sig = mix(sig, 0xFFFFFFFFu);
        if (!covered && dot(d, S.sun) >= S.cos_max)
          for (uint32_t q = 0; q < nv; ++q) L[q] += T[q] * S.sunL[b0 + q * G];
        break;
      }
      sig = mix(sig, prim);
      V3 p = o + t * d;
      V3 ng = normalize(cross(S.b[prim] - S.a[prim], S.c[prim] - S.a[prim]));
      V3 n = dot(ng, d) < 0.0 ? ng : -1.0 * ng;
      double cos_i = -dot(d, n);
      uint32_t m = S.mat[prim];
      size_t mb = (size_t)m * S.B + b0;
      int type = S.mtype[m];
      // carried bands
      bool carried[4] = {false, false, false, false};
      uint32_t n_car = 0;
      for (uint32_t q = 0; q < nv; ++q)
        if (T[q] != 0.0) {
          carried[q] = true;
          ++n_car;
        }
      if (n_car == 0) {
        for (uint32_t q = 0; q < nv; ++q) carried[q] = true;
        n_car = nv;
      }
      Ctr4 r = philox4x32_10(Ctr4{{pix, s, b0, 4u * k}}, k0, k1);
      if (type == M_LAMBERT || type == M_EMISSIVE) {
        if (type == M_EMISSIVE)
          for (uint32_t q = 0; q < nv; ++q) L[q] += T[q] * S.le[mb + q * G];
        double ct = 1.0 - u01(r.w[0]) * (1.0 - S.cos_max);
        double st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
        double ph = 2.0 * M_PI * u01(r.w[1]);
        V3 t1, t2;
        onb(S.sun, &t1, &t2);
        V3 w = (st * std::cos(ph)) * t1 + (st * std::sin(ph)) * t2 + ct * S.sun;
        double c = dot(n, w);
        if (c > 0.0) {
          uint32_t ngl = 0;
          for (uint32_t q = 0; q < nv; ++q) {
            double Tr = shadow_T(S, p + S.eps * n, w, b0 + q * G, &ngl);
            L[q] += T[q] * S.rho[mb + q * G] * c * S.sunL[b0 + q * G] * cone_w * Tr;
          }
          sig = mix(sig, ngl);
        }
        if (k == depth) break;
        double rr = std::sqrt(u01(r.w[2]));
        double ph2 = 2.0 * M_PI * u01(r.w[3]);
        double z = std::sqrt(std::max(0.0, 1.0 - u01(r.w[2])));
        V3 b1, b2;
        onb(n, &b1, &b2);
        d = (rr * std::cos(ph2)) * b1 + (rr * std::sin(ph2)) * b2 + z * n;
        o = p + S.eps * n;
        for (uint32_t q = 0; q < nv; ++q) T[q] *= S.rho[mb + q * G];
        covered = true;
      } else if (type == M_GLASS) {
        double Rs[4], Ts[4];
        for (uint32_t q = 0; q < nv; ++q)
          slab(cos_i, S.ntab[mb + q * G], S.ktab[mb + q * G], S.lam[b0 + q * G], S.mthick[m], &Rs[q], &Ts[q]);
        if (k == depth) break;
        Ctr4 r1 = philox4x32_10(Ctr4{{pix, s, b0, 4u * k + 1u}}, k0, k1);
        double pr = 0.0;
        for (uint32_t q = 0; q < nv; ++q)
          if (carried[q]) pr += Rs[q] / (Rs[q] + Ts[q]);
        pr /= n_car;
        if (u01(r1.w[0]) < pr) {
          for (uint32_t q = 0; q < nv; ++q) T[q] *= Rs[q] / pr;
          d = d - (2.0 * dot(d, n)) * n;
          o = p + S.eps * n;
          covered = false;
        } else {
          for (uint32_t q = 0; q < nv; ++q) T[q] *= Ts[q] / (1.0 - pr);
          o = p - S.eps * n;
        }
      } else if (type == M_DIELECTRIC) {
        const bool inside = dot(ng, d) > 0.0;
        double alpha[4];
        for (uint32_t q = 0; q < nv; ++q) {
          alpha[q] = 4.0 * M_PI * S.ktab[mb + q * G] / (S.lam[b0 + q * G] * 1e-9);
          if (inside) T[q] *= std::exp(-alpha[q] * t);
        }
        if (k == depth) break;
        double R[4], eta[4];
        for (uint32_t q = 0; q < nv; ++q) {
          eta[q] = inside ? 1.0 / S.ntab[mb + q * G] : S.ntab[mb + q * G];
          R[q] = fresnel_complex(cos_i, eta[q], 0.0);
        }
        Ctr4 r1 = philox4x32_10(Ctr4{{pix, s, b0, 4u * k + 1u}}, k0, k1);
        double pr = 0.0;
        for (uint32_t q = 0; q < nv; ++q)
          if (carried[q]) pr += R[q];
        pr /= n_car;
        if (u01(r1.w[0]) < pr) {
          for (uint32_t q = 0; q < nv; ++q) T[q] *= R[q] / pr;
          d = d - (2.0 * dot(d, n)) * n;
        } else {
          const uint32_t rank = std::min((uint32_t)(u01(r1.w[1]) * n_car), n_car - 1);
          uint32_t c = 0, seen = 0;
          for (uint32_t q = 0; q < nv; ++q)
            if (carried[q]) {
              if (seen == rank) c = q;
              ++seen;
            }
          const double wgt = n_car * (1.0 - R[c]) / (1.0 - pr);
          for (uint32_t q = 0; q < nv; ++q) T[q] = q == c ? T[q] * wgt : 0.0;
          V3 tdir;
          if (refract(d, n, eta[c], &tdir)) d = normalize(tdir);
          else d = d - (2.0 * dot(d, n)) * n;  // R = 1: the weight is 0
        }
        const double step = S.eps / std::max(std::fabs(dot(d, n)), 0.0625);
        if (dot(d, ng) < 0.0)
          for (uint32_t q = 0; q < nv; ++q) T[q] *= std::exp(-alpha[q] * step);
        o = p + step * d;
        covered = false;
      } else {  // conductor
        double R[4];
        for (uint32_t q = 0; q < nv; ++q) R[q] = fresnel_complex(cos_i, S.ntab[mb + q * G], S.ktab[mb + q * G]);
        if (k == depth) break;
        d = d - (2.0 * dot(d, n)) * n;
        o = p + S.eps * n;
        for (uint32_t q = 0; q < nv; ++q) T[q] *= R[q];
        covered = false;
      }
    }
    if (sig_out) *sig_out = sig;
  };

  std::atomic<uint64_t> next{0};
  auto worker = [&]() {
    for (;;) {
      uint64_t i = next.fetch_add(1);
      if (i >= n_pixels) break;
      uint32_t pix = pixels[i];
      for (uint32_t j = 0; j < band_count; ++j) spectral_sum[i * band_count + j] = 0.0;
      for (uint32_t s = 0; s < spp; ++s)
        for (uint32_t g = 0; g < groups; ++g) {
          uint32_t nv = 0;
          while (nv < 4 && g + nv * groups < band_count) ++nv;
          double L[4];
          uint32_t sg = 0;
          trace4(pix, s, band_first + g, groups, nv, L, path_sig ? &sg : nullptr);
          for (uint32_t q = 0; q < nv; ++q) {
            const uint32_t j = g + q * groups;
            spectral_sum[i * band_count + j] += L[q];
            size_t pi = ((size_t)i * spp + s) * band_count + j;
            if (path_L) path_L[pi] = L[q];
            if (path_sig) path_sig[pi] = sg;
          }
        }
    }
  };
  int nt = n_threads > 0 ? n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
  std::vector<std::thread> th;
  for (int i = 0; i < nt; ++i) th.emplace_back(worker);
  for (auto& t : th) t.join();
  return 0;
}

// XYZ of spectral sums: xyz[i][c] = sum_j (spectral_sum[i][j] / spp) * cmf_w[band_first + j][c]
void or_xyz(const double* spectral_sum, uint64_t n_pixels, uint32_t band_first, uint32_t band_count,
            uint32_t spp, const float* cmf_w, double* xyz) {
  for (uint64_t i = 0; i < n_pixels; ++i)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (uint32_t j = 0; j < band_count; ++j)
        acc += spectral_sum[i * band_count + j] / spp * (double)cmf_w[(band_first + j) * 3 + c];
      xyz[i * 3 + c] = acc;
    }
}

// ---------------------------------------------------------------------------
// photon mapping (section 4: photon maps filled from the light source, then
// direct and specular light by ray tracing, caustic and indirect diffuse light
// from the maps)
// ---------------------------------------------------------------------------

}  // extern "C"

namespace {

enum { PH_NONE = 0, PH_DIRECT = 1, PH_CAUSTIC = 2, PH_INDIRECT = 3 };

struct PhotonRec {
  V3 x{0, 0, 0};
  double phi = 0.0;
  int cls = PH_NONE;
};

// Photon k-th diffuse hit slots: (j * N + i) * depth + k for band
// band_first + j, photon i.
//
// Emission: the sun is a cone of radiance L_sun(lambda) and half angle a
// around the unit direction s.  Photons start on a disk perpendicular to s,
// tangent to the scene's bounding sphere (centre c, radius R) on the sun's
// side: centre c + R s, radius R_d = R (tan a + 1 / cos a), wide enough that
// every ray within the cone that meets the sphere starts on it.  Position
// uniform on the disk (sqrt radius), direction -w with w uniform in the cone
// (the sun-sampling formula of NEE).  A photon carries the flux
// L_sun(lambda) cos(w, s) Omega pi R_d^2 / N, Omega = 2 pi (1 - cos a): the
// Monte Carlo estimate of the flux the cone sends through the disk.
//
// Tracing: as the camera paths (the same material rules); at a Lambertian
// (or emissive) hit the photon is stored, classed DIRECT (no event before it
// but thin-glass transmissions, which next-event estimation already
// covers), CAUSTIC (a reflection or refraction before its first diffuse hit)
// or INDIRECT (after a diffuse hit), then continues by cosine sampling with
// flux * rho.  Philox key (seed_lo, seed_hi ^ 0x50484F54), counter
// (photon i, band, 0, 4 k + call).
struct PhotonSetup {
  V3 c0, t1, t2;
  double Rd = 0.0, omega = 0.0;
  // portal emission: thin-glass triangles with their sun-side normal and
  // the cumulative share of A |s . n| (the last entry 1)
  std::vector<uint32_t> portal;
  std::vector<V3> portal_n;
  std::vector<double> cdf;
  double W = 0.0;  // sum of A |s . n|
};

PhotonSetup photon_setup(const OScene& S) {
  PhotonSetup P;
  const V3 c = 0.5 * (S.lo + S.hi);
  const double R = 0.5 * std::sqrt(dot(S.hi - S.lo, S.hi - S.lo));
  const double sa = std::sqrt(std::max(0.0, 1.0 - S.cos_max * S.cos_max));
  P.c0 = c + R * S.sun;
  P.Rd = R * (sa / S.cos_max + 1.0 / S.cos_max);
  P.omega = 2.0 * M_PI * (1.0 - S.cos_max);
  onb(S.sun, &P.t1, &P.t2);
  for (uint32_t t = 0; t < S.a.size(); ++t) {
    if (S.mtype[S.mat[t]] != M_GLASS) continue;
    const V3 c = cross(S.b[t] - S.a[t], S.c[t] - S.a[t]);
    const double area2 = std::sqrt(dot(c, c));
    if (!(area2 > 0.0)) continue;
    V3 n = (1.0 / area2) * c;
    const double cs = dot(n, S.sun);
    if (cs == 0.0) continue;
    if (cs < 0.0) n = -1.0 * n;
    P.portal.push_back(t);
    P.portal_n.push_back(n);
    P.W += 0.5 * area2 * std::fabs(cs);
    P.cdf.push_back(P.W);
  }
  for (double& x : P.cdf) x /= P.W;
  if (!P.cdf.empty()) P.cdf.back() = 1.0;
  return P;
}

// Portal emission (emission = 1), for interiors lit through thin glass: a
// photon starts on a thin-glass triangle chosen with probability
// proportional to A |s . n| (u0, the first triangle whose cumulative share
// exceeds u0), at a uniform point (u1, u2: barycentrics (1 - sqrt u1,
// sqrt u1 (1 - u2), sqrt u1 u2)), eps off its sun side, with w uniform in
// the cone (counter call 1); it carries L_sun |w . n| Omega W / (N |s . n|),
// W = sum A |s . n|, or nothing when w grazes the face from behind or the
// way back to the sun is blocked.  Sunlight that reaches the glass only
// after a bounce outside is not emitted.
void trace_photons(const OScene& S, uint32_t band_first, uint32_t band_count, uint32_t N, uint32_t depth,
                   uint64_t seed, std::vector<PhotonRec>& out, int n_threads, int emission = 0) {
  out.assign((size_t)band_count * N * depth, PhotonRec{});
  const PhotonSetup P = photon_setup(S);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) ^ 0x50484F54u;
  auto one = [&](uint32_t j, uint32_t i) {
    const uint32_t b = band_first + j;
    Ctr4 r0 = philox4x32_10(Ctr4{{i, b, 0u, 0u}}, k0, k1);
    V3 o, d;
    double phi;
    if (emission == 0) {
      const double rad = P.Rd * std::sqrt(u01(r0.w[0]));
      const double ph = 2.0 * M_PI * u01(r0.w[1]);
      o = P.c0 + (rad * std::cos(ph)) * P.t1 + (rad * std::sin(ph)) * P.t2;
      const double ct = 1.0 - u01(r0.w[2]) * (1.0 - S.cos_max);
      const double st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
      const double ph2 = 2.0 * M_PI * u01(r0.w[3]);
      V3 w = (st * std::cos(ph2)) * P.t1 + (st * std::sin(ph2)) * P.t2 + ct * S.sun;
      d = -1.0 * w;
      phi = S.sunL[b] * ct * P.omega * M_PI * P.Rd * P.Rd / N;
    } else {
      const double u0 = u01(r0.w[0]);
      size_t q = 0;
      while (q + 1 < P.cdf.size() && P.cdf[q] <= u0) ++q;
      const uint32_t t = P.portal[q];
      const V3 n = P.portal_n[q];
      const double su = std::sqrt(u01(r0.w[1])), u2 = u01(r0.w[2]);
      const V3 pg = (1.0 - su) * S.a[t] + (su * (1.0 - u2)) * S.b[t] + (su * u2) * S.c[t];
      Ctr4 r1 = philox4x32_10(Ctr4{{i, b, 0u, 1u}}, k0, k1);
      const double ct = 1.0 - u01(r1.w[0]) * (1.0 - S.cos_max);
      const double st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
      const double ph2 = 2.0 * M_PI * u01(r1.w[1]);
      V3 w = (st * std::cos(ph2)) * P.t1 + (st * std::sin(ph2)) * P.t2 + ct * S.sun;
      const double wn = dot(w, n);
      if (!(wn > 0.0)) return;
      o = pg + S.eps * n;
      double tb;
      uint32_t pb;
      if (closest(S, o, w, &tb, &pb)) return;  // the sun does not see this point
      d = -1.0 * w;
      phi = S.sunL[b] * wn * P.omega * P.W / (N * dot(S.sun, n));
    }
    bool nee_path = true;
    uint32_t n_diff = 0;
    const size_t slot0 = ((size_t)j * N + i) * depth;
    for (uint32_t k = 1; k <= depth; ++k) {
      double t;
      uint32_t prim;
      if (!closest(S, o, d, &t, &prim)) break;
      V3 p = o + t * d;
      V3 ng = normalize(cross(S.b[prim] - S.a[prim], S.c[prim] - S.a[prim]));
      V3 n = dot(ng, d) < 0.0 ? ng : -1.0 * ng;
      double cos_i = -dot(d, n);
      uint32_t m = S.mat[prim];
      size_t mb = (size_t)m * S.B + b;
      int type = S.mtype[m];
      Ctr4 r = philox4x32_10(Ctr4{{i, b, 0u, 4u * k}}, k0, k1);
      if (type == M_LAMBERT || type == M_EMISSIVE) {
        PhotonRec& rec = out[slot0 + n_diff];
        rec.x = p;
        rec.phi = phi;
        rec.cls = n_diff > 0 ? PH_INDIRECT : (nee_path ? PH_DIRECT : PH_CAUSTIC);
        ++n_diff;
        if (k == depth) break;
        double rr = std::sqrt(u01(r.w[2]));
        double ph3 = 2.0 * M_PI * u01(r.w[3]);
        double z = std::sqrt(std::max(0.0, 1.0 - u01(r.w[2])));
        V3 b1, b2;
        onb(n, &b1, &b2);
        d = (rr * std::cos(ph3)) * b1 + (rr * std::sin(ph3)) * b2 + z * n;
        o = p + S.eps * n;
        phi *= S.rho[mb];
      } else if (type == M_GLASS) {
        double Rs, Ts;
        slab(cos_i, S.ntab[mb], S.ktab[mb], S.lam[b], S.mthick[m], &Rs, &Ts);
        if (k == depth) break;
        Ctr4 r1 = philox4x32_10(Ctr4{{i, b, 0u, 4u * k + 1u}}, k0, k1);
        if (u01(r1.w[0]) < Rs / (Rs + Ts)) {
          d = d - (2.0 * dot(d, n)) * n;
          o = p + S.eps * n;
          nee_path = false;
        } else {
          o = p - S.eps * n;
        }
        phi *= Rs + Ts;
      } else if (type == M_DIELECTRIC) {
        const bool inside = dot(ng, d) > 0.0;
        const double alpha = 4.0 * M_PI * S.ktab[mb] / (S.lam[b] * 1e-9);
        if (inside) phi *= std::exp(-alpha * t);
        const double eta = inside ? 1.0 / S.ntab[mb] : S.ntab[mb];
        const double R = fresnel_complex(cos_i, eta, 0.0);
        if (k == depth) break;
        Ctr4 r1 = philox4x32_10(Ctr4{{i, b, 0u, 4u * k + 1u}}, k0, k1);
        V3 tdir;
        if (u01(r1.w[0]) < R || !refract(d, n, eta, &tdir)) d = d - (2.0 * dot(d, n)) * n;
        else d = normalize(tdir);
        const double step = S.eps / std::max(std::fabs(dot(d, n)), 0.0625);
        if (dot(d, ng) < 0.0) phi *= std::exp(-alpha * step);
        o = p + step * d;
        nee_path = false;
      } else {  // conductor
        double R = fresnel_complex(cos_i, S.ntab[mb], S.ktab[mb]);
        if (k == depth) break;
        d = d - (2.0 * dot(d, n)) * n;
        o = p + S.eps * n;
        phi *= R;
        nee_path = false;
      }
    }
  };
  std::atomic<uint64_t> next{0};
  const uint64_t total = (uint64_t)band_count * N;
  auto worker = [&]() {
    for (;;) {
      uint64_t g = next.fetch_add(1);
      if (g >= total) break;
      one((uint32_t)(g / N), (uint32_t)(g % N));
    }
  };
  int nt = n_threads > 0 ? n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
  std::vector<std::thread> th;
  for (int q = 0; q < nt; ++q) th.emplace_back(worker);
  for (auto& q : th) q.join();
}

// Photons of one band and class in a uniform grid of cell size r; the
// kernel-weighted flux sum over the photons within distance r of x (27 cells
// cover the ball), with the Epanechnikov weight 1 - d^2 / r^2.
struct PhotonGrid {
  double r = 0.0;
  std::unordered_map<int64_t, std::vector<uint32_t>> cells;
  static int64_t key(int64_t ix, int64_t iy, int64_t iz) {
    return ((ix + (1 << 20)) << 42) | ((iy + (1 << 20)) << 21) | (iz + (1 << 20));
  }
  void add(const PhotonRec& p, uint32_t id) {
    cells[key((int64_t)std::floor(p.x.x / r), (int64_t)std::floor(p.x.y / r), (int64_t)std::floor(p.x.z / r))]
        .push_back(id);
  }
  double flux_within(const std::vector<PhotonRec>& recs, V3 x) const {
    const int64_t cx = (int64_t)std::floor(x.x / r), cy = (int64_t)std::floor(x.y / r),
                  cz = (int64_t)std::floor(x.z / r);
    double sum = 0.0;
    for (int64_t a = -1; a <= 1; ++a)
      for (int64_t b = -1; b <= 1; ++b)
        for (int64_t c = -1; c <= 1; ++c) {
          auto it = cells.find(key(cx + a, cy + b, cz + c));
          if (it == cells.end()) continue;
          for (uint32_t id : it->second) {
            const V3 dx = recs[id].x - x;
            const double d2 = dot(dx, dx);
            if (d2 < r * r) sum += recs[id].phi * (1.0 - d2 / (r * r));
          }
        }
    return sum;
  }
};

}  // namespace

extern "C" {

// Photon records of the photon pass: pos_phi[slot] = (x, y, z, flux) and
// cls[slot] = 0 empty, 1 direct, 2 caustic, 3 indirect.
int or_photon_records(void* scene, uint32_t band_first, uint32_t band_count, uint32_t n_photons, uint32_t depth,
                      uint64_t seed, int emission, double* pos_phi, uint8_t* cls, int n_threads) {
  const OScene& S = *(OScene*)scene;
  if (band_first + band_count > S.B || depth == 0 || n_photons == 0) return 1;
  if (emission == 1 && photon_setup(S).portal.empty()) return 2;
  std::vector<PhotonRec> recs;
  trace_photons(S, band_first, band_count, n_photons, depth, seed, recs, n_threads, emission);
  for (size_t q = 0; q < recs.size(); ++q) {
    pos_phi[4 * q] = recs[q].x.x;
    pos_phi[4 * q + 1] = recs[q].x.y;
    pos_phi[4 * q + 2] = recs[q].x.z;
    pos_phi[4 * q + 3] = recs[q].phi;
    cls[q] = (uint8_t)recs[q].cls;
  }
  return 0;
}

// Photon-mapping render of the listed pixels (same layout as or_render):
// camera paths follow thin-glass, conductor and solid-glass events as in
// the path tracer; at the first Lambertian vertex they add emission, the
// next-event estimate of the sun and the photon estimate of the reflected
// light (rho / pi) E, the irradiance E a kernel density estimate over the
// photons of the path's band within each map's radius r:
//   E = sum_maps (2 / (pi r^2)) sum_{d < r} phi (1 - d^2 / r^2)
// (the Epanechnikov kernel, normalised over the disk of radius r; section 4
// names no kernel, and one that vanishes at r keeps the estimate continuous
// in the photon positions), and stop.
int or_photon_render(void* scene, const or_camera* cams, uint32_t n_cams, uint32_t band_first, uint32_t band_count,
                     uint32_t spp, uint32_t depth, uint64_t seed, uint32_t n_photons, uint32_t photon_depth,
                     double r_caustic, double r_global, int emission, const uint32_t* pixels, uint64_t n_pixels,
                     double* spectral_sum, double* path_L, uint32_t* path_sig, int n_threads) {
  const OScene& S = *(OScene*)scene;
  if (band_first + band_count > S.B || depth == 0 || photon_depth == 0 || n_photons == 0 || !(r_caustic > 0.0) ||
      !(r_global > 0.0))
    return 1;
  if (emission == 1 && photon_setup(S).portal.empty()) return 2;
  std::vector<PhotonRec> recs;
  trace_photons(S, band_first, band_count, n_photons, photon_depth, seed, recs, n_threads, emission);
  std::vector<PhotonGrid> caus(band_count), glob(band_count);
  const size_t per_band = (size_t)n_photons * photon_depth;
  for (uint32_t j = 0; j < band_count; ++j) {
    caus[j].r = r_caustic;
    glob[j].r = r_global;
    for (size_t q = j * per_band; q < (j + 1) * per_band; ++q) {
      if (recs[q].cls == PH_CAUSTIC) caus[j].add(recs[q], (uint32_t)q);
      else if (recs[q].cls == PH_INDIRECT) glob[j].add(recs[q], (uint32_t)q);
    }
  }
  const std::vector<OCam> oc = setup_cams(cams, n_cams);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const double cone_w = 2.0 * (1.0 - S.cos_max);
  auto trace = [&](uint32_t pix, uint32_t s, uint32_t j, uint32_t* sig_out) -> double {
    const uint32_t b = band_first + j;
    V3 o, d;
    camera_ray(oc, pix, s, b, k0, k1, &o, &d);
    double T = 1.0, L = 0.0;
    bool covered = false;
    uint32_t sig = 2166136261u;
    for (uint32_t k = 1; k <= depth; ++k) {
      double t;
      uint32_t prim;
      if (!closest(S, o, d, &t, &prim)) {
        sig = mix(sig, 0xFFFFFFFFu);
        if (!covered && dot(d, S.sun) >= S.cos_max) L += T * S.sunL[b];
        break;
      }
      sig = mix(sig, prim);
      V3 p = o + t * d;
      V3 ng = normalize(cross(S.b[prim] - S.a[prim], S.c[prim] - S.a[prim]));
      V3 n = dot(ng, d) < 0.0 ? ng : -1.0 * ng;
      double cos_i = -dot(d, n);
      uint32_t m = S.mat[prim];
      size_t mb = (size_t)m * S.B + b;
      int type = S.mtype[m];
      Ctr4 r = philox4x32_10(Ctr4{{pix, s, b, 4u * k}}, k0, k1);
      if (type == M_LAMBERT || type == M_EMISSIVE) {
        if (type == M_EMISSIVE) L += T * S.le[mb];
        double ct = 1.0 - u01(r.w[0]) * (1.0 - S.cos_max);
        double st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
        double ph = 2.0 * M_PI * u01(r.w[1]);
        V3 t1, t2;
        onb(S.sun, &t1, &t2);
        V3 w = (st * std::cos(ph)) * t1 + (st * std::sin(ph)) * t2 + ct * S.sun;
        double c = dot(n, w);
        if (c > 0.0) {
          uint32_t ngl;
          double Tr = shadow_T(S, p + S.eps * n, w, b, &ngl);
          sig = mix(sig, ngl);
          L += T * S.rho[mb] * c * S.sunL[b] * cone_w * Tr;
        }
        const double E = caus[j].flux_within(recs, p) * 2.0 / (M_PI * r_caustic * r_caustic) +
                         glob[j].flux_within(recs, p) * 2.0 / (M_PI * r_global * r_global);
        L += T * S.rho[mb] / M_PI * E;
        break;
      } else if (type == M_GLASS) {
        double Rs, Ts;
        slab(cos_i, S.ntab[mb], S.ktab[mb], S.lam[b], S.mthick[m], &Rs, &Ts);
        if (k == depth) break;
        Ctr4 r1 = philox4x32_10(Ctr4{{pix, s, b, 4u * k + 1u}}, k0, k1);
        if (u01(r1.w[0]) < Rs / (Rs + Ts)) {
          d = d - (2.0 * dot(d, n)) * n;
          o = p + S.eps * n;
          covered = false;
        } else {
          o = p - S.eps * n;
        }
        T *= Rs + Ts;
      } else if (type == M_DIELECTRIC) {
        const bool inside = dot(ng, d) > 0.0;
        const double alpha = 4.0 * M_PI * S.ktab[mb] / (S.lam[b] * 1e-9);
        if (inside) T *= std::exp(-alpha * t);
        const double eta = inside ? 1.0 / S.ntab[mb] : S.ntab[mb];
        const double R = fresnel_complex(cos_i, eta, 0.0);
        if (k == depth) break;
        Ctr4 r1 = philox4x32_10(Ctr4{{pix, s, b, 4u * k + 1u}}, k0, k1);
        V3 tdir;
        if (u01(r1.w[0]) < R || !refract(d, n, eta, &tdir)) d = d - (2.0 * dot(d, n)) * n;
        else d = normalize(tdir);
        const double step = S.eps / std::max(std::fabs(dot(d, n)), 0.0625);
        if (dot(d, ng) < 0.0) T *= std::exp(-alpha * step);
        o = p + step * d;
        covered = false;
      } else {
        double R = fresnel_complex(cos_i, S.ntab[mb], S.ktab[mb]);
        if (k == depth) break;
        d = d - (2.0 * dot(d, n)) * n;
        o = p + S.eps * n;
        T *= R;
        covered = false;
      }
    }
    if (sig_out) *sig_out = sig;
    return L;
  };
  std::atomic<uint64_t> next{0};
  auto worker = [&]() {
    for (;;) {
      uint64_t q = next.fetch_add(1);
      if (q >= n_pixels) break;
      uint32_t pix = pixels[q];
      for (uint32_t j = 0; j < band_count; ++j) spectral_sum[q * band_count + j] = 0.0;
      for (uint32_t s = 0; s < spp; ++s)
        for (uint32_t j = 0; j < band_count; ++j) {
          uint32_t sg = 0;
          double L = trace(pix, s, j, path_sig ? &sg : nullptr);
          spectral_sum[q * band_count + j] += L;
          size_t pi = ((size_t)q * spp + s) * band_count + j;
          if (path_L) path_L[pi] = L;
          if (path_sig) path_sig[pi] = sg;
        }
    }
  };
  int nt = n_threads > 0 ? n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
  std::vector<std::thread> th;
  for (int q = 0; q < nt; ++q) th.emplace_back(worker);
  for (auto& q : th) q.join();
  return 0;
}

int or_hardware_threads(void) { return (int)std::thread::hardware_concurrency(); }

}  // extern "C"

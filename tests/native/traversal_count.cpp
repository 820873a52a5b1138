// Traversal-cost counter (test helper, built by tests/test_bvh_host.py): builds
// the library's default tree (spatial-split BVH collapsed to four-wide nodes)
// from a scene dump, then traces on the CPU, in FP64, the rays a render makes:
// one camera ray per pixel, three cosine-sampled bounces (thin glass passed
// straight through) and, at every opaque vertex facing the sun, a sun ray
// sampled in the sun cone.  It counts four-wide node visits and triangle
// tests per ray with the GPU kernels' visit rules:
//   - closest hit: entered children nearest first, entries beyond the
//     current hit skipped;
//   - sun rays: entered children in slot order, stopping at the first opaque
//     triangle, for two slot orders: the collapse's own order (the first
//     entered child, then the others from the last slot down, as the
//     traversal visited them before the children were ordered) and children
//     stored far-to-near along the sun (box centre . sun, largest first,
//     empty slots last), visited in slot order.
// It also counts closest-hit rays over an eight-wide tree collapsed the same
// greedy way from the same binary tree, with exact child boxes and with
// child boxes quantised to 8 bits on a per-node power-of-two grid (rounded
// outward), the layout a wider, compressed node would use.
// Prints "closest <nodes/ray> <tris/ray> <rays>", "sun_build_order ...",
// "sun_far_first ...", "closest_w8 ..." and "closest_w8q ...".
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

#include "rt_bvh.h"

using namespace srt;

namespace {

struct Scene {
  std::vector<float> v;
  std::vector<uint32_t> t;
  std::vector<uint8_t> glass;
};

struct Count {
  double nodes = 0, tris = 0, rays = 0;
};

using V3 = std::array<double, 3>;

V3 sub(const float* a, const float* b) { return {(double)a[0] - b[0], (double)a[1] - b[1], (double)a[2] - b[2]}; }
V3 cross(const V3& a, const V3& b) {
  return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
double dot(const V3& a, const V3& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
V3 unit(V3 a) {
  const double l = std::sqrt(dot(a, a));
  return {a[0] / l, a[1] / l, a[2] / l};
}

// ray parameter of the hit on triangle id, or -1 (Moller-Trumbore in FP64)
double hit_t(const Scene& S, uint32_t id, const V3& o, const V3& d) {
  const float* a = &S.v[3 * S.t[3 * id]];
  const float* b = &S.v[3 * S.t[3 * id + 1]];
  const float* c = &S.v[3 * S.t[3 * id + 2]];
  const V3 e1 = sub(b, a), e2 = sub(c, a), s = {o[0] - a[0], o[1] - a[1], o[2] - a[2]};
  const V3 p = cross(d, e2);
  const double det = dot(e1, p);
  if (std::fabs(det) < 1e-20) return -1;
  const double u = dot(s, p) / det;
  if (u < 0 || u > 1) return -1;
  const V3 q = cross(s, e1);
  const double w = dot(d, q) / det;
  if (w < 0 || u + w > 1) return -1;
  return dot(e2, q) / det;
}

V3 normal(const Scene& S, uint32_t id) {
  const float* a = &S.v[3 * S.t[3 * id]];
  return unit(cross(sub(&S.v[3 * S.t[3 * id + 1]], a), sub(&S.v[3 * S.t[3 * id + 2]], a)));
}

// entry distance of child slot i (INFINITY if missed or empty)
double enter(const Bvh4Node& n, int i, const V3& o, const V3& inv, double tmax) {
  if (n.cnt[i] == kEmpty4) return INFINITY;
  const double lo[3] = {n.lox[i], n.loy[i], n.loz[i]}, hi[3] = {n.hix[i], n.hiy[i], n.hiz[i]};
  double tn = 0, tf = tmax;
  for (int a = 0; a < 3; ++a) {
    double t0 = (lo[a] - o[a]) * inv[a], t1 = (hi[a] - o[a]) * inv[a];
    if (t0 > t1) std::swap(t0, t1);
    tn = std::max(tn, t0);
    tf = std::min(tf, t1);
  }
  return tn <= tf ? tn : INFINITY;
}

V3 inverse(const V3& d) {
  V3 r;
  for (int a = 0; a < 3; ++a) r[a] = 1.0 / (std::fabs(d[a]) > 1e-20 ? d[a] : std::copysign(1e-20, d[a]));
  return r;
}

struct Entry {
  uint32_t ref, cnt;
  double t;
};

double closest(const std::vector<Bvh4Node>& B, const std::vector<uint32_t>& order, const Scene& S, const V3& o,
               const V3& d, uint32_t& hid, Count& C) {
  const V3 inv = inverse(d);
  std::vector<Entry> st;
  double best = INFINITY;
  hid = 0xFFFFFFFFu;
  uint32_t ref = 0, cnt = 0;
  C.rays += 1;
  for (;;) {
    if (cnt == 0) {
      const Bvh4Node& n = B[ref];
      C.nodes += 1;
      Entry e[4];
      int m = 0;
      for (int i = 0; i < 4; ++i) {
        const double t = enter(n, i, o, inv, best);
        if (t < INFINITY) e[m++] = {n.ref[i], n.cnt[i], t};
      }
      std::stable_sort(e, e + m, [](const Entry& a, const Entry& b) { return a.t < b.t; });
      if (m > 0) {
        for (int i = m - 1; i >= 1; --i) st.push_back(e[i]);
        ref = e[0].ref;
        cnt = e[0].cnt;
        continue;
      }
    } else {
      for (uint32_t k = ref; k < ref + cnt; ++k) {
        C.tris += 1;
        const uint32_t id = order[k];
        const double t = hit_t(S, id, o, d);
        if (t > 1e-9 && (t < best || (t == best && id < hid))) {
          best = t;
          hid = id;
        }
      }
    }
    bool next = false;
    while (!st.empty()) {
      const Entry e = st.back();
      st.pop_back();
      if (e.t <= best) {
        ref = e.ref;
        cnt = e.cnt;
        next = true;
        break;
      }
    }
    if (!next) return best;
  }
}

// sun ray; slot_order: entered children visited in slot order, else the
// first entered one, then the others from the last slot down
void sun_ray(const std::vector<Bvh4Node>& B, const std::vector<uint32_t>& order, const Scene& S, const V3& o,
             const V3& d, bool slot_order, Count& C) {
  const V3 inv = inverse(d);
  std::vector<std::pair<uint32_t, uint32_t>> st;
  uint32_t ref = 0, cnt = 0;
  C.rays += 1;
  for (;;) {
    if (cnt == 0) {
      const Bvh4Node& n = B[ref];
      C.nodes += 1;
      int ent[4], m = 0;
      for (int i = 0; i < 4; ++i)
        if (enter(n, i, o, inv, INFINITY) < INFINITY) ent[m++] = i;
      if (m > 0) {
        if (slot_order)
          for (int q = m - 1; q >= 1; --q) st.push_back({n.ref[ent[q]], n.cnt[ent[q]]});
        else
          for (int q = 1; q < m; ++q) st.push_back({n.ref[ent[q]], n.cnt[ent[q]]});
        ref = n.ref[ent[0]];
        cnt = n.cnt[ent[0]];
        continue;
      }
    } else {
      for (uint32_t k = ref; k < ref + cnt; ++k) {
        C.tris += 1;
        const uint32_t id = order[k];
        if (!S.glass[id] && hit_t(S, id, o, d) > 1e-9) return;
      }
    }
    if (st.empty()) return;
    ref = st.back().first;
    cnt = st.back().second;
    st.pop_back();
  }
}

// children of every node far-to-near along s, empty slots last, ties by
// (ref, cnt) of the child
std::vector<Bvh4Node> far_first(std::vector<Bvh4Node> B, const V3& s) {
  for (Bvh4Node& n : B) {
    int idx[4] = {0, 1, 2, 3};
    double key[4];
    for (int c = 0; c < 4; ++c)
      key[c] = n.cnt[c] == kEmpty4 ? -INFINITY
                                    : (n.lox[c] + n.hix[c]) * s[0] + (n.loy[c] + n.hiy[c]) * s[1] +
                                          (n.loz[c] + n.hiz[c]) * s[2];
    std::sort(idx, idx + 4, [&](int a, int b) {
      if (key[a] != key[b]) return key[a] > key[b];
      if (n.ref[a] != n.ref[b]) return n.ref[a] > n.ref[b];
      if (n.cnt[a] != n.cnt[b]) return n.cnt[a] > n.cnt[b];
      return a < b;
    });
    Bvh4Node o = n;
    for (int r = 0; r < 4; ++r) {
      const int c = idx[r];
      o.lox[r] = n.lox[c];
      o.hix[r] = n.hix[c];
      o.loy[r] = n.loy[c];
      o.hiy[r] = n.hiy[c];
      o.loz[r] = n.loz[c];
      o.hiz[r] = n.hiz[c];
      o.ref[r] = n.ref[c];
      o.cnt[r] = n.cnt[c];
    }
    n = o;
  }
  return B;
}

// W-wide tree by the greedy collapse (open the interior child of largest
// area until W children); child boxes exact or quantised
struct WideNode {
  std::vector<std::array<double, 6>> box;  // lo xyz, hi xyz per child
  std::vector<int> child;                  // wide node index, or -1 for a leaf
  std::vector<uint32_t> first, count;      // leaf runs of the leaf order
};

std::vector<WideNode> collapse_wide(const BvhOut& b2, int W, bool quantise) {
  const std::vector<BvhNode>& nb = b2.nodes;
  auto area = [&](uint32_t i) {
    const BvhNode& b = nb[i];
    const double dx = b.hi[0] - b.lo[0], dy = b.hi[1] - b.lo[1], dz = b.hi[2] - b.lo[2];
    return 2.0 * (dx * dy + dy * dz + dz * dx);
  };
  std::vector<WideNode> out(1);
  std::vector<std::pair<uint32_t, int>> todo{{1u, 0}};
  while (!todo.empty()) {
    const auto [b, slot] = todo.back();
    todo.pop_back();
    std::vector<uint32_t> ch;
    if (nb[b].count != 0) {
      ch.push_back(b);
    } else {
      ch = {nb[b].ref, nb[b].ref + 1};
      while ((int)ch.size() < W) {
        int best = -1;
        double ba = -1.0;
        for (int i = 0; i < (int)ch.size(); ++i)
          if (nb[ch[i]].count == 0 && area(ch[i]) > ba) {
            ba = area(ch[i]);
            best = i;
          }
        if (best < 0) break;
        const uint32_t r = nb[ch[best]].ref;
        ch[best] = r;
        ch.push_back(r + 1);
      }
    }
    WideNode w;
    double L[3] = {INFINITY, INFINITY, INFINITY}, Hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (const uint32_t c : ch)
      for (int a = 0; a < 3; ++a) {
        L[a] = std::min(L[a], (double)nb[c].lo[a]);
        Hi[a] = std::max(Hi[a], (double)nb[c].hi[a]);
      }
    double scale[3];
    for (int a = 0; a < 3; ++a) scale[a] = std::ldexp(1.0, (int)std::ceil(std::log2(std::max(Hi[a] - L[a], 1e-30) / 255.0)));
    for (const uint32_t c : ch) {
      std::array<double, 6> bx;
      for (int a = 0; a < 3; ++a) {
        bx[a] = nb[c].lo[a];
        bx[3 + a] = nb[c].hi[a];
        if (quantise) {
          const double ql = std::min(255.0, std::max(0.0, std::floor((bx[a] - L[a]) / scale[a])));
          const double qh = std::min(255.0, std::max(0.0, std::ceil((bx[3 + a] - L[a]) / scale[a])));
          bx[a] = L[a] + ql * scale[a];
          bx[3 + a] = L[a] + qh * scale[a];
        }
      }
      w.box.push_back(bx);
      if (nb[c].count != 0) {
        w.child.push_back(-1);
        w.first.push_back(nb[c].ref);
        w.count.push_back(nb[c].count);
      } else {
        w.child.push_back((int)out.size());
        w.first.push_back(0);
        w.count.push_back(0);
        todo.push_back({c, (int)out.size()});
        out.emplace_back();
      }
    }
    out[slot] = std::move(w);
  }
  return out;
}

double closest_wide(const std::vector<WideNode>& T, const std::vector<uint32_t>& order, const Scene& S, const V3& o,
                    const V3& d, Count& C) {
  const V3 inv = inverse(d);
  struct E {
    int node;
    uint32_t first, count;
    double t;
  };
  std::vector<E> st;
  double best = INFINITY;
  uint32_t hid = 0xFFFFFFFFu;
  E cur{0, 0, 0, 0.0};
  C.rays += 1;
  for (;;) {
    if (cur.node >= 0) {
      const WideNode& n = T[cur.node];
      C.nodes += 1;
      std::vector<E> e;
      for (size_t i = 0; i < n.box.size(); ++i) {
        double tn = 0, tf = best;
        for (int a = 0; a < 3; ++a) {
          double t0 = (n.box[i][a] - o[a]) * inv[a], t1 = (n.box[i][3 + a] - o[a]) * inv[a];
          if (t0 > t1) std::swap(t0, t1);
          tn = std::max(tn, t0);
          tf = std::min(tf, t1);
        }
        if (tn <= tf) e.push_back({n.child[i], n.first[i], n.count[i], tn});
      }
      std::stable_sort(e.begin(), e.end(), [](const E& a, const E& b) { return a.t < b.t; });
      if (!e.empty()) {
        for (size_t i = e.size() - 1; i >= 1; --i) st.push_back(e[i]);
        cur = e[0];
        continue;
      }
    } else {
      for (uint32_t k = cur.first; k < cur.first + cur.count; ++k) {
        C.tris += 1;
        const uint32_t id = order[k];
        const double t = hit_t(S, id, o, d);
        if (t > 1e-9 && (t < best || (t == best && id < hid))) {
          best = t;
          hid = id;
        }
      }
    }
    bool next = false;
    while (!st.empty()) {
      const E e = st.back();
      st.pop_back();
      if (e.t <= best) {
        cur = e;
        next = true;
        break;
      }
    }
    if (!next) return best;
  }
}

// orthonormal vectors t1, t2 with n
void basis(const V3& n, V3& t1, V3& t2) {
  const double sg = std::copysign(1.0, n[2]);
  const double a = -1.0 / (sg + n[2]), b = n[0] * n[1] * a;
  t1 = {1 + sg * n[0] * n[0] * a, sg * b, -sg * n[0]};
  t2 = {b, sg + n[1] * n[1] * a, -n[1]};
}

}  // namespace

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  uint32_t nv = 0, nt = 0, W = 0, H = 0;
  if (fread(&nv, 4, 1, f) != 1 || fread(&nt, 4, 1, f) != 1) return 2;
  Scene S;
  S.v.resize(3 * (size_t)nv);
  S.t.resize(3 * (size_t)nt);
  S.glass.resize(nt);
  float cam[10], sunf[4];
  if (fread(S.v.data(), 4, S.v.size(), f) != S.v.size() || fread(S.t.data(), 4, S.t.size(), f) != S.t.size() ||
      fread(S.glass.data(), 1, nt, f) != nt || fread(cam, 4, 10, f) != 10 || fread(&W, 4, 1, f) != 1 ||
      fread(&H, 4, 1, f) != 1 || fread(sunf, 4, 4, f) != 4)
    return 2;
  fclose(f);
  std::vector<uint8_t> split(nt);
  for (uint32_t i = 0; i < nt; ++i) split[i] = !S.glass[i];
  BvhOut b2;
  build_sbvh(S.v.data(), S.t.data(), nt, split.data(), b2);
  std::vector<Bvh4Node> B;
  collapse_bvh4(b2, B, nullptr);
  const V3 sun = unit({sunf[0], sunf[1], sunf[2]});
  const double cos_max = std::cos((double)sunf[3]);
  const std::vector<Bvh4Node> Bf = far_first(B, sun);
  const std::vector<WideNode> W8 = collapse_wide(b2, 8, false), W8q = collapse_wide(b2, 8, true);

  // camera (pinhole, vertical field of view, y down)
  const V3 pos = {cam[0], cam[1], cam[2]};
  const V3 fw = unit({cam[3] - cam[0], cam[4] - cam[1], cam[5] - cam[2]});
  const V3 rt = unit(cross(fw, {cam[6], cam[7], cam[8]}));
  const V3 up = cross(rt, fw);
  const double th = std::tan(0.5 * cam[9] * M_PI / 180.0), asp = (double)W / H;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (size_t i = 0; i < S.v.size(); ++i) {
    lo[i % 3] = std::min(lo[i % 3], (double)S.v[i]);
    hi[i % 3] = std::max(hi[i % 3], (double)S.v[i]);
  }
  const double eps = 1e-4 * std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                      (hi[2] - lo[2]) * (hi[2] - lo[2]));
  V3 s1, s2;
  basis(sun, s1, s2);
  std::mt19937_64 rng(3);
  std::uniform_real_distribution<double> U(0, 1);
  Count ext, sun_build, sun_far, ext8, ext8q;
  for (uint32_t y = 0; y < H; ++y)
    for (uint32_t x = 0; x < W; ++x) {
      const double px = (2.0 * (x + U(rng)) / W - 1.0) * th * asp, py = (1.0 - 2.0 * (y + U(rng)) / H) * th;
      V3 o = pos, d = unit({fw[0] + px * rt[0] + py * up[0], fw[1] + px * rt[1] + py * up[1],
                            fw[2] + px * rt[2] + py * up[2]});
      for (int vtx = 0; vtx < 4; ++vtx) {
        uint32_t id;
        const double t = closest(B, b2.order, S, o, d, id, ext);
        const double t8 = closest_wide(W8, b2.order, S, o, d, ext8), t8q = closest_wide(W8q, b2.order, S, o, d, ext8q);
        if (!(t8 == t && t8q == t)) {
          printf("wide trees disagree with the four-wide tree: %.17g %.17g %.17g\n", t, t8, t8q);
          return 1;
        }
        if (!(t < INFINITY)) break;
        V3 n = normal(S, id);
        if (dot(n, d) > 0) n = {-n[0], -n[1], -n[2]};
        const V3 p = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        if (S.glass[id]) {  // through the sheet, same direction
          o = {p[0] - eps * n[0], p[1] - eps * n[1], p[2] - eps * n[2]};
          continue;
        }
        o = {p[0] + eps * n[0], p[1] + eps * n[1], p[2] + eps * n[2]};
        const double cz = 1 - U(rng) * (1 - cos_max), sz = std::sqrt(std::max(0.0, 1 - cz * cz));
        const double ph = 2 * M_PI * U(rng);
        const V3 sd = {cz * sun[0] + sz * (std::cos(ph) * s1[0] + std::sin(ph) * s2[0]),
                       cz * sun[1] + sz * (std::cos(ph) * s1[1] + std::sin(ph) * s2[1]),
                       cz * sun[2] + sz * (std::cos(ph) * s1[2] + std::sin(ph) * s2[2])};
        if (dot(n, sd) > 0) {
          sun_ray(B, b2.order, S, o, sd, false, sun_build);
          sun_ray(Bf, b2.order, S, o, sd, true, sun_far);
        }
        V3 t1, t2;
        basis(n, t1, t2);
        const double u1 = U(rng), r = std::sqrt(u1), phi = 2 * M_PI * U(rng);
        const double lx = r * std::cos(phi), ly = r * std::sin(phi), lz = std::sqrt(std::max(0.0, 1 - u1));
        d = unit({lx * t1[0] + ly * t2[0] + lz * n[0], lx * t1[1] + ly * t2[1] + lz * n[1],
                  lx * t1[2] + ly * t2[2] + lz * n[2]});
      }
    }
  printf("closest %.4f %.4f %.0f\n", ext.nodes / ext.rays, ext.tris / ext.rays, ext.rays);
  printf("sun_build_order %.4f %.4f %.0f\n", sun_build.nodes / sun_build.rays, sun_build.tris / sun_build.rays,
         sun_build.rays);
  printf("sun_far_first %.4f %.4f %.0f\n", sun_far.nodes / sun_far.rays, sun_far.tris / sun_far.rays, sun_far.rays);
  printf("closest_w8 %.4f %.4f %.0f\n", ext8.nodes / ext8.rays, ext8.tris / ext8.rays, ext8.rays);
  printf("closest_w8q %.4f %.4f %.0f\n", ext8q.nodes / ext8q.rays, ext8q.tris / ext8q.rays, ext8q.rays);
  return 0;
}

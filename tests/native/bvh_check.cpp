// Structural checks of the host BVH builders (test helper, built by
// tests/test_bvh_host.py): reads a scene dump, builds the plain SAH tree and
// the spatial-split tree, and checks for each that
//   - every triangle is referenced by a leaf, a non-splittable one exactly once;
//   - every node box contains its children's boxes;
//   - every sampled point of a triangle (vertices, edge midpoints, centroid and
//     a seeded set of interior points) lies in the box of some leaf that
//     references the triangle, so a traversal reaches the triangle wherever a
//     ray meets it;
//   - the four-wide collapse reaches every node once, its leaves (1..4
//     references each) tile the leaf order exactly, child boxes nest, and
//     every sampled point of a triangle lies in the box of a wide leaf that
//     references it;
//   - the spatial-split build on one thread gives the same tree bit for bit.
// Prints one line per tree: "<name> ok refs=<n> nodes4=<m>" or the failure.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <array>
#include <random>
#include <vector>

#include "rt_bvh.h"

using namespace srt;

static bool inside(const BvhNode& b, const double p[3], double tol) {
  for (int a = 0; a < 3; ++a)
    if (p[a] < b.lo[a] - tol || p[a] > b.hi[a] + tol) return false;
  return true;
}

static std::vector<std::array<double, 3>> sample_points(const std::vector<float>& v, const std::vector<uint32_t>& t,
                                                       uint32_t i, std::mt19937& rng) {
  std::uniform_real_distribution<double> U(0.0, 1.0);
  const float* P[3] = {&v[3 * t[3 * i]], &v[3 * t[3 * i + 1]], &v[3 * t[3 * i + 2]]};
  std::vector<std::array<double, 3>> pts;
  auto add = [&](double a, double b2, double c) {
    std::array<double, 3> p;
    for (int k = 0; k < 3; ++k) p[k] = a * P[0][k] + b2 * P[1][k] + c * P[2][k];
    pts.push_back(p);
  };
  add(1, 0, 0);
  add(0, 1, 0);
  add(0, 0, 1);
  add(0.5, 0.5, 0);
  add(0, 0.5, 0.5);
  add(0.5, 0, 0.5);
  add(1.0 / 3, 1.0 / 3, 1.0 / 3);
  for (int s = 0; s < 8; ++s) {
    const double su = std::sqrt(U(rng)), u2 = U(rng);
    add(1 - su, su * (1 - u2), su * u2);
  }
  return pts;
}

static int check4(const char* name, const std::vector<Bvh4Node>& b4, const std::vector<uint32_t>& order,
                  const std::vector<float>& v, const std::vector<uint32_t>& t, uint32_t nt) {
  if (b4.empty()) {
    printf("%s: empty four-wide tree\n", name);
    return 1;
  }
  std::vector<char> seen(b4.size(), 0);
  std::vector<std::pair<uint32_t, uint32_t>> runs;        // (first, count) of every wide leaf
  std::vector<std::vector<std::array<uint32_t, 2>>> leaves_of(nt);  // (node, slot) of the leaves holding t
  std::vector<uint32_t> stack{0};
  seen[0] = 1;
  size_t reached = 1;
  while (!stack.empty()) {
    const uint32_t n = stack.back();
    stack.pop_back();
    const Bvh4Node& nd = b4[n];
    for (uint32_t i = 0; i < 4; ++i) {
      if (nd.cnt[i] == kEmpty4) continue;
      if (nd.cnt[i] == 0) {
        const uint32_t c = nd.ref[i];
        if (c == 0 || c >= b4.size() || seen[c]) {
          printf("%s: wide node %u child %u reaches node %u twice or out of range\n", name, n, i, c);
          return 1;
        }
        seen[c] = 1;
        ++reached;
        stack.push_back(c);
        const Bvh4Node& cn = b4[c];
        for (int g = 0; g < 4; ++g) {
          if (cn.cnt[g] == kEmpty4) continue;
          if (cn.lox[g] < nd.lox[i] || cn.loy[g] < nd.loy[i] || cn.loz[g] < nd.loz[i] || cn.hix[g] > nd.hix[i] ||
              cn.hiy[g] > nd.hiy[i] || cn.hiz[g] > nd.hiz[i]) {
            printf("%s: wide child box outside its parent slot at node %u\n", name, c);
            return 1;
          }
        }
      } else {
        if (nd.cnt[i] > 4 || (size_t)nd.ref[i] + nd.cnt[i] > order.size()) {
          printf("%s: wide leaf (%u, %u) out of range\n", name, nd.ref[i], nd.cnt[i]);
          return 1;
        }
        runs.push_back({nd.ref[i], nd.cnt[i]});
        for (uint32_t k = 0; k < nd.cnt[i]; ++k) leaves_of[order[nd.ref[i] + k]].push_back({n, i});
      }
    }
  }
  if (reached != b4.size()) {
    printf("%s: %zu of %zu wide nodes reached\n", name, reached, b4.size());
    return 1;
  }
  std::sort(runs.begin(), runs.end());
  uint32_t next = 0;
  for (const auto& r : runs) {
    if (r.first != next) {
      printf("%s: wide leaves do not tile the leaf order at %u\n", name, next);
      return 1;
    }
    next += r.second;
  }
  if (next != order.size()) {
    printf("%s: wide leaves cover %u of %zu references\n", name, next, order.size());
    return 1;
  }
  std::mt19937 rng(11);
  double ext = 0.0;
  for (size_t i = 0; i < v.size(); ++i) ext = std::max(ext, std::fabs((double)v[i]));
  const double tol = 1e-6 * (ext + 1.0);
  for (uint32_t i = 0; i < nt; ++i) {
    for (const auto& p : sample_points(v, t, i, rng)) {
      bool found = false;
      for (const auto& L : leaves_of[i]) {
        const Bvh4Node& nd = b4[L[0]];
        const uint32_t s = L[1];
        if (p[0] >= nd.lox[s] - tol && p[0] <= nd.hix[s] + tol && p[1] >= nd.loy[s] - tol &&
            p[1] <= nd.hiy[s] + tol && p[2] >= nd.loz[s] - tol && p[2] <= nd.hiz[s] + tol) {
          found = true;
          break;
        }
      }
      if (!found) {
        printf("%s: a point of triangle %u lies in none of its wide leaves\n", name, i);
        return 1;
      }
    }
  }
  return 0;
}

static int check(const char* name, const BvhOut& o, const std::vector<float>& v, const std::vector<uint32_t>& t,
                 const std::vector<uint8_t>& split, uint32_t nt) {
  std::vector<int> cnt(nt, 0);
  for (uint32_t x : o.order) {
    if (x >= nt) {
      printf("%s: reference out of range\n", name);
      return 1;
    }
    cnt[x]++;
  }
  for (uint32_t i = 0; i < nt; ++i) {
    if (cnt[i] == 0) {
      printf("%s: triangle %u not referenced\n", name, i);
      return 1;
    }
    if (!split[i] && cnt[i] != 1) {
      printf("%s: unsplittable triangle %u referenced %d times\n", name, i, cnt[i]);
      return 1;
    }
  }
  // leaves referencing each triangle, child boxes inside parents
  std::vector<std::vector<uint32_t>> leaves_of(nt);
  size_t leaf_refs = 0;
  for (size_t i = 1; i < o.nodes.size(); ++i) {
    const BvhNode& b = o.nodes[i];
    if (b.count) {
      for (uint32_t k = 0; k < b.count; ++k) leaves_of[o.order[b.ref + k]].push_back((uint32_t)i);
      leaf_refs += b.count;
    } else if (b.ref) {
      for (int c = 0; c < 2; ++c) {
        const BvhNode& ch = o.nodes[b.ref + c];
        for (int a = 0; a < 3; ++a)
          if (ch.lo[a] < b.lo[a] || ch.hi[a] > b.hi[a]) {
            printf("%s: child box outside its parent at node %zu\n", name, i);
            return 1;
          }
      }
    }
  }
  if (leaf_refs != o.order.size()) {
    printf("%s: leaves hold %zu of %zu references\n", name, leaf_refs, o.order.size());
    return 1;
  }
  std::mt19937 rng(7);
  double ext = 0.0;
  for (size_t i = 0; i < v.size(); ++i) ext = std::max(ext, std::fabs((double)v[i]));
  const double tol = 1e-6 * (ext + 1.0);
  for (uint32_t i = 0; i < nt; ++i) {
    const std::vector<std::array<double, 3>> pts = sample_points(v, t, i, rng);
    for (const auto& p : pts) {
      bool found = false;
      for (uint32_t L : leaves_of[i])
        if (inside(o.nodes[L], p.data(), tol)) {
          found = true;
          break;
        }
      if (!found) {
        printf("%s: a point of triangle %u lies in none of its leaves\n", name, i);
        return 1;
      }
    }
  }
  std::vector<Bvh4Node> b4;
  collapse_bvh4(o, b4, nullptr);
  char wide[64];
  std::snprintf(wide, sizeof wide, "%s four-wide", name);
  if (check4(wide, b4, o.order, v, t, nt)) return 1;
  printf("%s ok refs=%zu nodes4=%zu\n", name, o.order.size(), b4.size());
  return 0;
}

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  uint32_t nv = 0, nt = 0;
  if (fread(&nv, 4, 1, f) != 1 || fread(&nt, 4, 1, f) != 1) return 2;
  std::vector<float> v(3 * (size_t)nv);
  std::vector<uint32_t> t(3 * (size_t)nt);
  std::vector<uint8_t> split(nt);
  if (fread(v.data(), 4, v.size(), f) != v.size() || fread(t.data(), 4, t.size(), f) != t.size() ||
      fread(split.data(), 1, nt, f) != nt)
    return 2;
  fclose(f);
  BvhOut a, b;
  build_bvh(v.data(), t.data(), nt, a);
  build_sbvh(v.data(), t.data(), nt, split.data(), b);
  int rc = check("sah", a, v, t, split, nt);
  rc |= check("sbvh", b, v, t, split, nt);
  // the spatial-split build on one thread: the same tree bit for bit
  BvhOut b1;
  build_sbvh(v.data(), t.data(), nt, split.data(), b1, 1);
  const bool same = b1.order == b.order && b1.nodes.size() == b.nodes.size() &&
                    std::memcmp(b1.nodes.data(), b.nodes.data(), b.nodes.size() * sizeof(BvhNode)) == 0;
  printf(same ? "sbvh one thread: same tree\n" : "sbvh one thread: a different tree\n");
  rc |= same ? 0 : 1;
  return rc;
}

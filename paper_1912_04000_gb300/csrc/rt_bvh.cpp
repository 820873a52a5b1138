// Binned SAH BVH2 builder (host, C++17), flattened to 32-byte nodes, and its
// collapse to a four-wide BVH.
//
// Method: binned surface-area heuristic over triangle centroids (Wald, "On
// fast construction of SAH-based bounding volume hierarchies", IEEE RT 2007),
// 32 bins per axis, leaves of at most 4 triangles.  Past depth 40 the builder
// switches to median splits so the tree depth, and with it the traversal
// stack, stays below 64.
//
// Layout (what the traversal kernels read): node i = {lo.xyz, ref}, {hi.xyz,
// count}; node 1 is the root; an interior node (count 0) has its two children
// at nodes ref and ref + 1 with ref even, so a sibling pair is one aligned
// 64-byte line; a leaf holds `count` triangles from position `ref` of the
// leaf-ordered triangle list.
//
// collapse_bvh4 turns the binary tree into a four-wide one (128-byte nodes,
// one cache line each) with the same leaves, which the default traversal
// reads: half the dependent node fetches per ray.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "rt_bvh.h"

namespace srt {

namespace {

struct Box {
  float lo[3] = {INFINITY, INFINITY, INFINITY};
  float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  void grow(const Box& b) {
    for (int i = 0; i < 3; ++i) {
      lo[i] = std::min(lo[i], b.lo[i]);
      hi[i] = std::max(hi[i], b.hi[i]);
    }
  }
  void grow(const float* p) {
    for (int i = 0; i < 3; ++i) {
      lo[i] = std::min(lo[i], p[i]);
      hi[i] = std::max(hi[i], p[i]);
    }
  }
  double area() const {
    if (!(lo[0] <= hi[0])) return 0.0;
    double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    return 2.0 * (dx * dy + dy * dz + dz * dx);
  }
};

struct Task {
  uint32_t node, begin, end, depth;
};

constexpr int kBins = 32;
constexpr uint32_t kMaxLeaf = 4;
constexpr uint32_t kMedianDepth = 40;

}  // namespace

int build_bvh(const float* verts, const uint32_t* tris, uint32_t nt, BvhOut& out) {
  std::vector<Box> tb(nt);
  std::vector<float> cen(3 * (size_t)nt);
  for (uint32_t t = 0; t < nt; ++t) {
    for (int v = 0; v < 3; ++v) tb[t].grow(verts + 3 * (size_t)tris[3 * (size_t)t + v]);
    for (int i = 0; i < 3; ++i) cen[3 * (size_t)t + i] = 0.5f * (tb[t].lo[i] + tb[t].hi[i]);
  }
  std::vector<uint32_t> idx(nt);
  for (uint32_t i = 0; i < nt; ++i) idx[i] = i;

  out.nodes.assign(2, BvhNode{});
  out.nodes.reserve(2 * (size_t)nt + 2);
  std::vector<Task> stack;
  stack.push_back({1, 0, nt, 0});
  uint32_t max_depth = 0;
  std::vector<uint32_t> bin_of;
  while (!stack.empty()) {
    Task tk = stack.back();
    stack.pop_back();
    max_depth = std::max(max_depth, tk.depth);
    const uint32_t n = tk.end - tk.begin;
    Box bb, cb;
    for (uint32_t i = tk.begin; i < tk.end; ++i) {
      bb.grow(tb[idx[i]]);
      cb.grow(&cen[3 * (size_t)idx[i]]);
    }
    BvhNode& nd = out.nodes[tk.node];
    for (int i = 0; i < 3; ++i) {
      nd.lo[i] = bb.lo[i];
      nd.hi[i] = bb.hi[i];
    }
    auto make_leaf = [&]() {
      out.nodes[tk.node].ref = tk.begin;
      out.nodes[tk.node].count = n;
    };
    if (n == 1) {
      make_leaf();
      continue;
    }
    // choose the split
    int best_axis = -1, best_bin = -1;
    double best_cost = INFINITY;
    if (tk.depth < kMedianDepth) {
      for (int ax = 0; ax < 3; ++ax) {
        const float ext = cb.hi[ax] - cb.lo[ax];
        if (!(ext > 0.0f)) continue;
        Box bins[kBins];
        uint32_t cnt[kBins] = {0};
        const float scale = kBins / ext;
        for (uint32_t i = tk.begin; i < tk.end; ++i) {
          const uint32_t t = idx[i];
          int b = (int)((cen[3 * (size_t)t + ax] - cb.lo[ax]) * scale);
          b = std::min(std::max(b, 0), kBins - 1);
          bins[b].grow(tb[t]);
          ++cnt[b];
        }
        double rarea[kBins];
        uint32_t rcnt[kBins];
        Box acc;
        uint32_t c = 0;
        for (int b = kBins - 1; b > 0; --b) {
          acc.grow(bins[b]);
          c += cnt[b];
          rarea[b] = acc.area();
          rcnt[b] = c;
        }
        Box lacc;
        uint32_t lc = 0;
        for (int b = 0; b < kBins - 1; ++b) {
          lacc.grow(bins[b]);
          lc += cnt[b];
          if (lc == 0 || rcnt[b + 1] == 0) continue;
          const double cost = lacc.area() * lc + rarea[b + 1] * rcnt[b + 1];
          if (cost < best_cost) {
            best_cost = cost;
            best_axis = ax;
            best_bin = b;
          }
        }
      }
      // SAH leaf test (traversal and intersection cost taken as equal)
      const double parea = bb.area();
      if (n <= kMaxLeaf && (best_axis < 0 || parea * n <= parea + best_cost)) {
        make_leaf();
        continue;
      }
    } else if (n <= kMaxLeaf) {
      make_leaf();
      continue;
    }
    uint32_t mid;
    if (best_axis >= 0) {
      const int ax = best_axis;
      const float ext = cb.hi[ax] - cb.lo[ax];
      const float scale = kBins / ext;
      auto it = std::partition(idx.begin() + tk.begin, idx.begin() + tk.end, [&](uint32_t t) {
        int b = (int)((cen[3 * (size_t)t + ax] - cb.lo[ax]) * scale);
        b = std::min(std::max(b, 0), kBins - 1);
        return b <= best_bin;
      });
      mid = (uint32_t)(it - idx.begin());
    } else {
      mid = tk.begin;  // force the median fallback below
    }
    if (mid == tk.begin || mid == tk.end) {
      // median split by count along the widest centroid axis (or by index)
      int ax = 0;
      for (int i = 1; i < 3; ++i)
        if (cb.hi[i] - cb.lo[i] > cb.hi[ax] - cb.lo[ax]) ax = i;
      mid = tk.begin + n / 2;
      std::nth_element(idx.begin() + tk.begin, idx.begin() + mid, idx.begin() + tk.end, [&](uint32_t a, uint32_t b) {
        const float ca = cen[3 * (size_t)a + ax], cb2 = cen[3 * (size_t)b + ax];
        return ca < cb2 || (ca == cb2 && a < b);
      });
    }
    const uint32_t left = (uint32_t)out.nodes.size();
    out.nodes.push_back(BvhNode{});
    out.nodes.push_back(BvhNode{});
    out.nodes[tk.node].ref = left;
    out.nodes[tk.node].count = 0;
    // right first so the left subtree is laid out right after its parent
    stack.push_back({left + 1, mid, tk.end, tk.depth + 1});
    stack.push_back({left, tk.begin, mid, tk.depth + 1});
  }
  out.order = std::move(idx);
  out.max_depth = max_depth;
  return 0;
}

int collapse_bvh4(const BvhOut& b2, std::vector<Bvh4Node>& out, uint32_t* max_depth) {
  const std::vector<BvhNode>& nb = b2.nodes;
  auto area = [&](uint32_t i) {
    const BvhNode& b = nb[i];
    const double dx = b.hi[0] - b.lo[0], dy = b.hi[1] - b.lo[1], dz = b.hi[2] - b.lo[2];
    return 2.0 * (dx * dy + dy * dz + dz * dx);
  };
  out.clear();
  out.reserve(nb.size() / 2 + 1);
  struct Item {
    uint32_t b2node, slot, depth;
  };
  std::vector<Item> todo;
  out.push_back(Bvh4Node{});
  todo.push_back({1u, 0u, 1u});
  uint32_t md = 0;
  while (!todo.empty()) {
    const Item it = todo.back();
    todo.pop_back();
    md = std::max(md, it.depth);
    // children of this four-wide node, as binary node indices
    uint32_t ch[4];
    int n = 0;
    if (nb[it.b2node].count != 0) {
      ch[n++] = it.b2node;  // a root that is a leaf
    } else {
      ch[n++] = nb[it.b2node].ref;
      ch[n++] = nb[it.b2node].ref + 1;
      while (n < 4) {
        int best = -1;
        double ba = -1.0;
        for (int i = 0; i < n; ++i)
          if (nb[ch[i]].count == 0 && area(ch[i]) > ba) {
            ba = area(ch[i]);
            best = i;
          }
        if (best < 0) break;
        const uint32_t r = nb[ch[best]].ref;
        ch[best] = r;
        ch[n++] = r + 1;
      }
    }
    Bvh4Node nd{};
    for (int i = 0; i < 4; ++i) {
      if (i < n) {
        const BvhNode& b = nb[ch[i]];
        nd.lox[i] = b.lo[0];
        nd.loy[i] = b.lo[1];
        nd.loz[i] = b.lo[2];
        nd.hix[i] = b.hi[0];
        nd.hiy[i] = b.hi[1];
        nd.hiz[i] = b.hi[2];
        if (b.count != 0) {
          nd.ref[i] = b.ref;
          nd.cnt[i] = b.count;
        } else {
          const uint32_t slot = (uint32_t)out.size();
          out.push_back(Bvh4Node{});
          nd.ref[i] = slot;
          nd.cnt[i] = 0;
          todo.push_back({ch[i], slot, it.depth + 1});
        }
      } else {
        nd.lox[i] = nd.loy[i] = nd.loz[i] = INFINITY;
        nd.hix[i] = nd.hiy[i] = nd.hiz[i] = -INFINITY;
        nd.ref[i] = 0;
        nd.cnt[i] = kEmpty4;
      }
    }
    out[it.slot] = nd;
  }
  if (max_depth) *max_depth = md;
  return 0;
}

}  // namespace srt

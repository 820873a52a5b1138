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
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
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
// SAH: cost of a node visit relative to one triangle test, and the largest
// leaf (the node format holds counts up to 7)
#ifndef SRT_SAH_CT
#define SRT_SAH_CT 1.0
#endif
#ifndef SRT_MAX_LEAF
#define SRT_MAX_LEAF 4
#endif
constexpr double kCt = SRT_SAH_CT;
constexpr uint32_t kMaxLeaf = SRT_MAX_LEAF;
static_assert(kMaxLeaf >= 1 && kMaxLeaf <= 7, "leaf size");
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
      // SAH leaf test: n triangle tests against a visit and the children's tests
      const double parea = bb.area();
      if (n <= kMaxLeaf && (best_axis < 0 || parea * n <= kCt * parea + best_cost)) {
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

// ---------------------------------------------------------------------------
// Spatial-split BVH (Stich, Friedrich and Dietrich, "Spatial splits in
// bounding volume hierarchies", HPG 2009): besides the binned object split
// over reference centroids, every node whose object split leaves the two
// children overlapping by more than 1e-5 of the root's area also tries 32
// spatial split planes per axis, with each reference's share of a bin the box
// of its triangle clipped to the bin; a spatial split that wins divides the
// references that straddle its plane in two, each with the box of its side
// of the clipped triangle.  References of non-splittable triangles (those
// that must appear once in the tree) stay whole and follow their centroid.
// The duplicates stop once the references reach twice the triangle count
// (per subtree job, twice its own references).  Below the top of the tree the
// subtrees are built on all host threads, with the same result as one thread.
// ---------------------------------------------------------------------------

namespace {

struct Ref {
  uint32_t t;
  Box b;
};

// Box of triangle (v0, v1, v2) clipped to the slab lo <= x[ax] <= hi (either
// bound may be infinite) and to box `in`; empty if nothing is left.  The
// clipping runs in FP64 and the box is rounded outward to float.
Box clip_box(const double* v[3], int ax, double lo, double hi, const Box& in) {
  double poly[9][3], tmp[9][3];
  int n = 3;
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a) poly[k][a] = v[k][a];
  auto clip = [&](double plane, bool keep_above) {
    int m = 0;
    for (int i = 0; i < n; ++i) {
      const double* P = poly[i];
      const double* Q = poly[(i + 1) % n];
      const bool pin = keep_above ? P[ax] >= plane : P[ax] <= plane;
      const bool qin = keep_above ? Q[ax] >= plane : Q[ax] <= plane;
      if (pin) {
        for (int a = 0; a < 3; ++a) tmp[m][a] = P[a];
        ++m;
      }
      if (pin != qin) {
        const double s = (plane - P[ax]) / (Q[ax] - P[ax]);
        for (int a = 0; a < 3; ++a) tmp[m][a] = P[a] + s * (Q[a] - P[a]);
        tmp[m][ax] = plane;
        ++m;
      }
    }
    n = m;
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < 3; ++a) poly[i][a] = tmp[i][a];
  };
  if (std::isfinite(lo)) clip(lo, true);
  if (n > 0 && std::isfinite(hi)) clip(hi, false);
  Box out;
  if (n == 0) return out;
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      float lo_f = (float)poly[i][a], hi_f = lo_f;
      if ((double)lo_f > poly[i][a]) lo_f = std::nextafter(lo_f, -INFINITY);
      if ((double)hi_f < poly[i][a]) hi_f = std::nextafter(hi_f, INFINITY);
      out.lo[a] = std::min(out.lo[a], lo_f);
      out.hi[a] = std::max(out.hi[a], hi_f);
    }
  for (int a = 0; a < 3; ++a) {
    out.lo[a] = std::max(out.lo[a], in.lo[a]);
    out.hi[a] = std::min(out.hi[a], in.hi[a]);
    if (out.lo[a] > out.hi[a]) return Box{};
  }
  return out;
}

double overlap_area(const Box& a, const Box& b) {
  Box o;
  for (int i = 0; i < 3; ++i) {
    o.lo[i] = std::max(a.lo[i], b.lo[i]);
    o.hi[i] = std::min(a.hi[i], b.hi[i]);
    if (!(o.lo[i] <= o.hi[i])) return 0.0;
  }
  return o.area();
}

}  // namespace

int build_sbvh(const float* verts, const uint32_t* tris, uint32_t nt, const uint8_t* splittable, BvhOut& out,
               unsigned threads) {
  std::vector<double> vd(9 * (size_t)nt);
  std::vector<Ref> root(nt);
  Box world;
  for (uint32_t t = 0; t < nt; ++t) {
    root[t].t = t;
    for (int k = 0; k < 3; ++k) {
      const float* p = verts + 3 * (size_t)tris[3 * (size_t)t + k];
      root[t].b.grow(p);
      for (int a = 0; a < 3; ++a) vd[9 * (size_t)t + 3 * k + a] = p[a];
    }
    world.grow(root[t].b);
  }
  const double root_area = world.area();
  const size_t budget = 2 * (size_t)nt;  // references at most
  size_t n_refs = nt;
  out.nodes.assign(2, BvhNode{});
  out.order.clear();
  out.order.reserve(budget);
  struct STask {
    uint32_t node, depth;
    std::vector<Ref> refs;
  };
  std::vector<STask> stack;
  stack.push_back({1, 0, std::move(root)});
  uint32_t max_depth = 0;
  auto cen = [](const Ref& r, int a) { return 0.5f * (r.b.lo[a] + r.b.hi[a]); };
  // one node: its split (or leaf) into nodes / order, children onto stk
  auto step = [&](STask tk, std::vector<BvhNode>& nodes, std::vector<uint32_t>& order, std::vector<STask>& stk,
                  size_t& refs_count, size_t bud, uint32_t& maxd) {
    maxd = std::max(maxd, tk.depth);
    std::vector<Ref>& R = tk.refs;
    const uint32_t n = (uint32_t)R.size();
    Box bb, cb;
    for (const Ref& r : R) {
      bb.grow(r.b);
      const float c[3] = {cen(r, 0), cen(r, 1), cen(r, 2)};
      cb.grow(c);
    }
    BvhNode& nd = nodes[tk.node];
    for (int i = 0; i < 3; ++i) {
      nd.lo[i] = bb.lo[i];
      nd.hi[i] = bb.hi[i];
    }
    auto make_leaf = [&]() {
      nodes[tk.node].ref = (uint32_t)order.size();
      nodes[tk.node].count = n;
      for (const Ref& r : R) order.push_back(r.t);
    };
    if (n == 1) {
      make_leaf();
      return;
    }
    // object split
    int ob_axis = -1, ob_bin = -1;
    double ob_cost = INFINITY;
    Box ob_l, ob_r;
    // spatial split
    int sp_axis = -1, sp_bin = -1;
    double sp_cost = INFINITY;
    if (tk.depth < kMedianDepth) {
      for (int ax = 0; ax < 3; ++ax) {
        const float ext = cb.hi[ax] - cb.lo[ax];
        if (!(ext > 0.0f)) continue;
        Box bins[kBins];
        uint32_t cnt[kBins] = {0};
        const float scale = kBins / ext;
        for (const Ref& r : R) {
          int b = (int)((cen(r, ax) - cb.lo[ax]) * scale);
          b = std::min(std::max(b, 0), kBins - 1);
          bins[b].grow(r.b);
          ++cnt[b];
        }
        Box rbox[kBins];
        uint32_t rcnt[kBins];
        Box acc;
        uint32_t c = 0;
        for (int b = kBins - 1; b > 0; --b) {
          acc.grow(bins[b]);
          c += cnt[b];
          rbox[b] = acc;
          rcnt[b] = c;
        }
        Box lacc;
        uint32_t lc = 0;
        for (int b = 0; b < kBins - 1; ++b) {
          lacc.grow(bins[b]);
          lc += cnt[b];
          if (lc == 0 || rcnt[b + 1] == 0) continue;
          const double cost = lacc.area() * lc + rbox[b + 1].area() * rcnt[b + 1];
          if (cost < ob_cost) {
            ob_cost = cost;
            ob_axis = ax;
            ob_bin = b;
            ob_l = lacc;
            ob_r = rbox[b + 1];
          }
        }
      }
      const bool try_spatial = refs_count < bud && (ob_axis < 0 || overlap_area(ob_l, ob_r) > 1e-5 * root_area);
      if (try_spatial) {
        for (int ax = 0; ax < 3; ++ax) {
          const double lo = bb.lo[ax], ext = (double)bb.hi[ax] - lo;
          if (!(ext > 0.0)) continue;
          Box bins[kBins];
          uint32_t ent[kBins] = {0}, ext_[kBins] = {0};
          auto bin_of = [&](double x) {
            int b = (int)((x - lo) / ext * kBins);
            return std::min(std::max(b, 0), kBins - 1);
          };
          for (const Ref& r : R) {
            if (!splittable[r.t]) {
              const int b = bin_of(cen(r, ax));
              bins[b].grow(r.b);
              ++ent[b];
              ++ext_[b];
              continue;
            }
            const int b0 = bin_of(r.b.lo[ax]), b1 = bin_of(r.b.hi[ax]);
            if (b0 == b1) {
              bins[b0].grow(r.b);
            } else {
              const double* v[3] = {&vd[9 * (size_t)r.t], &vd[9 * (size_t)r.t + 3], &vd[9 * (size_t)r.t + 6]};
              for (int b = b0; b <= b1; ++b) {
                const double pl = lo + ext * b / kBins, ph = lo + ext * (b + 1) / kBins;
                const Box cbx = clip_box(v, ax, b == b0 ? -INFINITY : pl, b == b1 ? INFINITY : ph, r.b);
                bins[b].grow(cbx);
              }
            }
            ++ent[b0];
            ++ext_[b1];
          }
          double rarea[kBins];
          uint32_t rcnt[kBins];
          Box acc;
          uint32_t c = 0;
          for (int b = kBins - 1; b > 0; --b) {
            acc.grow(bins[b]);
            c += ext_[b];
            rarea[b] = acc.area();
            rcnt[b] = c;
          }
          Box lacc;
          uint32_t lc = 0;
          for (int b = 0; b < kBins - 1; ++b) {
            lacc.grow(bins[b]);
            lc += ent[b];
            if (lc == 0 || rcnt[b + 1] == 0) continue;
            const double cost = lacc.area() * lc + rarea[b + 1] * rcnt[b + 1];
            if (cost < sp_cost) {
              sp_cost = cost;
              sp_axis = ax;
              sp_bin = b;
            }
          }
        }
      }
      const double best = std::min(ob_cost, sp_cost);
      const double parea = bb.area();
      if (n <= kMaxLeaf && ((ob_axis < 0 && sp_axis < 0) || parea * n <= kCt * parea + best)) {
        make_leaf();
        return;
      }
    } else if (n <= kMaxLeaf) {
      make_leaf();
      return;
    }
    std::vector<Ref> L, Rt;
    L.reserve(n);
    Rt.reserve(n);
    if (sp_axis >= 0 && sp_cost < ob_cost) {
      const int ax = sp_axis;
      const double lo = bb.lo[ax], ext = (double)bb.hi[ax] - lo;
      const double plane = lo + ext * (sp_bin + 1) / kBins;
      for (const Ref& r : R) {
        if (!splittable[r.t]) {
          (cen(r, ax) < plane ? L : Rt).push_back(r);
        } else if (r.b.hi[ax] <= plane) {
          L.push_back(r);
        } else if (r.b.lo[ax] >= plane) {
          Rt.push_back(r);
        } else {
          const double* v[3] = {&vd[9 * (size_t)r.t], &vd[9 * (size_t)r.t + 3], &vd[9 * (size_t)r.t + 6]};
          const Box lb = clip_box(v, ax, -INFINITY, plane, r.b), rb = clip_box(v, ax, plane, INFINITY, r.b);
          const bool lok = lb.lo[0] <= lb.hi[0], rok = rb.lo[0] <= rb.hi[0];
          if (lok) L.push_back({r.t, lb});
          if (rok) Rt.push_back({r.t, rb});
          if (!lok && !rok) L.push_back(r);
          if (lok && rok) ++refs_count;
        }
      }
    } else if (ob_axis >= 0) {
      const int ax = ob_axis;
      const float ext = cb.hi[ax] - cb.lo[ax];
      const float scale = kBins / ext;
      for (const Ref& r : R) {
        int b = (int)((cen(r, ax) - cb.lo[ax]) * scale);
        b = std::min(std::max(b, 0), kBins - 1);
        (b <= ob_bin ? L : Rt).push_back(r);
      }
    }
    if (L.empty() || Rt.empty()) {
      // median split by count along the widest centroid axis (or by order)
      L.clear();
      Rt.clear();
      int ax = 0;
      for (int i = 1; i < 3; ++i)
        if (cb.hi[i] - cb.lo[i] > cb.hi[ax] - cb.lo[ax]) ax = i;
      std::vector<Ref> S = R;
      const uint32_t mid = n / 2;
      std::nth_element(S.begin(), S.begin() + mid, S.end(), [&](const Ref& a, const Ref& b) {
        const float ca = cen(a, ax), cb2 = cen(b, ax);
        return ca < cb2 || (ca == cb2 && a.t < b.t);
      });
      L.assign(S.begin(), S.begin() + mid);
      Rt.assign(S.begin() + mid, S.end());
    }
    R.clear();
    R.shrink_to_fit();
    const uint32_t left = (uint32_t)nodes.size();
    nodes.push_back(BvhNode{});
    nodes.push_back(BvhNode{});
    nodes[tk.node].ref = left;
    nodes[tk.node].count = 0;
    stk.push_back({left + 1, tk.depth + 1, std::move(Rt)});
    stk.push_back({left, tk.depth + 1, std::move(L)});
  };
  // the top of the tree on this thread; subtrees of at most kParRefs
  // references become independent jobs, built in parallel into their own
  // node and order arrays (root at local node 0, child pairs from node 2)
  // and stitched back in job order, so the tree does not depend on the
  // thread count
  const size_t kParRefs = std::max<size_t>(4096, nt / 256);
  std::vector<STask> jobs;
  while (!stack.empty()) {
    STask tk = std::move(stack.back());
    stack.pop_back();
    if (tk.depth > 0 && tk.refs.size() <= kParRefs) {
      jobs.push_back(std::move(tk));
      continue;
    }
    step(std::move(tk), out.nodes, out.order, stack, n_refs, budget, max_depth);
  }
  struct Local {
    std::vector<BvhNode> nodes;
    std::vector<uint32_t> order;
    uint32_t maxd = 0;
  };
  std::vector<Local> loc(jobs.size());
  std::atomic<size_t> next{0};
  auto worker = [&]() {
    for (;;) {
      const size_t j = next.fetch_add(1);
      if (j >= jobs.size()) break;
      Local& L = loc[j];
      L.nodes.assign(2, BvhNode{});
      std::vector<STask> stk;
      const size_t nref = jobs[j].refs.size();
      size_t cnt = nref;
      STask root_task{0, jobs[j].depth, std::move(jobs[j].refs)};
      stk.push_back(std::move(root_task));
      while (!stk.empty()) {
        STask tk = std::move(stk.back());
        stk.pop_back();
        step(std::move(tk), L.nodes, L.order, stk, cnt, 2 * nref, L.maxd);
      }
    }
  };
  const unsigned nth =
      threads ? threads : std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 64u));
  std::vector<std::thread> th;
  for (unsigned q = 0; q + 1 < nth && q + 1 < jobs.size(); ++q) th.emplace_back(worker);
  worker();
  for (auto& q : th) q.join();
  for (size_t j = 0; j < jobs.size(); ++j) {
    const Local& L = loc[j];
    const uint32_t base = (uint32_t)out.nodes.size();
    const uint32_t obase = (uint32_t)out.order.size();
    auto remap = [&](BvhNode b) {
      if (b.count) b.ref += obase;
      else b.ref = base + (b.ref - 2);
      return b;
    };
    out.nodes[jobs[j].node] = remap(L.nodes[0]);
    for (size_t i = 2; i < L.nodes.size(); ++i) out.nodes.push_back(remap(L.nodes[i]));
    out.order.insert(out.order.end(), L.order.begin(), L.order.end());
    max_depth = std::max(max_depth, L.maxd);
  }
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

int collapse_bvh8(const BvhOut& b2, std::vector<Bvh8Node>& out, uint32_t* max_depth) {
  const std::vector<BvhNode>& nb = b2.nodes;
  auto area = [&](uint32_t i) {
    const BvhNode& b = nb[i];
    const double dx = b.hi[0] - b.lo[0], dy = b.hi[1] - b.lo[1], dz = b.hi[2] - b.lo[2];
    return 2.0 * (dx * dy + dy * dz + dz * dx);
  };
  out.clear();
  out.reserve(nb.size() / 4 + 1);
  struct Item {
    uint32_t b2node, slot, depth;
  };
  std::vector<Item> todo;
  out.push_back(Bvh8Node{});
  todo.push_back({1u, 0u, 1u});
  uint32_t md = 0;
  while (!todo.empty()) {
    const Item it = todo.back();
    todo.pop_back();
    md = std::max(md, it.depth);
    uint32_t ch[8];
    int n = 0;
    if (nb[it.b2node].count != 0) {
      ch[n++] = it.b2node;  // a root that is a leaf
    } else {
      ch[n++] = nb[it.b2node].ref;
      ch[n++] = nb[it.b2node].ref + 1;
      while (n < 8) {
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
    // corner slots
    double plo[3] = {INFINITY, INFINITY, INFINITY}, phi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < 3; ++a) {
        plo[a] = std::min(plo[a], (double)nb[ch[i]].lo[a]);
        phi[a] = std::max(phi[a], (double)nb[ch[i]].hi[a]);
      }
    double score[8][8];
    for (int i = 0; i < n; ++i)
      for (int sl = 0; sl < 8; ++sl) {
        double sc = 0.0;
        for (int a = 0; a < 3; ++a) {
          const double ext = phi[a] - plo[a];
          const double d = ext > 0.0 ? ((double)nb[ch[i]].lo[a] + nb[ch[i]].hi[a] - plo[a] - phi[a]) / ext : 0.0;
          sc += ((sl >> a) & 1) ? d : -d;
        }
        score[i][sl] = sc;
      }
    int slot_of[8];
    bool used_c[8] = {false}, used_s[8] = {false};
    for (int k = 0; k < n; ++k) {
      int bi = -1, bs = -1;
      double bv = -INFINITY;
      for (int i = 0; i < n; ++i)
        if (!used_c[i])
          for (int sl = 0; sl < 8; ++sl)
            if (!used_s[sl] && score[i][sl] > bv) {
              bv = score[i][sl];
              bi = i;
              bs = sl;
            }
      used_c[bi] = used_s[bs] = true;
      slot_of[bi] = bs;
    }
    Bvh8Node nd{};
    for (int sl = 0; sl < 8; ++sl) {
      nd.lox[sl] = nd.loy[sl] = nd.loz[sl] = INFINITY;
      nd.hix[sl] = nd.hiy[sl] = nd.hiz[sl] = -INFINITY;
      nd.ref[sl] = 0;
      nd.cnt[sl] = kEmpty4;
    }
    for (int i = 0; i < n; ++i) {
      const int sl = slot_of[i];
      const BvhNode& b = nb[ch[i]];
      nd.lox[sl] = b.lo[0];
      nd.loy[sl] = b.lo[1];
      nd.loz[sl] = b.lo[2];
      nd.hix[sl] = b.hi[0];
      nd.hiy[sl] = b.hi[1];
      nd.hiz[sl] = b.hi[2];
      if (b.count != 0) {
        nd.ref[sl] = b.ref;
        nd.cnt[sl] = b.count;
      } else {
        const uint32_t slot = (uint32_t)out.size();
        out.push_back(Bvh8Node{});
        nd.ref[sl] = slot;
        nd.cnt[sl] = 0;
        todo.push_back({ch[i], slot, it.depth + 1});
      }
    }
    out[it.slot] = nd;
  }
  if (max_depth) *max_depth = md;
  return 0;
}

}  // namespace srt

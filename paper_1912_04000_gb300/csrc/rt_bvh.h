// Host BVH builder interface.
#pragma once

#include <cstdint>
#include <vector>

namespace srt {

struct BvhNode {
  float lo[3] = {0, 0, 0};
  uint32_t ref = 0;
  float hi[3] = {0, 0, 0};
  uint32_t count = 0;
};
static_assert(sizeof(BvhNode) == 32, "32-byte node");

struct BvhOut {
  std::vector<BvhNode> nodes;   // [0] unused, [1] root
  std::vector<uint32_t> order;  // leaf-order position -> input triangle id
  uint32_t max_depth = 0;
};

// Builds the BVH of nt triangles (indices into verts[.][3]).  Returns 0.
int build_bvh(const float* verts, const uint32_t* tris, uint32_t nt, BvhOut& out);

// Builds a spatial-split BVH: order may list a triangle in several leaves
// (at most 2 nt references), never one whose splittable[t] is 0.  threads:
// host threads to use (0 = all); the tree does not depend on it.  Returns 0.
int build_sbvh(const float* verts, const uint32_t* tris, uint32_t nt, const uint8_t* splittable, BvhOut& out,
               unsigned threads = 0);

// Four-wide node: child boxes in structure-of-arrays order (one float4 per
// plane), child i an interior node (cnt[i] = 0, ref[i] = node index), a leaf
// (cnt[i] = 1..4 triangles from leaf position ref[i]) or empty (cnt[i] =
// kEmpty4, box lo = +inf, hi = -inf, which no slab test enters).  The upload
// packs ref[i] as ref << 3 | count for the device and zeroes cnt.
constexpr uint32_t kEmpty4 = 0xFFFFFFFFu;
struct Bvh4Node {
  float lox[4], hix[4], loy[4], hiy[4], loz[4], hiz[4];
  uint32_t ref[4], cnt[4];
};
static_assert(sizeof(Bvh4Node) == 128, "128-byte node");

// Collapses the binary BVH into a four-wide one (node 0 the root): every
// interior node takes the children of its binary node and repeatedly replaces
// the interior child of largest surface area by its two children until it
// has four.  Leaves and the leaf order are those of the binary tree.
int collapse_bvh4(const BvhOut& b2, std::vector<Bvh4Node>& out, uint32_t* max_depth);

// Eight-wide node: the same child encoding as the four-wide node, the
// planes of each axis as lo of the eight children then hi of the eight.
// Slot s holds the child that lies towards the corner ((s & 1) ? +x : -x,
// (s & 2) ? +y : -y, (s & 4) ? +z : -z) of the node, so that a ray that
// visits slots in the order i ^ octant meets the near corner first.
struct Bvh8Node {
  float lox[8], hix[8], loy[8], hiy[8], loz[8], hiz[8];
  uint32_t ref[8], cnt[8];
};
static_assert(sizeof(Bvh8Node) == 256, "256-byte host node");

// Collapses the binary BVH into an eight-wide one (node 0 the root) by the
// greedy rule of collapse_bvh4 with up to eight children, then places the
// children in the corner slots: repeatedly the free (child, slot) pair whose
// child centre, relative to the node centre and scaled by the node's extent
// per axis, points furthest towards the slot's corner.
int collapse_bvh8(const BvhOut& b2, std::vector<Bvh8Node>& out, uint32_t* max_depth);

}  // namespace srt

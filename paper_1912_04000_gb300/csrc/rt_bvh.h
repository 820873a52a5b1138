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

}  // namespace srt

// Device BVH builder: linear BVH of Karras ("Maximizing parallelism in the
// construction of BVHs, octrees, and k-d trees", HPG 2012) over 30-bit
// Morton codes of the triangle centroids, bottom-up boxes, and a top-down
// collapse to the four-wide layout the traversal reads.
//
//   1. per triangle: box, centroid Morton code (10 bits per axis over the
//      scene box), value = triangle index;
//   2. stable LSD radix sort of (code, index), four 8-bit passes: per-block
//      digit counts, one exclusive scan over (digit, block), a stable scatter
//      that ranks equal digits inside a warp with match_any and across the
//      warps of a block through shared counters;
//   3. Karras hierarchy: internal node i covers a key range found by
//      exponential and binary search on the common-prefix length (ties of
//      equal codes broken by the index), split where that length first drops;
//   4. boxes bottom-up: a leaf climbs to its parent, the second child to
//      arrive (atomic counter) forms the union and climbs on;
//   5. collapse, one launch per level: a four-wide node takes its binary
//      node's children and repeatedly replaces the interior child of largest
//      surface area by its two children (the host collapse's rule); interior
//      children get new node slots on the next level's queue;
//   6. triangle and normal records gathered into leaf (sorted) order.
// A subtree of at most 4 triangles becomes one leaf.  Boxes are padded outward by `pad` with directed
// rounding, the same margin the host builder applies, so the traversal's FMA
// slab test stays conservative.  No kernel waits on another thread.
#include <cstdint>

#include "rt_internal.h"

namespace srt {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr uint32_t kSortTile = kSortThreads * kSortRounds;  // keys per block
constexpr int kMaxLevels = 64;

// 10 bits of v to bit positions 0, 3, 6, ..., 27.
__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v = (v * 0x00010001u) & 0xFF0000FFu;
  v = (v * 0x00000101u) & 0x0F00F00Fu;
  v = (v * 0x00000011u) & 0xC30C30C3u;
  v = (v * 0x00000005u) & 0x49249249u;
  return v;
}

__global__ void k_lbvh_keys(const float* __restrict__ verts, const uint32_t* __restrict__ tri, uint32_t n,
                            float3 lo, float3 inv_ext, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                            float4* __restrict__ tbox) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    float3 a = make_float3(INFINITY, INFINITY, INFINITY), b = make_float3(-INFINITY, -INFINITY, -INFINITY);
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      const float* p = verts + 3 * (size_t)tri[3 * (size_t)t + v];
      a = make_float3(fminf(a.x, p[0]), fminf(a.y, p[1]), fminf(a.z, p[2]));
      b = make_float3(fmaxf(b.x, p[0]), fmaxf(b.y, p[1]), fmaxf(b.z, p[2]));
    }
    tbox[2 * t] = make_float4(a.x, a.y, a.z, 0.0f);
    tbox[2 * t + 1] = make_float4(b.x, b.y, b.z, 0.0f);
    const float cx = fminf(fmaxf((0.5f * (a.x + b.x) - lo.x) * inv_ext.x, 0.0f), 1.0f);
    const float cy = fminf(fmaxf((0.5f * (a.y + b.y) - lo.y) * inv_ext.y, 0.0f), 1.0f);
    const float cz = fminf(fmaxf((0.5f * (a.z + b.z) - lo.z) * inv_ext.z, 0.0f), 1.0f);
    const uint32_t x = min((uint32_t)(cx * 1024.0f), 1023u), y = min((uint32_t)(cy * 1024.0f), 1023u),
                   z = min((uint32_t)(cz * 1024.0f), 1023u);
    keys[t] = (spread10(x) << 2) | (spread10(y) << 1) | spread10(z);
    vals[t] = t;
  }
}

// Digit counts of one block's tile, digit-major: hist[d * nblocks + block].
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys, uint32_t n,
                                                             uint32_t shift, uint32_t* __restrict__ hist,
                                                             uint32_t nblocks) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0u;
  __syncthreads();
  const uint32_t base = blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    const uint32_t i = base + (uint32_t)r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: element i goes to offset(digit, block) + (elements of the
// same digit before it in the block's tile).  Rounds take 256 consecutive
// keys, one per thread in index order; inside a warp equal digits are ranked
// with match_any, across the block's warps through warp_cnt.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t* __restrict__ kin,
                                                                const uint32_t* __restrict__ vin, uint32_t n,
                                                                uint32_t shift, const uint32_t* __restrict__ hist,
                                                                const uint32_t* __restrict__ totals,
                                                                uint32_t nblocks, uint32_t* __restrict__ kout,
                                                                uint32_t* __restrict__ vout) {
  __shared__ uint32_t base_off[256];
  __shared__ uint32_t warp_cnt[kSortThreads / 32][256];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  {
    const uint32_t e = tid * nblocks + blockIdx.x;
    base_off[tid] = hist[e] + totals[e >> 10];
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) warp_cnt[w][tid] = 0u;
  }
  __syncthreads();
  const uint32_t base = blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    const uint32_t i = base + (uint32_t)r * kSortThreads + tid;
    const bool valid = i < n;
    const uint32_t key = valid ? kin[i] : 0u;
    const uint32_t val = valid ? vin[i] : 0u;
    const uint32_t d = (key >> shift) & 255u;
    const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 256u + lane);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0u) warp_cnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t pos = base_off[d] + rank;
      for (uint32_t w = 0; w < warp; ++w) pos += warp_cnt[w][d];
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    uint32_t add = 0u;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) {
      add += warp_cnt[w][tid];
      warp_cnt[w][tid] = 0u;
    }
    base_off[tid] += add;
    __syncthreads();
  }
}

// Common-prefix length of sorted keys i and j (-1 outside [0, n)); equal keys
// are told apart by their indices.
__device__ __forceinline__ int delta(const uint32_t* __restrict__ k, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  const uint32_t a = k[i], b = k[j];
  return a != b ? __clz(a ^ b) : 32 + __clz((uint32_t)i ^ (uint32_t)j);
}

// Internal node i of n - 1: children in the combined index space (internal
// nodes 0 .. n-2, leaf of sorted position p at n - 1 + p); parent links.
__global__ void k_lbvh_hierarchy(const uint32_t* __restrict__ k, int n, int2* __restrict__ child,
                                 int2* __restrict__ range, int* __restrict__ parent) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n - 1; i += gridDim.x * blockDim.x) {
    const int d = delta(k, n, i, i + 1) - delta(k, n, i, i - 1) > 0 ? 1 : -1;
    const int dmin = delta(k, n, i, i - d);
    int lmax = 2;
    while (lmax < 2 * n && delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
      if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta(k, n, i, j);
    int s = 0, step = l;
    do {
      step = (step + 1) >> 1;
      if (delta(k, n, i, i + (s + step) * d) > dnode) s += step;
    } while (step > 1);
    const int g = i + s * d + min(d, 0);
    const int left = min(i, j) == g ? n - 1 + g : g;
    const int right = max(i, j) == g + 1 ? n - 1 + g + 1 : g + 1;
    child[i] = make_int2(left, right);
    range[i] = make_int2(min(i, j), max(i, j));
    parent[left] = i;
    parent[right] = i;
  }
}

// Boxes bottom-up.  box[node] = {lo, hi} for every node of the combined
// space; flag[internal] counts the children done.
__global__ void k_lbvh_boxes(const uint32_t* __restrict__ vals, const float4* __restrict__ tbox, int n,
                             const int2* __restrict__ child, const int* __restrict__ parent, float4* box,
                             uint32_t* flag) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint32_t t = vals[p];
    int node = n - 1 + p;
    box[2 * node] = tbox[2 * t];
    box[2 * node + 1] = tbox[2 * t + 1];
    __threadfence();
    node = parent[node];
    // each climb step moves one level up: at most n - 1 steps
    for (int steps = 0; node >= 0 && steps < n; ++steps) {
      if (atomicAdd(flag + node, 1u) == 0u) break;  // the sibling is not done yet
      const int2 c = child[node];
      const float4 al = __ldcg(box + 2 * c.x), ah = __ldcg(box + 2 * c.x + 1);
      const float4 bl = __ldcg(box + 2 * c.y), bh = __ldcg(box + 2 * c.y + 1);
      box[2 * node] = make_float4(fminf(al.x, bl.x), fminf(al.y, bl.y), fminf(al.z, bl.z), 0.0f);
      box[2 * node + 1] = make_float4(fmaxf(ah.x, bh.x), fmaxf(ah.y, bh.y), fmaxf(ah.z, bh.z), 0.0f);
      __threadfence();
      node = parent[node];
    }
  }
}

__device__ __forceinline__ float box_area(const float4* box, int node) {
  const float4 l = __ldcg(box + 2 * node), h = __ldcg(box + 2 * node + 1);
  const float dx = h.x - l.x, dy = h.y - l.y, dz = h.z - l.z;
  return 2.0f * (dx * dy + dy * dz + dz * dx);
}

// One level of the collapse.  qin[e] = {binary node, four-wide slot};
// counts: [0] four-wide nodes allocated, [1 + L] entries of level L's queue.
// An interior node whose key range holds at most kLbvhLeaf triangles becomes
// one leaf (its triangles are consecutive in the sorted order).
constexpr int kLbvhLeaf = 4;

__device__ __forceinline__ bool small_subtree(const int2* __restrict__ range, int n, int node) {
  if (node >= n - 1) return true;
  const int2 r = range[node];
  return r.y - r.x + 1 <= kLbvhLeaf;
}

__global__ void k_lbvh_collapse(int n, const int2* __restrict__ child, const int2* __restrict__ range,
                                const float4* __restrict__ box, float pad, const int2* __restrict__ qin,
                                int2* __restrict__ qout, uint32_t* counts, int level, float4* __restrict__ nodes4) {
  const uint32_t m = counts[1 + level];
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
    const int2 item = qin[e];
    int ch[4];
    int nc = 0;
    if (small_subtree(range, n, item.x)) {
      ch[nc++] = item.x;  // the whole tree is one leaf
    } else {
      ch[nc++] = child[item.x].x;
      ch[nc++] = child[item.x].y;
      while (nc < 4) {
        int best = -1;
        float ba = -1.0f;
        for (int c = 0; c < nc; ++c)
          if (!small_subtree(range, n, ch[c])) {
            const float a = box_area(box, ch[c]);
            if (a > ba) {
              ba = a;
              best = c;
            }
          }
        if (best < 0) break;
        const int2 cc = child[ch[best]];
        ch[best] = cc.x;
        ch[nc++] = cc.y;
      }
    }
    float lo[3][4], hi[3][4];
    uint32_t pk[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (c < nc) {
        const float4 l = __ldcg(box + 2 * ch[c]), h = __ldcg(box + 2 * ch[c] + 1);
        lo[0][c] = __fsub_rd(l.x, pad);
        lo[1][c] = __fsub_rd(l.y, pad);
        lo[2][c] = __fsub_rd(l.z, pad);
        hi[0][c] = __fadd_ru(h.x, pad);
        hi[1][c] = __fadd_ru(h.y, pad);
        hi[2][c] = __fadd_ru(h.z, pad);
        if (ch[c] >= n - 1) {
          pk[c] = ((uint32_t)(ch[c] - (n - 1)) << 3) | 1u;
        } else if (small_subtree(range, n, ch[c])) {
          const int2 r = range[ch[c]];
          pk[c] = ((uint32_t)r.x << 3) | (uint32_t)(r.y - r.x + 1);
        } else {
          const uint32_t slot = atomicAdd(counts, 1u);
          pk[c] = slot << 3;
          qout[atomicAdd(counts + 2 + level, 1u)] = make_int2(ch[c], (int)slot);
        }
      } else {
        lo[0][c] = lo[1][c] = lo[2][c] = INFINITY;
        hi[0][c] = hi[1][c] = hi[2][c] = -INFINITY;
        pk[c] = 0u;
      }
    }
    float4* o = nodes4 + 8 * (size_t)item.y;
    o[0] = make_float4(lo[0][0], lo[0][1], lo[0][2], lo[0][3]);
    o[1] = make_float4(hi[0][0], hi[0][1], hi[0][2], hi[0][3]);
    o[2] = make_float4(lo[1][0], lo[1][1], lo[1][2], lo[1][3]);
    o[3] = make_float4(hi[1][0], hi[1][1], hi[1][2], hi[1][3]);
    o[4] = make_float4(lo[2][0], lo[2][1], lo[2][2], lo[2][3]);
    o[5] = make_float4(hi[2][0], hi[2][1], hi[2][2], hi[2][3]);
    o[6] = make_float4(__uint_as_float(pk[0]), __uint_as_float(pk[1]), __uint_as_float(pk[2]),
                       __uint_as_float(pk[3]));
    o[7] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
}

__global__ void k_lbvh_gather(const uint32_t* __restrict__ vals, uint32_t n, const float4* __restrict__ tri_in,
                              const float4* __restrict__ nrm_in, float4* __restrict__ tri_out,
                              float4* __restrict__ nrm_out) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint32_t t = vals[p];
    tri_out[3 * (size_t)p] = tri_in[3 * (size_t)t];
    tri_out[3 * (size_t)p + 1] = tri_in[3 * (size_t)t + 1];
    tri_out[3 * (size_t)p + 2] = tri_in[3 * (size_t)t + 2];
    nrm_out[p] = nrm_in[t];
  }
}

// The root item: combined index 0 is internal node 0, or for one triangle
// the single leaf (n - 1 = 0); four-wide slot 0.
__global__ void k_lbvh_init(int2* q0, uint32_t* counts, int* parent) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    counts[0] = 1u;  // four-wide nodes allocated: the root
    counts[1] = 1u;  // level 0's queue: the root
    q0[0] = make_int2(0, 0);
    parent[0] = -1;
  }
}

}  // namespace

size_t radix_sort_hist_words(uint32_t n) {
  const size_t nb = (n + kSortTile - 1) / kSortTile;
  const size_t hist = (256 * nb + 32767) / 32768 * 32768;
  return hist + hist / 1024;
}

int launch_radix_sort(uint32_t* keys[2], uint32_t* vals[2], uint32_t n, uint32_t key_bits, uint32_t* hist,
                      cudaStream_t st) {
  const uint32_t nb = (n + kSortTile - 1) / kSortTile;
  const size_t hist_n = ((size_t)256 * nb + 32767) / 32768 * 32768;
  int cur = 0;
  for (uint32_t shift = 0; shift < key_bits; shift += 8) {
    cudaMemsetAsync(hist, 0, 4 * hist_n, st);
    k_radix_hist<<<nb, kSortThreads, 0, st>>>(keys[cur], n, shift, hist, nb);
    launch_scan(hist, hist_n, st);
    k_radix_scatter<<<nb, kSortThreads, 0, st>>>(keys[cur], vals[cur], n, shift, hist, hist + hist_n, nb,
                                                keys[cur ^ 1], vals[cur ^ 1]);
    cur ^= 1;
  }
  return cur;
}

size_t lbvh_scratch_bytes(uint32_t n) {
  const size_t nb = (n + kSortTile - 1) / kSortTile;
  const size_t hist = (256 * nb + 32767) / 32768 * 32768;
  return 4 * (size_t)n * 4                   // keys, vals (two copies)
         + (size_t)n * 32                    // triangle boxes
         + (size_t)n * 16                    // children, key ranges
         + (2 * (size_t)n) * 4               // parents
         + (2 * (size_t)n) * 32              // node boxes
         + (size_t)n * 4                     // arrival counters
         + 2 * (size_t)n * 8                 // collapse queues
         + (hist + hist / 1024) * 4          // radix histogram and chunk offsets
         + (2 + kMaxLevels) * 4 + 4096;      // counters, alignment slack
}

// Builds on stream st (n <= kLbvhMaxTris).  verts [nv][3], tri [n][3]
// (device); tri_in / nrm_in the records in input order; outputs: nodes4
// (capacity max(n - 1, 1) nodes), tri_out, nrm_out in leaf order;
// *counts_out (device) = {four-wide nodes allocated, then the queue size of
// each collapse level}: a non-zero last entry means the tree was deeper than
// the levels launched.
void launch_lbvh(const float* verts, const uint32_t* tri, uint32_t n, const float lo[3], const float hi[3], float pad,
                 const float4* tri_in, const float4* nrm_in, void* scratch, float4* nodes4, float4* tri_out,
                 float4* nrm_out, uint32_t** counts_out, int sms, cudaStream_t st) {
  const uint32_t nb = (n + kSortTile - 1) / kSortTile;
  const size_t hist_n = ((size_t)256 * nb + 32767) / 32768 * 32768;
  unsigned char* p = (unsigned char*)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
  auto take = [&](size_t bytes) {
    void* r = p;
    p += (bytes + 255) & ~(size_t)255;
    return r;
  };
  uint32_t* keys[2] = {(uint32_t*)take(4 * (size_t)n), (uint32_t*)take(4 * (size_t)n)};
  uint32_t* vals[2] = {(uint32_t*)take(4 * (size_t)n), (uint32_t*)take(4 * (size_t)n)};
  float4* tbox = (float4*)take(32 * (size_t)n);
  int2* child = (int2*)take(8 * (size_t)n);
  int2* range = (int2*)take(8 * (size_t)n);
  int* parent = (int*)take(8 * (size_t)n);
  float4* box = (float4*)take(64 * (size_t)n);
  uint32_t* flag = (uint32_t*)take(4 * (size_t)n);
  int2* q[2] = {(int2*)take(8 * (size_t)n), (int2*)take(8 * (size_t)n)};
  uint32_t* hist = (uint32_t*)take(4 * (hist_n + hist_n / 1024));
  uint32_t* counts = (uint32_t*)take(4 * (2 + kMaxLevels));
  *counts_out = counts;
  const int g = (sms > 0 ? sms : 1) * 8;
  float3 lo3 = make_float3(lo[0], lo[1], lo[2]);
  float3 inv = make_float3(hi[0] > lo[0] ? 1.0f / (hi[0] - lo[0]) : 0.0f, hi[1] > lo[1] ? 1.0f / (hi[1] - lo[1]) : 0.0f,
                           hi[2] > lo[2] ? 1.0f / (hi[2] - lo[2]) : 0.0f);
  k_lbvh_keys<<<g, 256, 0, st>>>(verts, tri, n, lo3, inv, keys[0], vals[0], tbox);
  // radix sort, 4 x 8 bits
  int cur = 0;
  for (uint32_t shift = 0; shift < 32; shift += 8) {
    cudaMemsetAsync(hist, 0, 4 * hist_n, st);
    k_radix_hist<<<nb, kSortThreads, 0, st>>>(keys[cur], n, shift, hist, nb);
    launch_scan(hist, hist_n, st);
    k_radix_scatter<<<nb, kSortThreads, 0, st>>>(keys[cur], vals[cur], n, shift, hist, hist + hist_n, nb,
                                                keys[cur ^ 1], vals[cur ^ 1]);
    cur ^= 1;
  }
  const uint32_t* sk = keys[cur];
  const uint32_t* sv = vals[cur];
  cudaMemsetAsync(flag, 0, 4 * (size_t)n, st);
  cudaMemsetAsync(counts, 0, 4 * (2 + kMaxLevels), st);
  k_lbvh_init<<<1, 32, 0, st>>>(q[0], counts, parent);
  if (n > 1) k_lbvh_hierarchy<<<g, 256, 0, st>>>(sk, (int)n, child, range, parent);
  k_lbvh_boxes<<<g, 256, 0, st>>>(sv, tbox, (int)n, child, parent, box, flag);
  for (int L = 0; L < kMaxLevels - 1; ++L)
    k_lbvh_collapse<<<g, 128, 0, st>>>((int)n, child, range, box, pad, q[L & 1], q[(L + 1) & 1], counts, L, nodes4);
  k_lbvh_gather<<<g, 256, 0, st>>>(sv, n, tri_in, nrm_in, tri_out, nrm_out);
}

}  // namespace srt

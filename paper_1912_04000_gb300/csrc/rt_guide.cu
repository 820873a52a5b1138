// Learned path guide on the GB300: hash-grid + SH encoding, a fused
// 64-64-64-64-48 MLP on tcgen05 tensor cores (BF16 operands, FP32
// accumulators in tensor memory), an 8-lobe von Mises-Fisher mixture head,
// and online training (forward, loss gradient, backward, Adam) by the same
// kernels.
//
// Definition (shared with the CPU oracle, written there in FP64):
//   X (64)  = [hash-grid features of the position (8 levels x 4, trilinear;
//              after Mueller et al. 2022, primes 1, 2654435761, 805459861),
//              real SH of the normal up to degree 3 (16), one-hot band group
//              (9), zeros (7)]
//   H1 = relu(X W1), H2 = relu(H1 W2), H3 = relu(H2 W3), Y = H3 W4 (48)
//   lobe j: pi = softmax(Y[5j]), mu = Y[5j+1..3] / |.|,
//           kappa = 0.5 + softplus(Y[5j+4])
//   q(w) = sum_j pi_j kappa_j / (2 pi (1 - e^{-2 kappa_j})) e^{kappa_j (mu_j.w - 1)}
//   loss = -(1/N) sum_r (w_r / mean w) log q_r(omega_r)
//
// Tensor-core layout: a tile is 128 records (M = 128 = TMEM lanes).  Every
// GEMM operand sits in shared memory in the K-major canonical layout
// (rt_tc.cuh).  Forward B operands are W^T (N = out rows, K = in); backward
// data-gradient B operands are W (N = in rows, K = out).  Weight gradients
// dW = H^T dZ use A' = [H^T; 0] (128 rows, the upper 64 the input features,
// K = the tile's 128 records) and B' = dZ^T, accumulated in TMEM across all
// tiles of a CTA and summed over the CTAs by k_dw_reduce at the end.
#include <cmath>
#include <cstdint>

#include "rt_device.cuh"
#include "rt_internal.h"
#include "rt_tc.cuh"

namespace srt {

namespace {

constexpr int kIn = 64, kHid = 64, kOut = 48, kLevels = kGuideLevels, kFeat = kGuideFeatures, kLobes = 8;
static_assert(kLevels * kFeat == 32, "32 grid features in the network input");
constexpr int kRows = 128;
constexpr uint32_t kATileB = 16384;   // [128 x 64] BF16 activations
constexpr uint32_t kSliceA = 4096;    // one 128 x 16 K-slice
constexpr uint32_t kWPack = 61440;    // bytes of packed BF16 weights
constexpr int kWSize = 15360;
// byte offsets of layer l's forward (W^T) and backward (W) BF16 tiles in the
// packed weights, and element offset of its FP32 master weights
__host__ __device__ constexpr uint32_t wf_off(int l) { return 8192u * (uint32_t)l; }
__host__ __device__ constexpr uint32_t wb_off(int l) { return 30720u + 8192u * (uint32_t)l; }
__host__ __device__ constexpr int w_off(int l) { return 4096 * l; }

__device__ __forceinline__ int layer_out(int l) { return l == 3 ? kOut : kHid; }

// ---------------------------------------------------------------------------
// encoding
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sh16(float x, float y, float z, float* o) {
  const float pi = 3.14159265358979323846f;
  const float rp = 1.0f / sqrtf(pi);
  const float c0 = 0.5f * rp, c1 = sqrtf(3.0f) * 0.5f * rp, c2 = sqrtf(15.0f) * 0.5f * rp;
  const float c3 = sqrtf(5.0f) * 0.25f * rp, c4 = sqrtf(15.0f) * 0.25f * rp;
  const float c5 = sqrtf(35.0f / (2.0f * pi)) * 0.25f, c6 = sqrtf(105.0f) * 0.5f * rp;
  const float c7 = sqrtf(21.0f / (2.0f * pi)) * 0.25f, c8 = sqrtf(7.0f) * 0.25f * rp, c9 = sqrtf(105.0f) * 0.25f * rp;
  o[0] = c0;
  o[1] = -c1 * y;
  o[2] = c1 * z;
  o[3] = -c1 * x;
  o[4] = c2 * x * y;
  o[5] = -c2 * y * z;
  o[6] = c3 * (3.0f * z * z - 1.0f);
  o[7] = -c2 * x * z;
  o[8] = c4 * (x * x - y * y);
  o[9] = -c5 * y * (3.0f * x * x - y * y);
  o[10] = c6 * x * y * z;
  o[11] = -c7 * y * (5.0f * z * z - 1.0f);
  o[12] = c8 * z * (5.0f * z * z - 3.0f);
  o[13] = -c7 * x * (5.0f * z * z - 1.0f);
  o[14] = c9 * z * (x * x - y * y);
  o[15] = -c5 * x * (x * x - 3.0f * y * y);
}

// Corner c (0..7) of level l at cell (cx, cy, cz): grid entry index.
__device__ __forceinline__ uint32_t grid_index(const GuideDev& g, int l, uint32_t x, uint32_t y, uint32_t z) {
  const uint32_t T = 1u << g.log2T;
  if ((g.dense_mask >> l) & 1u) {
    const uint32_t r1 = g.res[l] + 1u;
    return x + y * r1 + z * r1 * r1;
  }
  return (x * 1u ^ y * 2654435761u ^ z * 805459861u) & (T - 1u);
}

struct LevelPos {
  uint32_t c[3];
  float f[3];
};

__device__ __forceinline__ LevelPos level_pos(const GuideDev& g, const float u[3], int l) {
  LevelPos lp;
  const float r = (float)g.res[l];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float s = u[a] * r;
    float fl = floorf(s);
    fl = fminf(fl, r - 1.0f);
    lp.c[a] = (uint32_t)fl;
    lp.f[a] = s - fl;
  }
  return lp;
}

__device__ __forceinline__ void unit_pos(const GuideDev& g, float3 p, float u[3]) {
  u[0] = fminf(fmaxf((p.x - g.lo[0]) * g.inv_ext[0], 0.0f), 1.0f);
  u[1] = fminf(fmaxf((p.y - g.lo[1]) * g.inv_ext[1], 0.0f), 1.0f);
  u[2] = fminf(fmaxf((p.z - g.lo[2]) * g.inv_ext[2], 0.0f), 1.0f);
}

// X row of one record (FP32).
__device__ __forceinline__ void encode(const GuideDev& g, float3 p, float3 n, uint32_t group, float* X) {
  float u[3];
  unit_pos(g, p, u);
  const uint32_t T = 1u << g.log2T;
#pragma unroll 1
  for (int l = 0; l < kLevels; ++l) {
    const LevelPos lp = level_pos(g, u, l);
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
      const float w = (dx ? lp.f[0] : 1.0f - lp.f[0]) * (dy ? lp.f[1] : 1.0f - lp.f[1]) * (dz ? lp.f[2] : 1.0f - lp.f[2]);
      const uint32_t id = grid_index(g, l, lp.c[0] + dx, lp.c[1] + dy, lp.c[2] + dz);
      const float4 v = __ldg((const float4*)g.grid + (size_t)l * T + id);
      a0 = fmaf(w, v.x, a0);
      a1 = fmaf(w, v.y, a1);
      a2 = fmaf(w, v.z, a2);
      a3 = fmaf(w, v.w, a3);
    }
    X[4 * l] = a0;
    X[4 * l + 1] = a1;
    X[4 * l + 2] = a2;
    X[4 * l + 3] = a3;
  }
  sh16(n.x, n.y, n.z, X + 32);
#pragma unroll
  for (int i = 48; i < kIn; ++i) X[i] = 0.0f;
  if (group < 9u) X[48 + group] = 1.0f;
}

// ---------------------------------------------------------------------------
// head
// ---------------------------------------------------------------------------
__device__ __forceinline__ float softplusf(float x) { return x > 30.0f ? x : log1pf(expf(x)); }

struct Mix {
  float pi[kLobes], mu[kLobes][3], kappa[kLobes], mnorm[kLobes];
};

__device__ __forceinline__ void mixture(const float* Y, Mix& h) {
  float mx = -INFINITY;
#pragma unroll
  for (int j = 0; j < kLobes; ++j) mx = fmaxf(mx, Y[5 * j]);
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kLobes; ++j) {
    h.pi[j] = expf(Y[5 * j] - mx);
    s += h.pi[j];
  }
  const float is = 1.0f / s;
#pragma unroll
  for (int j = 0; j < kLobes; ++j) {
    h.pi[j] *= is;
    const float m0 = Y[5 * j + 1], m1 = Y[5 * j + 2], m2 = Y[5 * j + 3];
    const float nm = fmaxf(sqrtf(m0 * m0 + m1 * m1 + m2 * m2), 1e-6f);
    h.mnorm[j] = nm;
    h.mu[j][0] = m0 / nm;
    h.mu[j][1] = m1 / nm;
    h.mu[j][2] = m2 / nm;
    h.kappa[j] = 0.5f + softplusf(Y[5 * j + 4]);
  }
}

__device__ __forceinline__ float vmf_pdf(float kappa, const float* mu, float3 w) {
  const float c = mu[0] * w.x + mu[1] * w.y + mu[2] * w.z;
  return kappa / (2.0f * 3.14159265358979323846f * (-expm1f(-2.0f * kappa))) * expf(kappa * (c - 1.0f));
}

__device__ __forceinline__ float mix_pdf(const Mix& h, float3 w) {
  float q = 0.0f;
#pragma unroll
  for (int j = 0; j < kLobes; ++j) q += h.pi[j] * vmf_pdf(h.kappa[j], h.mu[j], w);
  return q;
}

// ---------------------------------------------------------------------------
// shared-memory operand helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void put_row(unsigned char* A, uint32_t r, const float* v, int ncols) {
  for (int c = 0; c < ncols; ++c)
    *(uint16_t*)(A + (c >> 4) * kSliceA + tc_kmajor_off(r, c & 15)) = tc_bf16_bits(v[c]);
}

// D (TMEM) = A B over nslices K-slices of 16.
__device__ __forceinline__ void gemm(uint32_t d, const unsigned char* A, uint32_t a_slice, const unsigned char* B,
                                     uint32_t b_slice, int nslices, uint32_t idesc, bool accumulate) {
  for (int s = 0; s < nslices; ++s)
    tc_mma_bf16(d, tc_smem_desc(smem_u32(A + s * a_slice)), tc_smem_desc(smem_u32(B + s * b_slice)), idesc,
                (s > 0 || accumulate) ? 1u : 0u);
}

struct Sync {
  uint64_t* mbar;
  uint32_t phase;
  bool ok;
};

// Thread 0 commits the issued MMAs; every thread waits for completion.
__device__ __forceinline__ void mma_wait(Sync& s, uint32_t* status) {
  if (threadIdx.x == 0) tc_commit(s.mbar);
  const int bad = __syncthreads_or(tc_mbar_wait(s.mbar, s.phase, 1u << 24) ? 0 : 1);
  s.phase ^= 1u;
  if (bad) {
    if (threadIdx.x == 0) atomicOr(status, ST_ITER);
    s.ok = false;
  }
  tc_fence_after();
}

// All threads: generic smem writes done -> the next MMA may read them.
__device__ __forceinline__ void publish() {
  tc_fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ __forceinline__ void load_row(uint32_t tmem, uint32_t col, int ncols, float* v) {
  const uint32_t warp = threadIdx.x >> 5;
  for (int c = 0; c < ncols; c += 16) tc_tmem_ld16(tmem + ((warp * 32u) << 16) + col + (uint32_t)c, v + c);
}

__device__ __forceinline__ void load_weights(unsigned char* smem, const uint4* wpack) {
  for (uint32_t i = threadIdx.x; i < kWPack / 16u; i += blockDim.x) ((uint4*)smem)[i] = __ldg(wpack + i);
}

// Record layout: 12 floats {pos.xyz, weight, nrm.xyz, group, omega.xyz, 0}.
struct Rec {
  float3 p, n, w;
  float weight;
  uint32_t group;
};

__device__ __forceinline__ Rec load_rec(const float4* rec, uint64_t i) {
  const float4 a = __ldg(rec + 3 * i), b = __ldg(rec + 3 * i + 1), c = __ldg(rec + 3 * i + 2);
  Rec r;
  r.p = make_float3(a.x, a.y, a.z);
  r.weight = a.w;
  r.n = make_float3(b.x, b.y, b.z);
  r.group = (uint32_t)b.w;
  r.w = make_float3(c.x, c.y, c.z);
  return r;
}

// ---------------------------------------------------------------------------
// forward (evaluation): Y and q(omega) per record
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRows) k_guide_eval(GuideDev g, const uint4* __restrict__ wpack,
                                                      const float4* __restrict__ rec, uint64_t n,
                                                      float* __restrict__ Yout, float* __restrict__ qout,
                                                      uint32_t* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* A0 = smem + kWPack;
  unsigned char* A1 = A0 + kATileB;
  uint64_t* mbar = (uint64_t*)(A1 + kATileB);
  uint32_t* tslot = (uint32_t*)(mbar + 1);
  const uint32_t tid = threadIdx.x, warp = tid >> 5;
  load_weights(smem, wpack);
  if (tid == 0) {
    tc_mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc_tmem_alloc(tslot, 64);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  Sync sy{mbar, 0u, true};
  const uint32_t id64 = tc_idesc_bf16(kRows, 64), id48 = tc_idesc_bf16(kRows, kOut);
  const uint64_t ntiles = (n + kRows - 1) / kRows;
  for (uint64_t tile = blockIdx.x; tile < ntiles && sy.ok; tile += gridDim.x) {
    const uint64_t i = tile * kRows + tid;
    float v[kIn];
    Rec r{};
    if (i < n) {
      r = load_rec(rec, i);
      encode(g, r.p, r.n, r.group, v);
    } else {
      for (int c = 0; c < kIn; ++c) v[c] = 0.0f;
    }
    put_row(A0, tid, v, kIn);
    unsigned char* src = A0;
    unsigned char* dst = A1;
    for (int l = 0; l < 3; ++l) {
      publish();
      if (tid == 0) gemm(tmem, src, kSliceA, smem + wf_off(l), 2048, 4, id64, false);
      mma_wait(sy, status);
      load_row(tmem, 0, kHid, v);
      for (int c = 0; c < kHid; ++c) v[c] = fmaxf(v[c], 0.0f);
      put_row(dst, tid, v, kHid);
      unsigned char* t = src;
      src = dst;
      dst = t;
    }
    publish();
    if (tid == 0) gemm(tmem, src, kSliceA, smem + wf_off(3), kOut * 32, 4, id48, false);
    mma_wait(sy, status);
    load_row(tmem, 0, kOut, v);
    if (i < n && sy.ok) {
      for (int c = 0; c < kOut; ++c) Yout[i * kOut + c] = v[c];
      Mix h;
      mixture(v, h);
      qout[i] = mix_pdf(h, r.w);
    }
    tc_fence_before();
    __syncthreads();
  }
  tc_fence_after();
  if (warp == 0) tc_tmem_dealloc(tmem, 64);
}

// Eight BF16 values to the K-major tile: columns c0 .. c0 + 7 (c0 % 8 == 0)
// of row r form one 16-byte core-matrix row.
__device__ __forceinline__ void put8(unsigned char* A, uint32_t r, int c0, const float* v) {
  uint4 q;
  q.x = tc_bf16x2_bits(v[0], v[1]);
  q.y = tc_bf16x2_bits(v[2], v[3]);
  q.z = tc_bf16x2_bits(v[4], v[5]);
  q.w = tc_bf16x2_bits(v[6], v[7]);
  *(uint4*)(A + (c0 >> 4) * kSliceA + tc_kmajor_off(r, (uint32_t)(c0 & 15))) = q;
}

// Grid entries of the 8 corners k = dx + 2 dy + 4 dz of the level-l cell c:
// the index arithmetic of grid_index() with the per-axis terms formed once
// (identical results: the sums and products wrap modulo 2^32 alike).
__device__ __forceinline__ void corner_ids(const GuideDev& g, const uint32_t* res, int l, const uint32_t c[3],
                                           uint32_t T, uint32_t id[8]) {
  if ((g.dense_mask >> l) & 1u) {
    const uint32_t r1 = res[l] + 1u, r2 = r1 * r1;
    const uint32_t base = c[0] + c[1] * r1 + c[2] * r2;
#pragma unroll
    for (int k = 0; k < 8; ++k) id[k] = base + (uint32_t)(k & 1) + ((k >> 1) & 1 ? r1 : 0u) + ((k >> 2) & 1 ? r2 : 0u);
  } else {
    const uint32_t hy0 = c[1] * 2654435761u, hz0 = c[2] * 805459861u;
    const uint32_t hy1 = hy0 + 2654435761u, hz1 = hz0 + 805459861u;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      id[k] = ((c[0] + (uint32_t)(k & 1)) ^ ((k >> 1) & 1 ? hy1 : hy0) ^ ((k >> 2) & 1 ? hz1 : hz0)) & (T - 1u);
  }
}

// Trilinear weights of the 8 corners, each (w_x w_y) w_z as in encode().
__device__ __forceinline__ void corner_weights(const float fr[3], float w[8]) {
  const float wx[2] = {1.0f - fr[0], fr[0]}, wy[2] = {1.0f - fr[1], fr[1]}, wz[2] = {1.0f - fr[2], fr[2]};
  float wxy[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) wxy[j] = wx[j & 1] * wy[j >> 1];
#pragma unroll
  for (int k = 0; k < 8; ++k) w[k] = wxy[k & 3] * wz[k >> 2];
}

// Hash-grid features of levels l0 .. l0 + 3, 16 values (the arithmetic of
// encode()); res: the per-level resolutions, staged in shared memory.
__device__ __forceinline__ void encode_levels4(const GuideDev& g, const uint32_t* res, const float u[3], int l0,
                                               float* f) {
  const uint32_t T = 1u << g.log2T;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int l = l0 + i;
    const float rl = (float)res[l];
    uint32_t c[3];
    float fr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float sa = u[a] * rl;
      const float fl = fminf(floorf(sa), rl - 1.0f);
      c[a] = (uint32_t)fl;
      fr[a] = sa - fl;
    }
    uint32_t id[8];
    corner_ids(g, res, l, c, T, id);
    float w[8];
    corner_weights(fr, w);
    const float4* tab = (const float4*)g.grid + (size_t)l * T;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float4 v = __ldg(tab + id[k]);
      a0 = fmaf(w[k], v.x, a0);
      a1 = fmaf(w[k], v.y, a1);
      a2 = fmaf(w[k], v.z, a2);
      a3 = fmaf(w[k], v.w, a3);
    }
    f[4 * i] = a0;
    f[4 * i + 1] = a1;
    f[4 * i + 2] = a2;
    f[4 * i + 3] = a3;
  }
}

// ---------------------------------------------------------------------------
// training: forward, loss gradient, backward, gradient accumulation
// ---------------------------------------------------------------------------
// A CTA of 256 threads serves 128 records per tile, two threads per record
// (half h = t / 128; threads t and t + 128 share a TMEM lane).  Records of
// zero weight add nothing to the loss or its gradient and are skipped: each
// CTA walks a contiguous chunk of the batch, four records per thread and
// round, and compacts the indices of the weighted records into full tiles.
// Weight gradients dW_l = H_{l-1}^T dZ_l use A' = [H_{l-1}^T; 0] (M = 128)
// and B' = dZ_l^T, both made from the K-major activation tiles by 8 x 8
// transposes (ldmatrix / stmatrix.trans), and accumulate in TMEM over all
// tiles of the CTA; each CTA then stores its sums as one partial (layer l's
// block column-major: element (in, o) at w_off(l) + 64 o + in) and
// k_dw_reduce adds the partials in a fixed order.
constexpr int kTrainThreads = 2 * kRows;
constexpr uint32_t kTrX = kWPack;
constexpr uint32_t kTrH1 = kTrX + kATileB;
constexpr uint32_t kTrH2 = kTrH1 + kATileB;
constexpr uint32_t kTrH3 = kTrH2 + kATileB;
constexpr uint32_t kTrDZ = kTrH3 + kATileB;
constexpr uint32_t kTrAp = kTrDZ + kATileB;           // [128 x 128] = 32 KB
constexpr uint32_t kTrBp = kTrAp + 8 * kSliceA;       // <= [64 x 128] = 16 KB
constexpr uint32_t kTrScan = 4;                       // records per thread and scan round
constexpr uint32_t kTrListN = kRows + kTrScan * kTrainThreads;  // a short tile + one round
constexpr uint32_t kTrList = kTrBp + 8 * 64 * 32;     // record indices
constexpr uint32_t kTrMisc = kTrList + kTrListN * 4;
constexpr uint32_t kTrainSmem = kTrMisc + 128;
static_assert(kTrainSmem <= 227 * 1024, "training kernel shared memory");

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
               : "r"(addr)
               : "memory");
}

__device__ __forceinline__ void stsm_x4_trans(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b),
               "r"(c), "r"(d)
               : "memory");
}

// Core matrix (row group g, column block b) of a K-major tile whose 16-wide
// K-slices are `slice` bytes apart: address of its row i.
__device__ __forceinline__ uint32_t core_row(uint32_t base, uint32_t slice, uint32_t g, uint32_t b, uint32_t i) {
  return base + (b >> 1) * slice + i * 16u + g * 256u + (b & 1u) * 128u;
}

// Transposes of the 8 x 8 core matrices of a [128 records x ncols] K-major
// tile (slices 4096 B) into a [ncols rows x 128 records] K-major tile
// (slices dst_slice B): core (record group g, column block b) -> core
// (column group b, record block g).  The whole CTA, 4 cores per warp op.
__device__ __forceinline__ void transpose_tile(const unsigned char* src, unsigned char* dst, uint32_t dst_slice,
                                               uint32_t ncols) {
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t ncores = 16u * (ncols / 8u);
  const uint32_t s = smem_u32(src), d = smem_u32(dst);
  for (uint32_t c0 = warp * 4u; c0 < ncores; c0 += (blockDim.x >> 5) * 4u) {
    const uint32_t c = c0 + (lane >> 3), i = lane & 7u;
    const uint32_t g = c & 15u, b = c >> 4;
    uint32_t r0, r1, r2, r3;
    ldsm_x4(core_row(s, kSliceA, g, b, i), r0, r1, r2, r3);
    stsm_x4_trans(core_row(d, dst_slice, b, g, i), r0, r1, r2, r3);
  }
}

__global__ void __launch_bounds__(kTrainThreads, 1)
    k_guide_train(GuideDev g, const uint4* __restrict__ wpack, const float4* __restrict__ rec, uint64_t n,
                  const float* __restrict__ wsum, float* __restrict__ dWpart, float* __restrict__ dgrid,
                  float* __restrict__ loss, uint32_t* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* AX = smem + kTrX;
  unsigned char* ADZ = smem + kTrDZ;
  unsigned char* Ap = smem + kTrAp;
  unsigned char* Bp = smem + kTrBp;
  uint32_t* list = (uint32_t*)(smem + kTrList);
  uint64_t* mbar = (uint64_t*)(smem + kTrMisc);
  uint32_t* tslot = (uint32_t*)(mbar + 1);
  float* lsum = (float*)(tslot + 1);
  uint32_t* wcnt = (uint32_t*)(lsum + 1);  // [8] per-warp counts, [8] list length
  uint32_t* sres = wcnt + 9;               // [kLevels] grid resolutions
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
  const uint32_t r = tid & (kRows - 1), h = tid >> 7;
  load_weights(smem, wpack);
  // A' rows 64..127 stay zero
  for (uint32_t i = tid; i < 8u * kSliceA / 16u; i += blockDim.x) ((uint4*)Ap)[i] = make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int l = 0; l < kLevels; ++l)
    if (tid == (uint32_t)l) sres[l] = g.res[l];
  if (tid == 0) {
    tc_mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *lsum = 0.0f;
    wcnt[8] = 0u;
  }
  if (warp == 0) tc_tmem_alloc(tslot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t trow = tmem + (((warp & 3u) * 32u) << 16);
  Sync sy{mbar, 0u, true};
  const uint32_t id64 = tc_idesc_bf16(kRows, 64), id48 = tc_idesc_bf16(kRows, kOut);
  const float total = *wsum;
  const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
  const uint64_t c0 = min((uint64_t)blockIdx.x * per, n), c1 = min(c0 + per, n);
  uint64_t cur = c0;
  bool first = true;
  float my_loss = 0.0f;
  while (sy.ok) {
    // compact the indices of weighted records until a tile is full
    uint32_t nl = wcnt[8];
    while (nl < (uint32_t)kRows && cur < c1) {
      // records cur + tid + 256 q, q < 4: independent loads, one scan
      bool take[kTrScan];
      uint32_t cnt_t = 0;
#pragma unroll
      for (uint32_t q = 0; q < kTrScan; ++q) {
        const uint64_t i = cur + tid + (uint64_t)q * kTrainThreads;
        take[q] = i < c1 && __ldg((const float*)(rec + 3 * i) + 3) > 0.0f;
        cnt_t += take[q] ? 1u : 0u;
      }
      uint32_t incl = cnt_t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += v;
      }
      if (lane == 31) wcnt[warp] = incl;
      __syncthreads();
      uint32_t off = nl + incl - cnt_t;
      for (uint32_t w2 = 0; w2 < warp; ++w2) off += wcnt[w2];
#pragma unroll
      for (uint32_t q = 0; q < kTrScan; ++q)
        if (take[q]) list[off++] = (uint32_t)(cur + tid + (uint64_t)q * kTrainThreads - c0);
      uint32_t tot = 0;
      for (uint32_t w2 = 0; w2 < (blockDim.x >> 5); ++w2) tot += wcnt[w2];
      __syncthreads();
      nl += tot;
      cur += (uint64_t)kTrScan * kTrainThreads;
    }
    if (nl == 0) break;
    const uint32_t nt = min(nl, (uint32_t)kRows);
    const bool valid = r < nt;
    const uint64_t ri = valid ? c0 + list[r] : 0;
    Rec rc{};
    if (valid) rc = load_rec(rec, ri);
    // carry the surplus indices over to the next tile
    __syncthreads();
    uint32_t carry[kTrScan];
#pragma unroll
    for (uint32_t q = 0; q < kTrScan; ++q) {
      const uint32_t t = tid + q * kTrainThreads;
      carry[q] = t < nl - nt ? list[kRows + t] : 0u;
    }
    __syncthreads();
#pragma unroll
    for (uint32_t q = 0; q < kTrScan; ++q) {
      const uint32_t t = tid + q * kTrainThreads;
      if (t < nl - nt) list[t] = carry[q];
    }
    if (tid == 0) wcnt[8] = nl - nt;
    // encoding: half 0 grid levels 0-3 and SH, half 1 levels 4-7 and group
    {
      float u[3], f[16];
      unit_pos(g, rc.p, u);
      if (valid) {
        encode_levels4(g, sres, u, 4 * (int)h, f);
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) f[c] = 0.0f;
      }
      put8(AX, r, 16 * (int)h, f);
      put8(AX, r, 16 * (int)h + 8, f + 8);
      if (h == 0) {
        if (valid) sh16(rc.n.x, rc.n.y, rc.n.z, f);
        put8(AX, r, 32, f);
        put8(AX, r, 40, f + 8);
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) f[c] = (valid && (uint32_t)c == rc.group) ? 1.0f : 0.0f;
        put8(AX, r, 48, f);
        put8(AX, r, 56, f + 8);
      }
    }
    // forward
    for (int l = 0; l < 3; ++l) {
      publish();
      if (tid == 0) gemm(tmem, smem + kTrX + kATileB * (uint32_t)l, kSliceA, smem + wf_off(l), 2048, 4, id64, false);
      mma_wait(sy, status);
      float v[32];
      tc_tmem_ld16x2(trow + 32u * h, v);
      unsigned char* Hl = smem + kTrH1 + kATileB * (uint32_t)l;
#pragma unroll
      for (int c = 0; c < 32; c += 8) {
        float t[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) t[e] = fmaxf(v[c + e], 0.0f);
        put8(Hl, r, 32 * (int)h + c, t);
      }
    }
    publish();
    if (tid == 0) gemm(tmem, smem + kTrH3, kSliceA, smem + wf_off(3), kOut * 32, 4, id48, false);
    mma_wait(sy, status);
    // head (half 0): loss and dL/dY, written as dZ_3 into ADZ
    if (h == 0) {
      float y[48];
      tc_tmem_ld16x2(trow, y);
      tc_tmem_ld16(trow + 32u, y + 32);
      const float a = (valid && total > 0.0f) ? rc.weight / total : 0.0f;
      float dY[kOut];
#pragma unroll
      for (int c = 0; c < kOut; ++c) dY[c] = 0.0f;
      if (a > 0.0f) {
        Mix mx;
        mixture(y, mx);
        float pj[kLobes], q = 0.0f;
#pragma unroll
        for (int j = 0; j < kLobes; ++j) {
          pj[j] = vmf_pdf(mx.kappa[j], mx.mu[j], rc.w);
          q += mx.pi[j] * pj[j];
        }
        my_loss -= a * logf(q);
        const float3 w = rc.w;
#pragma unroll
        for (int j = 0; j < kLobes; ++j) {
          const float rj = mx.pi[j] * pj[j] / q;
          const float c = mx.mu[j][0] * w.x + mx.mu[j][1] * w.y + mx.mu[j][2] * w.z;
          dY[5 * j] = -a * (rj - mx.pi[j]);
          const float fj = -a * rj * mx.kappa[j] / mx.mnorm[j];
          dY[5 * j + 1] = fj * (w.x - c * mx.mu[j][0]);
          dY[5 * j + 2] = fj * (w.y - c * mx.mu[j][1]);
          dY[5 * j + 3] = fj * (w.z - c * mx.mu[j][2]);
          const float k = mx.kappa[j];
          const float dlogp = 1.0f / k - 2.0f / expm1f(2.0f * k) + (c - 1.0f);
          dY[5 * j + 4] = -a * rj * dlogp / (1.0f + expf(-y[5 * j + 4]));
        }
      }
#pragma unroll
      for (int c = 0; c < kOut; c += 8) put8(ADZ, r, c, dY + c);
    }
    // backward: layer l = 3 (W4, out 48) down to 0 (W1)
    for (int l = 3; l >= 0; --l) {
      const uint32_t out = (uint32_t)layer_out(l);
      const unsigned char* Hin = smem + kTrX + kATileB * (uint32_t)l;  // H_{l-1} (X for l = 0)
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      transpose_tile(ADZ, Bp, out * 32u, out);
      transpose_tile(Hin, Ap, kSliceA, kHid);
      publish();
      if (tid == 0) {
        // dW_l (+)= H_{l-1}^T dZ_l : M 128 (64 used), N = out, K = 128 records
        gemm(tmem + 64u * (uint32_t)(l + 1), Ap, kSliceA, Bp, out * 32u, 8, tc_idesc_bf16(kRows, out), !first);
        // dH_{l-1} = dZ_l W_l^T : M 128, N 64, K = out
        gemm(tmem, ADZ, kSliceA, smem + wb_off(l), 2048, (int)out / 16, id64, false);
      }
      mma_wait(sy, status);
      if (l > 0) {
        // dZ_{l-1} = dH_{l-1} where the forward activation was positive
        float v[32];
        tc_tmem_ld16x2(trow + 32u * h, v);
        const unsigned char* Hm = smem + kTrX + kATileB * (uint32_t)l;
#pragma unroll
        for (int c = 0; c < 32; c += 8) {
          const int col = 32 * (int)h + c;
          const uint4 hb = *(const uint4*)(Hm + (col >> 4) * kSliceA + tc_kmajor_off(r, (uint32_t)(col & 15)));
          const uint32_t hw[4] = {hb.x, hb.y, hb.z, hb.w};
          float t[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const uint32_t bits = (hw[e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
            t[e] = tc_bf16_val((uint16_t)bits) > 0.0f ? v[c + e] : 0.0f;
          }
          put8(ADZ, r, col, t);
        }
      } else {
        // dX of grid levels 4h .. 4h + 3 -> grid gradient
        float dx[16];
        tc_tmem_ld16(trow + 16u * h, dx);
        if (valid && rc.weight > 0.0f && total > 0.0f) {
          float u[3];
          unit_pos(g, rc.p, u);
          const uint32_t T = 1u << g.log2T;
#pragma unroll 1
          for (int i = 0; i < 4; ++i) {
            const int l2 = 4 * (int)h + i;
            const float d0 = dx[4 * i], d1 = dx[4 * i + 1], d2 = dx[4 * i + 2], d3 = dx[4 * i + 3];
            if (d0 == 0.0f && d1 == 0.0f && d2 == 0.0f && d3 == 0.0f) continue;
            const float rl = (float)sres[l2];
            uint32_t c[3];
            float fr[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              const float sa = u[a] * rl;
              const float fl = fminf(floorf(sa), rl - 1.0f);
              c[a] = (uint32_t)fl;
              fr[a] = sa - fl;
            }
            uint32_t id[8];
            corner_ids(g, sres, l2, c, T, id);
            float w[8];
            corner_weights(fr, w);
            float4* dst = (float4*)dgrid + (size_t)l2 * T;
#pragma unroll
            for (int k = 0; k < 8; ++k) atomicAdd(dst + id[k], make_float4(w[k] * d0, w[k] * d1, w[k] * d2, w[k] * d3));
          }
        }
      }
    }
    first = false;
  }
  // accumulated weight gradients: TMEM lanes 0..63 (warps 0, 1, 4, 5) =
  // input rows; this CTA's partial, element (in, o) of layer l at
  // w_off(l) + 64 o + in (a warp stores 32 consecutive floats per column)
  float* part = dWpart + (size_t)blockIdx.x * kWSize;
  if (!first && sy.ok) {
    if ((warp & 3u) < 2u) {
      const uint32_t in = (warp & 1u) * 32u + lane;
      for (int l = 0; l < 4; ++l) {
        const int out = layer_out(l);
        float row[32];
        // half 0 columns 0..31, half 1 columns 32..out-1
        const int o0 = 32 * (int)h, nc = min(32, out - o0);
        const uint32_t col0 = 64u * (uint32_t)(l + 1) + (uint32_t)o0;
        if (nc == 32) {
          tc_tmem_ld16x2(trow + col0, row);
        } else {
          tc_tmem_ld16(trow + col0, row);
        }
        for (int o = 0; o < nc; ++o) part[w_off(l) + 64 * (o0 + o) + in] = row[o];
      }
    }
  } else {
    for (int e = (int)tid; e < kWSize; e += (int)blockDim.x) part[e] = 0.0f;
  }
  if (my_loss != 0.0f) atomicAdd(lsum, my_loss);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) atomicAdd(loss, *lsum);
  if (warp == 0) tc_tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// small kernels: weight sum, Adam, BF16 packing, initialisation
// ---------------------------------------------------------------------------
__global__ void k_weight_sum(const float4* __restrict__ rec, uint64_t n, float* out) {
  float s = 0.0f;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    s += __ldg(rec + 3 * i).w;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// dW = sum over the CTAs' partials (column-major blocks, see k_guide_train):
// 32 weights per block, warp w adds partials w, w + 8, ..., then the eight
// warp sums are added in warp order (the same order every call).
__global__ void __launch_bounds__(256) k_dw_reduce(const float* __restrict__ part, int nparts, float* __restrict__ dW) {
  __shared__ float acc[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * 32 + lane;
  float s = 0.0f;
  if (e < kWSize)
    for (int c = warp; c < nparts; c += 8) s += __ldg(part + (size_t)c * kWSize + e);
  acc[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && e < kWSize) {
    float t = acc[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) t += acc[w][lane];
    const int l = e / 4096, loc = e - 4096 * l;
    const int out = layer_out(l), o = loc / 64, in = loc - 64 * o;
    if (o < out) dW[w_off(l) + in * out + o] = t;
  }
}

__device__ __forceinline__ void adam1(float& p, float& m, float& v, float g, float lr, float b1, float b2, float eps,
                                      float c1, float c2) {
  m = b1 * m + (1.0f - b1) * g;
  v = b2 * v + (1.0f - b2) * g * g;
  p -= lr * (m * c1) / (sqrtf(v * c2) + eps);
}

// One Adam step over n parameters: four per thread and iteration with
// 16-byte accesses (the arrays come from cudaMalloc), the last n % 4 one by
// one; the same arithmetic per element.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, uint64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const uint64_t n4 = n / 4, stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 gi = ((const float4*)g)[i];
    float4 mi = ((float4*)m)[i], vi = ((float4*)v)[i], pi = ((float4*)p)[i];
    adam1(pi.x, mi.x, vi.x, gi.x, lr, b1, b2, eps, c1, c2);
    adam1(pi.y, mi.y, vi.y, gi.y, lr, b1, b2, eps, c1, c2);
    adam1(pi.z, mi.z, vi.z, gi.z, lr, b1, b2, eps, c1, c2);
    adam1(pi.w, mi.w, vi.w, gi.w, lr, b1, b2, eps, c1, c2);
    ((float4*)m)[i] = mi;
    ((float4*)v)[i] = vi;
    ((float4*)p)[i] = pi;
  }
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t < n - 4 * n4) {
    const uint64_t i = 4 * n4 + t;
    adam1(p[i], m[i], v[i], g[i], lr, b1, b2, eps, c1, c2);
  }
}

// FP32 master weights -> BF16 operand tiles (forward W^T, backward W).
__global__ void k_pack_weights(const float* __restrict__ W, unsigned char* __restrict__ pack) {
  for (int l = 0; l < 4; ++l) {
    const int out = layer_out(l);
    const float* Wl = W + w_off(l);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kIn * out; e += gridDim.x * blockDim.x) {
      const int i = e / out, o = e - i * out;  // W_l[i][o]
      const uint16_t b = tc_bf16_bits(Wl[e]);
      // forward B: row o (N = out), K = i
      *(uint16_t*)(pack + wf_off(l) + (i >> 4) * (out * 32) + tc_kmajor_off(o, i & 15)) = b;
      // backward B: row i (N = in), K = o
      *(uint16_t*)(pack + wb_off(l) + (o >> 4) * (kHid * 32) + tc_kmajor_off(i, o & 15)) = b;
    }
  }
}

__device__ __forceinline__ float philox_u(uint32_t seed0, uint32_t seed1, uint32_t a, uint32_t b) {
  uint32_t k0 = seed0, k1 = seed1;
  uint4 c = make_uint4(a, b, 0x6775u, 0x1de);
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return (float)(c.x >> 8) * 5.9604644775390625e-8f;
}

__global__ void k_guide_init(float* grid, uint64_t n_grid, float* W, uint32_t s0, uint32_t s1) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_grid; i += (uint64_t)gridDim.x * blockDim.x)
    grid[i] = (philox_u(s0, s1, (uint32_t)i, (uint32_t)(i >> 32)) - 0.5f) * 2e-4f;
  for (int l = 0; l < 4; ++l) {
    const int out = layer_out(l);
    const float s = sqrtf(6.0f / (float)(kIn + out));
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kIn * out; e += gridDim.x * blockDim.x)
      W[w_off(l) + e] = (2.0f * philox_u(s0, s1, 0x80000000u + w_off(l) + e, 7u) - 1.0f) * s;
  }
}

// ---------------------------------------------------------------------------
// guided sampling inside the wavefront (one-sample MIS with cosine sampling)
// ---------------------------------------------------------------------------
// vMF direction (Jakob, "Numerically stable sampling of the von Mises-Fisher
// distribution on S^2", 2012): w = 1 + log(u + (1 - u) e^{-2 kappa}) / kappa.
__device__ __forceinline__ float3 vmf_sample(const float* mu, float kappa, float u, float v) {
  const float w = 1.0f + logf(u + (1.0f - u) * expf(-2.0f * kappa)) / kappa;
  const float r = sqrtf(fmaxf(0.0f, 1.0f - w * w));
  float sp, cp;
  sincospif(2.0f * v, &sp, &cp);
  float3 t1, t2;
  const float3 m = make_float3(mu[0], mu[1], mu[2]);
  onb(m, t1, t2);
  return make_float3(r * cp * t1.x + r * sp * t2.x + w * m.x, r * cp * t1.y + r * sp * t2.y + w * m.y,
                     r * cp * t1.z + r * sp * t2.z + w * m.z);
}

constexpr uint32_t kSmWf = 30720;                      // forward weight tiles
constexpr int kSampleThreads = 2 * kRows;              // two threads per query
constexpr int kXch = 12;                               // head exchange floats per query
constexpr uint32_t kSmXch = kSmWf + kATileB;           // one activation tile, updated in place
constexpr uint32_t kSampleSmem = kSmXch + kRows * kXch * 4u + 128u;
// three CTAs per SM (85 registers, no spills): measured 614 ms per guided
// sample pass of the 2M-triangle nave against 911 ms with four (64
// registers, spilled) and 668 ms with two, queries in queue order
#ifndef SRT_GUIDE_SAMPLE_CTAS
#define SRT_GUIDE_SAMPLE_CTAS 3
#endif
constexpr int kSampleCtasPerSm = SRT_GUIDE_SAMPLE_CTAS;

// Guided continuation at the wave's guide queries of vertex k.  A CTA takes
// tiles of 128 queries; thread t serves query t % 128 as half h = t / 128
// (threads t and t + 128 share a TMEM lane).  Encoding: half 0 the grid
// levels 0-3 and the SH of the normal, half 1 levels 4-7 and the band
// group; each hidden layer runs on the tensor cores and the epilogue (ReLU,
// BF16) rewrites the activation tile in place, half h taking columns
// 32h .. 32h + 31.  Head: half h owns lobes 4h .. 4h + 3; the softmax
// maximum and sum, the sampled direction and the two partial mixture
// densities are exchanged through shared memory.  Half 0 then finishes the
// query (MIS pdf, sun-sample weight, continuation ray, training slot).
__global__ void __launch_bounds__(kSampleThreads, kSampleCtasPerSm)
    k_guide_sample(GuideDev g, const uint4* __restrict__ wpack, DevSpectra P, WaveParams w, uint32_t k, GuideWave gw,
                   float4* __restrict__ qout, float4* __restrict__ sq, float* __restrict__ Lbuf,
                   uint32_t* __restrict__ sigbuf, Counters* cnt, uint32_t cap, double* __restrict__ accum, Probe probe,
                   bool record, uint32_t* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* A = smem + kSmWf;
  float* xch = (float*)(smem + kSmXch);
  uint64_t* mbar = (uint64_t*)(smem + kSmXch + kRows * kXch * 4u);
  uint32_t* tslot = (uint32_t*)(mbar + 1);
  uint32_t* sres = tslot + 1;
  const uint32_t tid = threadIdx.x, warp = tid >> 5;
  const uint32_t r = tid & (kRows - 1), h = tid >> 7;
#pragma unroll
  for (int l = 0; l < kLevels; ++l)
    if (tid == (uint32_t)l) sres[l] = g.res[l];
  float* X = xch + r * kXch;
  for (uint32_t i = tid; i < kSmWf / 16u; i += blockDim.x) ((uint4*)smem)[i] = __ldg(wpack + i);
  if (tid == 0) {
    tc_mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc_tmem_alloc(tslot, 64);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t trow = tmem + (((warp & 3u) * 32u) << 16);
  Sync sy{mbar, 0u, true};
  const uint32_t id64 = tc_idesc_bf16(kRows, 64), id48 = tc_idesc_bf16(kRows, kOut);
  const uint32_t count = min(cnt[k].g_count, cap);
  const uint64_t ntiles = (count + kRows - 1) / kRows;
  const float alpha = gw.alpha;
  const float inv_pi = 0.31830988618379067f;
  const float p_cone = 1.0f / (2.0f * 3.14159265358979323846f * P.one_minus_cos);
  for (uint64_t tile = blockIdx.x; tile < ntiles && sy.ok; tile += gridDim.x) {
    const uint32_t jq = (uint32_t)(tile * kRows) + r;
    const bool valid = jq < count;
    float4 q0 = make_float4(0, 0, 0, 0), q1 = make_float4(0, 0, 1, 0), q2 = make_float4(0, 0, 0, 0);
    if (valid) {
      const uint32_t i = gw.perm ? __ldg(gw.perm + jq) : jq;
      q0 = __ldg(gw.gq + 3 * i);
      q1 = __ldg(gw.gq + 3 * i + 1);
      q2 = __ldg(gw.gq + 3 * i + 2);
    }
    const uint32_t bits = __float_as_uint(q0.w), pid = bits & kPidMask;
    const PathId id = path_id(w, pid);
    const uint32_t band = w.band_first + id.j;
    const uint32_t group = band * 9u / w.n_bands;
    {
      float u[3], f[16];
      unit_pos(g, f3(q0), u);
      encode_levels4(g, sres, u, 4 * (int)h, f);
      put8(A, r, 16 * (int)h, f);
      put8(A, r, 16 * (int)h + 8, f + 8);
      if (h == 0) {
        sh16(q1.x, q1.y, q1.z, f);
        put8(A, r, 32, f);
        put8(A, r, 40, f + 8);
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) f[c] = (uint32_t)c == group ? 1.0f : 0.0f;
        put8(A, r, 48, f);
        put8(A, r, 56, f + 8);
      }
    }
    for (int l = 0; l < 3; ++l) {
      publish();
      if (tid == 0) gemm(tmem, A, kSliceA, smem + wf_off(l), 2048, 4, id64, false);
      mma_wait(sy, status);
      float v[32];
      tc_tmem_ld16x2(trow + 32u * h, v);
#pragma unroll
      for (int c = 0; c < 32; c += 8) {
        float t[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) t[e] = fmaxf(v[c + e], 0.0f);
        put8(A, r, 32 * (int)h + c, t);
      }
    }
    publish();
    if (tid == 0) gemm(tmem, A, kSliceA, smem + wf_off(3), kOut * 32, 4, id48, false);
    mma_wait(sy, status);
    // head: lobes 4h .. 4h + 3 are Y[20h .. 20h + 19]; half 1 loads columns 16 .. 47
    float y[32];
    tc_tmem_ld16x2(trow + 16u * h, y);
#pragma unroll
    for (int c = 0; c < 20; ++c) y[c] = h ? y[c + 4] : y[c];
    float mx = -INFINITY;
#pragma unroll
    for (int j = 0; j < 4; ++j) mx = fmaxf(mx, y[5 * j]);
    X[h] = mx;
    tc_fence_before();
    __syncthreads();
    mx = fmaxf(X[0], X[1]);
    float e[4], s = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      e[j] = expf(y[5 * j] - mx);
      s += e[j];
    }
    X[2 + h] = s;
    __syncthreads();
    const float s0 = X[2], S = s0 + X[3];
    const float is = 1.0f / S;
    float pi[4], mu[4][3], kap[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      pi[j] = e[j] * is;
      const float m0 = y[5 * j + 1], m1 = y[5 * j + 2], m2 = y[5 * j + 3];
      const float nm = fmaxf(sqrtf(m0 * m0 + m1 * m1 + m2 * m2), 1e-6f);
      mu[j][0] = m0 / nm;
      mu[j][1] = m1 / nm;
      mu[j][2] = m2 / nm;
      kap[j] = 0.5f + softplusf(y[5 * j + 4]);
    }
    // one-sample MIS: guide with probability alpha, else cosine sampling;
    // lobe choice on the unnormalised cumulative sum (half 0 first)
    const uint4 u1 = philox4x32_10(make_uint4(id.pix, id.s, band, 4u * k + 1u), w.key0, w.key1);
    const bool guide = u01(u1.x) < alpha;
    const float U = u01(u1.y) * S;
    const bool mine = guide ? (h == 0 ? U < s0 : !(U < s0)) : h == 0;
    const float3 n = f3(q1);
    if (valid && mine) {
      float3 om;
      if (guide) {
        float acc = h == 0 ? 0.0f : s0;
        int sel = 3;
        bool found = false;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc += e[j];
          if (!found && U < acc) {
            sel = j;
            found = true;
          }
        }
        float m[3] = {mu[0][0], mu[0][1], mu[0][2]}, kk = kap[0];
#pragma unroll
        for (int j = 1; j < 4; ++j)
          if (sel == j) {
            m[0] = mu[j][0];
            m[1] = mu[j][1];
            m[2] = mu[j][2];
            kk = kap[j];
          }
        om = vmf_sample(m, kk, u01(u1.z), u01(u1.w));
      } else {
        const uint4 u0 = philox4x32_10(make_uint4(id.pix, id.s, band, 4u * k), w.key0, w.key1);
        const float rr = sqrtf(u01(u0.z));
        const float zz = sqrtf(fmaxf(0.0f, 1.0f - u01(u0.z)));
        float s2, c2;
        sincospif(2.0f * u01(u0.w), &s2, &c2);
        float3 b1, b2;
        onb(n, b1, b2);
        om = make_float3(rr * c2 * b1.x + rr * s2 * b2.x + zz * n.x, rr * c2 * b1.y + rr * s2 * b2.y + zz * n.y,
                         rr * c2 * b1.z + rr * s2 * b2.z + zz * n.z);
      }
      X[4] = om.x;
      X[5] = om.y;
      X[6] = om.z;
    }
    __syncthreads();
    const float3 om = make_float3(X[4], X[5], X[6]);
    // partial mixture densities at the continuation and at the pending sun sample
    const uint32_t ss = __float_as_uint(q2.y);
    const bool has_sun = valid && ss != 0xFFFFFFFFu;
    float4 sv = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
    if (has_sun) sv = sq[2 * ss + 1];
    const float3 wn = has_sun ? f3(sv) : make_float3(0, 0, 1);
    float qo = 0.0f, qn = 0.0f;
    if (valid) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        qo += pi[j] * vmf_pdf(kap[j], mu[j], om);
        qn += pi[j] * vmf_pdf(kap[j], mu[j], wn);
      }
    }
    X[7 + 2 * h] = qo;
    X[8 + 2 * h] = qn;
    __syncthreads();
    if (h != 0) continue;  // half 1 goes on to the next tile's encoding; no barrier is skipped
    bool cont = false;
    float4 r0 = make_float4(0, 0, 0, 0), r1 = r0;
    if (valid && sy.ok) {
      const float c = dot(n, om);
      const float pdf = alpha * (X[7] + X[9]) + (1.0f - alpha) * fmaxf(c, 0.0f) * inv_pi;
      // direct sun by two strategies, balance heuristic: rescale the pending
      // sun sample, weight a later escape of the continuation into the cone
      float cn = 0.0f;
      if (has_sun) {
        cn = dot(n, wn);
        const float pm = alpha * (X[8] + X[10]) + (1.0f - alpha) * fmaxf(cn, 0.0f) * inv_pi;
        sq[2 * ss + 1].w = sv.w * (p_cone / (p_cone + pm));
      }
      float Tn = 0.0f;
      if (c > 0.0f && pdf > 0.0f) {
        cont = true;
        Tn = q1.w * q2.x * inv_pi * c / pdf;
        const bool in_cone = dot(om, P.sun) >= P.cos_max;
        gw.wesc[pid] = in_cone ? pdf / (pdf + p_cone) : 0.0f;
        r0 = make_float4(q0.x, q0.y, q0.z, __uint_as_float(bits | kFlagGuidedEsc));
        r1 = make_float4(om.x, om.y, om.z, Tn);
      } else {
        // no continuation: the path ends here, after its pending sun ray
        if (has_sun) {
          float4* t = sq + 2 * ss;
          t->w = __uint_as_float(__float_as_uint(t->w) | kFlagTerm);
        } else {
          const float Lp = Lbuf[pid];
          finalize(w, id, Lp, record ? sigbuf[pid] : 0u, accum, probe, record);
          if (gw.Lfinal) gw.Lfinal[pid] = Lp;
        }
      }
      if (gw.collect != 0u && pid % gw.collect == 0u) {
        float4* raw = gw.raw + kRawF4 * ((k - 1u) * gw.slots_per_vertex + pid / gw.collect);
        raw[0] = make_float4(q0.x, q0.y, q0.z, (float)group);
        float* r1p = (float*)(raw + 1);
        r1p[0] = q1.x;
        r1p[1] = q1.y;
        r1p[2] = q1.z;
        raw[2] = make_float4(om.x, om.y, om.z, pdf);
        raw[3] = make_float4(c, Tn, 1.0f, (float)pid);
        raw[4] = make_float4(wn.x, wn.y, wn.z, cn);
        float* r5p = (float*)(raw + 5);  // r5.x (sun radiance) is written by the sun-ray kernel
        r5p[1] = p_cone;
        r5p[2] = (has_sun && cn > 0.0f) ? 1.0f : 0.0f;
      }
    }
    const uint32_t slot = warp_append(&cnt[k + 1].q_count, cont);
    if (cont) {
      if (slot < cap) {
        __stcs(qout + 2 * slot, r0);
        __stcs(qout + 2 * slot + 1, r1);
      } else {
        atomicOr(status, ST_QUEUE);
      }
    }
  }
  tc_fence_after();
  if (warp == 0) tc_tmem_dealloc(tmem, 64);
}

// ---------------------------------------------------------------------------
// spatial order of a wave's guide queries (counting sort on a 64^3 Morton
// grid): queries of one 128-query tile then lie in one or a few cells, so
// their hash-grid gathers share cache lines at all but the finest levels
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  // bits b0..b5 -> positions 0, 3, 6, .., 15
  uint32_t r = 0;
#pragma unroll
  for (uint32_t b = 0; b < kGuideSortBits; ++b) r |= ((v >> b) & 1u) << (3u * b);
  return r;
}

__global__ void k_gsort_hist(GuideDev g, GuideWave gw, const Counters* __restrict__ cnt, uint32_t k, uint32_t cap) {
  const uint32_t count = min(cnt[k].g_count, cap);
  const float cells = (float)(1u << kGuideSortBits);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const float4 q0 = __ldg(gw.gq + 3 * i);
    float u[3];
    unit_pos(g, f3(q0), u);
    uint32_t c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = min((uint32_t)(u[a] * cells), (1u << kGuideSortBits) - 1u);
    const uint32_t key = spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
    gw.skey[i] = key;
    atomicAdd(gw.bins + key, 1u);
  }
}

__global__ void k_gsort_scatter(GuideWave gw, const Counters* __restrict__ cnt, uint32_t k, uint32_t cap) {
  const uint32_t count = min(cnt[k].g_count, cap);
  const uint32_t* totals = gw.bins + kGuideSortBins;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const uint32_t key = gw.skey[i];
    gw.perm[__ldg(totals + (key >> 10)) + atomicAdd(gw.bins + key, 1u)] = i;
  }
}

// Training records from the wave's slots, two per slot: the continuation,
// with incident radiance L_in = (final radiance - radiance before the next
// vertex) / throughput after the vertex and weight L_in cos / MIS pdf; and
// the sun sample, weight (sun radiance x transmittance) cos / p_cone.  Record
// r goes to position (r * perm_mul) mod (2 n_slots) so that any contiguous
// batch spans the whole image.
__device__ __forceinline__ void put_record(float4* out, uint32_t pos, float3 p, float wt, float3 n, float group,
                                           float3 om) {
  float4* o = out + 3u * pos;
  if (wt > 0.0f) {
    o[0] = make_float4(p.x, p.y, p.z, wt);
    o[1] = make_float4(n.x, n.y, n.z, group);
    o[2] = make_float4(om.x, om.y, om.z, 0.0f);
  } else {
    o[0] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    o[1] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
    o[2] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
  }
}

__global__ void k_guide_records(GuideWave gw, uint32_t n_slots, uint32_t perm_mul, float4* __restrict__ out) {
  const uint64_t n_rec = 2ull * n_slots;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_slots; s += gridDim.x * blockDim.x) {
    const float4* raw = gw.raw + kRawF4 * s;
    const float4 a = raw[0], b = raw[1], c = raw[2], d = raw[3], e = raw[4], f = raw[5];
    float wt = 0.0f;
    if (d.z > 0.5f && d.y > 0.0f && c.w > 0.0f) {
      const uint32_t pid = (uint32_t)d.w;
      const float Lin = (gw.Lfinal[pid] - b.w) / d.y;
      wt = fmaxf(Lin, 0.0f) * d.x / c.w;
    }
    float ws = 0.0f;
    if (d.z > 0.5f && f.z > 0.5f && f.y > 0.0f) ws = fmaxf(f.x, 0.0f) * e.w / f.y;
    put_record(out, (uint32_t)(((uint64_t)(2u * s) * perm_mul) % n_rec), f3(a), wt, f3(b), a.w, f3(c));
    put_record(out, (uint32_t)(((uint64_t)(2u * s + 1u) * perm_mul) % n_rec), f3(a), ws, f3(b), a.w, f3(e));
  }
}

// ---------------------------------------------------------------------------
// one guided step on caller-given vertices (rt_guide_sample_step): the
// vertices become the guide queries and pending sun samples of a one-wave
// wavefront in the layout k_shade writes, k_guide_sample runs on them
// unchanged, and its outputs (continuation rays, rescaled sun samples,
// escape weights, training slots) are gathered per vertex
// ---------------------------------------------------------------------------
__global__ void k_guide_step_pack(const float4* __restrict__ v, uint32_t n, float4* __restrict__ gq,
                                  float4* __restrict__ sq) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 a = v[4 * i], b = v[4 * i + 1], c = v[4 * i + 2], d = v[4 * i + 3];
    const bool has_sun = __float_as_uint(d.x) != 0u;
    gq[3 * i] = make_float4(a.x, a.y, a.z, __uint_as_float(i | kFlagCovered));
    gq[3 * i + 1] = make_float4(b.x, b.y, b.z, a.w);
    gq[3 * i + 2] = make_float4(b.w, __uint_as_float(has_sun ? i : 0xFFFFFFFFu), 0.0f, 0.0f);
    sq[2 * i] = make_float4(a.x, a.y, a.z, __uint_as_float(i));
    sq[2 * i + 1] = c;
  }
}

__global__ void k_guide_step_gather(const float4* __restrict__ v, uint32_t n, uint32_t k, const Counters* cnt,
                                    const float4* __restrict__ qout, const float4* __restrict__ sq,
                                    const float* __restrict__ wesc, const float4* __restrict__ raw,
                                    float4* __restrict__ out) {
  const uint32_t n_cont = min(cnt[k + 1].q_count, n);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4* r = raw + kRawF4 * i;
    const float4 c = r[2], d = r[3];
    const bool has_sun = __float_as_uint(v[4 * i + 3].x) != 0u;
    out[3 * i] = make_float4(c.x, c.y, c.z, c.w);
    out[3 * i + 1] = make_float4(d.x, 0.0f, has_sun ? sq[2 * i + 1].w : 0.0f, 0.0f);
    out[3 * i + 2] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
  __syncthreads();
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n_cont; j += gridDim.x * blockDim.x) {
    const float4 r0 = qout[2 * j], r1 = qout[2 * j + 1];
    const uint32_t pid = __float_as_uint(r0.w) & kPidMask;
    if (pid < n) {
      float* o = (float*)(out + 3 * pid);
      o[5] = r1.w;
      o[7] = wesc[pid];
      ((uint32_t*)o)[8] = 1u;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
size_t guide_eval_smem() { return kWPack + 2 * kATileB + 64; }
size_t guide_train_smem() { return kTrainSmem; }
uint32_t guide_wsize() { return kWSize; }
uint32_t guide_wpack_bytes() { return kWPack; }

void launch_guide_init(float* grid, uint64_t n_grid, float* W, uint64_t seed, cudaStream_t st) {
  k_guide_init<<<512, 256, 0, st>>>(grid, n_grid, W, (uint32_t)seed, (uint32_t)(seed >> 32));
}

void launch_guide_pack(const float* W, void* pack, cudaStream_t st) {
  k_pack_weights<<<16, 256, 0, st>>>(W, (unsigned char*)pack);
}

void launch_guide_eval(const GuideDev& g, const void* pack, const float* rec, uint64_t n, float* Y, float* q,
                       uint32_t* status, int sms, cudaStream_t st) {
  const size_t smem = guide_eval_smem();
  cudaFuncSetAttribute(k_guide_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const uint64_t tiles = (n + kRows - 1) / kRows;
  uint64_t grid = (uint64_t)sms * 2;
  if (grid > tiles) grid = tiles;
  if (grid == 0) return;
  k_guide_eval<<<(unsigned)grid, kRows, smem, st>>>(g, (const uint4*)pack, (const float4*)rec, n, Y, q, status);
}

void launch_guide_train(const GuideDev& g, const void* pack, const float* rec, uint64_t n, float* wsum, float* dW,
                        float* dWpart, float* dgrid, float* loss, uint32_t* status, int sms, cudaStream_t st) {
  cudaMemsetAsync(wsum, 0, sizeof(float), st);
  k_weight_sum<<<sms * 4, 256, 0, st>>>((const float4*)rec, n, wsum);
  const size_t smem = guide_train_smem();
  cudaFuncSetAttribute(k_guide_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const uint64_t tiles = (n + kRows - 1) / kRows;
  uint64_t grid = (uint64_t)sms;
  if (grid > tiles) grid = tiles;
  if (grid == 0) return;
  k_guide_train<<<(unsigned)grid, kTrainThreads, smem, st>>>(g, (const uint4*)pack, (const float4*)rec, n, wsum, dWpart,
                                                             dgrid, loss, status);
  k_dw_reduce<<<(kWSize + 31) / 32, 256, 0, st>>>(dWpart, (int)grid, dW);
}

void launch_adam(float* p, const float* g, float* m, float* v, uint64_t n, float lr, float b1, float b2, float eps,
                 float c1, float c2, cudaStream_t st) {
  k_adam<<<1024, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
}

void launch_guide_sample(const GuideDev& g, const void* pack, const DevSpectra& P, const WaveParams& w, uint32_t k,
                         const GuideWave& gw, const WaveBufs& b, double* accum, const Probe& probe, bool record,
                         int sms, cudaStream_t st) {
  if (gw.perm) {
    cudaMemsetAsync(gw.bins, 0, kGuideSortBins * sizeof(uint32_t), st);
    k_gsort_hist<<<sms * 8, 256, 0, st>>>(g, gw, b.cnt, k, b.cap);
    launch_cell_scan(gw.bins, st);
    k_gsort_scatter<<<sms * 8, 256, 0, st>>>(gw, b.cnt, k, b.cap);
  }
  cudaFuncSetAttribute(k_guide_sample, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSampleSmem);
  k_guide_sample<<<sms * kSampleCtasPerSm, kSampleThreads, kSampleSmem, st>>>(g, (const uint4*)pack, P, w, k, gw, b.q[(k + 1) & 1], b.sq, b.L,
                                                      b.sig, b.cnt, b.cap, accum, probe, record, b.status);
}

void launch_guide_step_pack(const void* v, uint32_t n, float4* gq, float4* sq, cudaStream_t st) {
  k_guide_step_pack<<<256, 256, 0, st>>>((const float4*)v, n, gq, sq);
}

void launch_guide_step_gather(const void* v, uint32_t n, uint32_t k, const GuideWave& gw, const WaveBufs& b, void* out,
                              cudaStream_t st) {
  // one block: the per-vertex fields are written before the continuations scatter theirs
  k_guide_step_gather<<<1, 1024, 0, st>>>((const float4*)v, n, k, b.cnt, b.q[(k + 1) & 1], b.sq, gw.wesc, gw.raw,
                                          (float4*)out);
}

void launch_guide_records(const GuideWave& gw, uint32_t n_slots, uint32_t perm_mul, float* train_rec, cudaStream_t st) {
  k_guide_records<<<1024, 256, 0, st>>>(gw, n_slots, perm_mul, (float4*)train_rec);
}

}  // namespace srt

// Spectrum -> CIE XYZ contraction (section 6: colorimetry from spectra).
//
//   xyz[p][c] = sum_j (spectral[p][j] / spp) * w[j][c]
//
// RT_XYZ_BF16X3 / RT_XYZ_BF16: 5th-generation tensor cores (tcgen05.mma,
// accumulator in tensor memory).  One CTA (128 threads) processes tiles of
// 128 pixels: the FP64 rows are streamed from HBM with coalesced 16-byte
// loads, rounded to FP32 (integer operations on the IEEE fields), scaled by
// 1/spp and split into BF16 terms v = hi + mid + lo (each the BF16 rounding of
// the remainder), written to shared memory in the K-major, non-swizzled
// canonical layout (8 x 16-byte core matrices).
// One thread issues D[128 x 16] += A[128 x 16] B[16 x 16]
// for every 16-band slice: with the three-term split of both operands the six
// products hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid carry FP32-level
// accuracy (the dropped terms are below 2^-26 relative, after Henry, Tang and
// Heinecke, ARITH 2019); RT_XYZ_BF16 uses hi.hi only.  The FP32 accumulator is
// read back with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = pixels).
//
// RT_XYZ_FP64: CUDA cores, FP64, the reference mode.
#include <cstdint>

#include "rt_internal.h"
#include "rt_tc.cuh"

namespace srt {

namespace {

// ---------------------------------------------------------------------------
// FP64 reference kernel
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_xyz_fp64(const double* __restrict__ s, uint64_t np, uint32_t bc,
                                                  const float* __restrict__ w, double inv_spp, float* __restrict__ xyz) {
  extern __shared__ double tile[];  // [blockDim][bc]
  const uint64_t p0 = (uint64_t)blockIdx.x * blockDim.x;
  const uint64_t rows = (np - p0) < blockDim.x ? (np - p0) : blockDim.x;
  const uint64_t elems = rows * bc;
  const double* src = s + p0 * bc;
  for (uint64_t e = threadIdx.x; e < elems; e += blockDim.x) tile[e] = src[e];
  __syncthreads();
  if (threadIdx.x < rows) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    const double* row = tile + (size_t)threadIdx.x * bc;
    for (uint32_t j = 0; j < bc; ++j) {
      const double v = row[j] * inv_spp;
      a0 += v * (double)w[3 * j];
      a1 += v * (double)w[3 * j + 1];
      a2 += v * (double)w[3 * j + 2];
    }
    float* o = xyz + 3 * (p0 + threadIdx.x);
    o[0] = (float)a0;
    o[1] = (float)a1;
    o[2] = (float)a2;
  }
}

// FP64 -> FP32 by integer operations on the IEEE-754 fields (this GPU's FP64
// pipe is slow; a conversion instruction per spectral value made the
// contraction compute-bound).  RN rounds to nearest even, RZ truncates.
// Values below the FP32 normal range become signed zero, values above it
// infinity.
template <bool RN>
__device__ __forceinline__ float f64_to_f32(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  const uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);  // top 23 of the 52 fraction bits
  uint32_t bits = ((uint32_t)e << 23) | m;
  if (RN) {
    const uint32_t rem = lo & 0x1FFFFFFFu;  // the 29 bits dropped
    if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) bits += 1u;  // a carry moves into the exponent
  }
  return __uint_as_float(sign | bits);
}

// FP64 -> FP32 truncated, from the double's two words: rebias the exponent
// inside the high word, then one funnel shift joins its 20 fraction bits with
// the top 3 of the low word.  Magnitudes below the FP32 normal range (zero
// included) give signed zero; the spectral sums never exceed its range.
__device__ __forceinline__ float f64_to_f32_rz(uint32_t lo, uint32_t hi) {
  const uint32_t t = (hi & 0x7FFFFFFFu) - (896u << 20);  // exponent 1023 -> 127
  const uint32_t bits = __funnelshift_l(lo, t, 3);       // (t << 3) | (lo >> 29)
  const uint32_t sign = hi & 0x80000000u;
  return __uint_as_float(((hi >> 20) & 0x7FFu) > 896u ? (bits | sign) : sign);
}

// v = hi + mid + lo exactly, each term a BF16 value: hi keeps the top 8
// significant bits of v (truncation), mid the top 8 of the remainder, lo the
// rest (at most 8 bits, exact).  Returned as the BF16 bit patterns in the
// upper halves of three words.
__device__ __forceinline__ void split3_trunc(float v, uint32_t& h, uint32_t& m, uint32_t& l) {
  h = __float_as_uint(v) & 0xFFFF0000u;
  const float r1 = v - __uint_as_float(h);
  m = __float_as_uint(r1) & 0xFFFF0000u;
  l = __float_as_uint(r1 - __uint_as_float(m));
}

constexpr int kTileM = 128;        // pixels per tile = MMA M = TMEM lanes
constexpr int kMmaN = 16;          // XYZ padded to 16 columns
constexpr int kTmemCols = 32;      // smallest TMEM allocation
constexpr uint32_t kATile = 4096;  // one 128 x 16 BF16 K-slice
constexpr uint32_t kBTile = 512;   // one 16 x 16 BF16 K-slice
constexpr uint32_t kIdesc = tc_idesc_bf16(kTileM, kMmaN);

constexpr int kXyzThreads = 256;
constexpr int kUnroll = 8;

// inv_bc = ceil(2^32 / bc): __umulhi(e, inv_bc) == e / bc for every element
// index of a tile (e < 128 * 192).
__global__ void __launch_bounds__(kXyzThreads) k_xyz_tc(const double* __restrict__ s, uint64_t np, uint32_t bc,
                                                        uint32_t nk, uint32_t inv_bc, const float* __restrict__ w,
                                                        double inv_spp, float* __restrict__ xyz, int n_split,
                                                        uint32_t* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* A = smem;                                   // [3][nk][4096]
  unsigned char* Bm = smem + 3u * nk * kATile;               // [3][nk][512]
  uint64_t* mbar = (uint64_t*)(Bm + 3u * nk * kBTile);
  uint32_t* tslot = (uint32_t*)(mbar + 1);
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;

  // zero A (its padded K columns stay zero) and build the split weights
  for (uint32_t i = tid; i < 3u * nk * kATile / 16u; i += blockDim.x) ((uint4*)A)[i] = make_uint4(0, 0, 0, 0);
  for (uint32_t i = tid; i < (uint32_t)kMmaN * nk * 16u; i += blockDim.x) {
    const uint32_t n = i / (nk * 16u), k = i - n * nk * 16u;
    const float v = (n < 3u && k < bc) ? w[3u * k + n] : 0.0f;
    uint16_t h, m, l;
    tc_split3(v, h, m, l);
    const uint32_t off = (k >> 4) * kBTile + tc_kmajor_off(n, k & 15u);
    *(uint16_t*)(Bm + off) = h;
    *(uint16_t*)(Bm + nk * kBTile + off) = m;
    *(uint16_t*)(Bm + 2u * nk * kBTile + off) = l;
  }
  if (tid == 0) {
    tc_mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc_tmem_alloc(tslot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // products (a split, b split)
  const uint32_t pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
  const uint64_t ntiles = (np + kTileM - 1) / kTileM;
  const float inv_spp_f = (float)inv_spp;
  uint32_t phase = 0;
  bool ok = true;
  for (uint64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const uint64_t p0 = tile * kTileM;
    const uint32_t rows = (uint32_t)((np - p0) < (uint64_t)kTileM ? (np - p0) : (uint64_t)kTileM);
    const uint32_t nel = rows * bc;
    const double* src = s + p0 * bc;
    // coalesced 16-byte loads over the tile's contiguous rows, kUnroll in
    // flight per thread before any conversion
    const uint32_t npair = (nel + 1u) >> 1;
    for (uint32_t q0 = tid; q0 < npair; q0 += blockDim.x * kUnroll) {
      double2 v[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const uint32_t q = q0 + (uint32_t)u * blockDim.x;
        if (2u * q + 1u < nel) {
          v[u] = __ldcs((const double2*)src + q);
        } else if (2u * q < nel) {
          v[u] = make_double2(__ldcs(src + 2u * q), 0.0);
        } else {
          v[u] = make_double2(0.0, 0.0);
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const uint32_t q = q0 + (uint32_t)u * blockDim.x;
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const uint32_t ee = 2u * q + (uint32_t)h2;
          if (ee < nel) {
            const uint32_t r = __umulhi(ee, inv_bc), k = ee - r * bc;
            const float val = f64_to_f32<true>(h2 ? v[u].y : v[u].x) * inv_spp_f;
            uint16_t hh, mm, ll;
            tc_split3(val, hh, mm, ll);
            const uint32_t off = (k >> 4) * kATile + tc_kmajor_off(r, k & 15u);
            *(uint16_t*)(A + off) = hh;
            if (n_split > 1) {
              *(uint16_t*)(A + nk * kATile + off) = mm;
              *(uint16_t*)(A + 2u * nk * kATile + off) = ll;
            }
          }
        }
      }
    }
    tc_fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const int nprod = n_split > 1 ? 6 : 1;
      uint32_t acc = 0;
      for (uint32_t kb = 0; kb < nk; ++kb)
        for (int pr = 0; pr < nprod; ++pr) {
          const uint64_t da = tc_smem_desc(smem_u32(A + pa[pr] * nk * kATile + kb * kATile));
          const uint64_t db = tc_smem_desc(smem_u32(Bm + pb[pr] * nk * kBTile + kb * kBTile));
          tc_mma_bf16(tmem, da, db, kIdesc, acc);
          acc = 1;
        }
      tc_commit(mbar);
    }
    const int timed_out = __syncthreads_or(tc_mbar_wait(mbar, phase, 1u << 24) ? 0 : 1);
    if (timed_out) {
      if (tid == 0) atomicOr(status, ST_ITER);
      ok = false;
    }
    phase ^= 1u;
    tc_fence_after();
    if (warp < 4) {  // warp w reads TMEM lanes 32w..32w+31 (pixels)
      float x, y, z, pad;
      tc_tmem_ld4(tmem + ((warp * 32u) << 16), x, y, z, pad);
      const uint32_t r = warp * 32u + lane;
      if (ok && r < rows) {
        float* o = xyz + 3 * (p0 + r);
        o[0] = x;
        o[1] = y;
        o[2] = z;
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  tc_fence_after();
  if (warp == 0) tc_tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// TMA-pipelined variant (the default when it fits in shared memory): a tile of
// 128 pixels arrives as two halves of 64 rows, each one bulk copy (the rows
// are contiguous) into its own shared buffer, completion counted on an
// mbarrier.  Each half is converted (divide by spp, FP32, three-term BF16
// split, 16-byte stores of 8 K-consecutive values into the canonical layout)
// as soon as it lands, and the copy of the same half of the CTA's next tile is
// issued as soon as the buffer is read, so HBM traffic overlaps conversion,
// MMA and epilogue.  A tail tile whose halves are not full is read with
// plain loads.
// ---------------------------------------------------------------------------
constexpr uint32_t kHalf = 64;

__device__ __forceinline__ bool half_full(uint64_t tile, uint32_t h, uint64_t np) {
  return tile * kTileM + (uint64_t)(h + 1) * kHalf <= np;
}

constexpr int kXyzTmaThreads = 512;

__global__ void __launch_bounds__(kXyzTmaThreads, 1) k_xyz_tma(const double* __restrict__ s, uint64_t np, uint32_t bc,
                                                            uint32_t nk, const float* __restrict__ w, double inv_spp,
                                                            float* __restrict__ xyz, int n_split, uint32_t* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const uint32_t half_bytes = kHalf * bc * 8u;  // a multiple of 512
  unsigned char* raw0 = smem;
  unsigned char* A = smem + 2u * half_bytes;
  unsigned char* Bm = A + 3u * nk * kATile;
  uint64_t* mb = (uint64_t*)(Bm + 3u * nk * kBTile);  // [0], [1]: raw halves, [2]: MMA
  uint32_t* tslot = (uint32_t*)(mb + 3);
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
  for (uint32_t i = tid; i < 3u * nk * kATile / 16u; i += blockDim.x) ((uint4*)A)[i] = make_uint4(0, 0, 0, 0);
  for (uint32_t i = tid; i < (uint32_t)kMmaN * nk * 16u; i += blockDim.x) {
    const uint32_t n = i / (nk * 16u), k = i - n * nk * 16u;
    const float v = (n < 3u && k < bc) ? w[3u * k + n] : 0.0f;
    uint16_t h, m, l;
    tc_split3(v, h, m, l);
    const uint32_t off = (k >> 4) * kBTile + tc_kmajor_off(n, k & 15u);
    *(uint16_t*)(Bm + off) = h;
    *(uint16_t*)(Bm + nk * kBTile + off) = m;
    *(uint16_t*)(Bm + 2u * nk * kBTile + off) = l;
  }
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) tc_mbar_init(mb + i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc_tmem_alloc(tslot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint64_t ntiles = (np + kTileM - 1) / kTileM;
  const float inv_spp_f = (float)inv_spp;
  auto issue = [&](uint64_t tile, uint32_t h) {
    tc_mbar_expect_tx(mb + h, half_bytes);
    tc_bulk_g2s(raw0 + h * half_bytes, s + (tile * kTileM + h * kHalf) * bc, half_bytes, mb + h);
  };
  // every thread tracks which halves have a copy in flight (the conditions
  // are the same in all threads; thread 0 issues)
  bool inflight[2] = {false, false};
  if ((uint64_t)blockIdx.x < ntiles)
    for (uint32_t h = 0; h < 2u; ++h)
      if (half_full(blockIdx.x, h, np)) {
        inflight[h] = true;
        if (tid == 0) issue(blockIdx.x, h);
      }
  const uint32_t pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
  uint32_t ph[2] = {0u, 0u}, phm = 0u;
  bool ok = true;
  for (uint64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const uint64_t p0 = tile * kTileM;
    const uint32_t rows = (uint32_t)((np - p0) < (uint64_t)kTileM ? (np - p0) : (uint64_t)kTileM);
    for (uint32_t h = 0; h < 2u && ok; ++h) {
      unsigned char* raw = raw0 + h * half_bytes;
      const uint32_t rh = rows > h * kHalf ? min(rows - h * kHalf, kHalf) : 0u;
      if (half_full(tile, h, np)) {
        const int bad = __syncthreads_or(tc_mbar_wait(mb + h, ph[h], 1u << 24) ? 0 : 1);
        if (bad) {
          if (tid == 0) atomicOr(status, ST_ITER);
          ok = false;
          break;
        }
        ph[h] ^= 1u;
        inflight[h] = false;
      } else {
        const double* src = s + (p0 + h * kHalf) * bc;
        for (uint32_t e = tid; e < rh * bc; e += blockDim.x) ((double*)raw)[e] = src[e];
        __syncthreads();
      }
      // (row, group of 8 K values) items, rows fastest
      const uint32_t items = kHalf * 2u * nk;
      for (uint32_t it = tid; it < items; it += blockDim.x) {
        const uint32_t r = it % kHalf, g8 = it / kHalf;
        uint32_t hb[8], mb_[8], lb[8];
        const double* rowp = (const double*)raw + r * bc + 8u * g8;
        if (r < rh && 8u * g8 + 8u <= bc) {
          // full group: no bounds checks
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const uint2 wv = *(const uint2*)(rowp + e);
            const float v = f64_to_f32_rz(wv.x, wv.y) * inv_spp_f;
            if (n_split > 1) {
              split3_trunc(v, hb[e], mb_[e], lb[e]);
            } else {
              const uint32_t u = __float_as_uint(v);
              hb[e] = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;  // BF16, round to nearest even
            }
          }
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const uint32_t j = 8u * g8 + (uint32_t)e;
            float v = 0.0f;
            if (r < rh && j < bc) {
              const uint2 wv = *(const uint2*)(rowp + e);
              v = f64_to_f32_rz(wv.x, wv.y) * inv_spp_f;
            }
            if (n_split > 1) {
              split3_trunc(v, hb[e], mb_[e], lb[e]);
            } else {
              const uint32_t u = __float_as_uint(v);
              hb[e] = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
            }
          }
        }
        // pairs of upper halves into words, the first value in the low half
        const uint32_t off = (g8 >> 1) * kATile + tc_kmajor_off(h * kHalf + r, (g8 & 1u) * 8u);
        *(uint4*)(A + off) = make_uint4(__byte_perm(hb[0], hb[1], 0x7632), __byte_perm(hb[2], hb[3], 0x7632),
                                        __byte_perm(hb[4], hb[5], 0x7632), __byte_perm(hb[6], hb[7], 0x7632));
        if (n_split > 1) {
          *(uint4*)(A + nk * kATile + off) =
              make_uint4(__byte_perm(mb_[0], mb_[1], 0x7632), __byte_perm(mb_[2], mb_[3], 0x7632),
                         __byte_perm(mb_[4], mb_[5], 0x7632), __byte_perm(mb_[6], mb_[7], 0x7632));
          *(uint4*)(A + 2u * nk * kATile + off) =
              make_uint4(__byte_perm(lb[0], lb[1], 0x7632), __byte_perm(lb[2], lb[3], 0x7632),
                         __byte_perm(lb[4], lb[5], 0x7632), __byte_perm(lb[6], lb[7], 0x7632));
        }
      }
      // the buffer is read: refill it with the same half of the next tile
      __syncthreads();
      const uint64_t next = tile + gridDim.x;
      if (next < ntiles && half_full(next, h, np)) {
        inflight[h] = true;
        if (tid == 0) {
          tc_fence_async_smem();
          issue(next, h);
        }
      }
    }
    if (!ok) break;
    tc_fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const int nprod = n_split > 1 ? 6 : 1;
      uint32_t acc = 0;
      for (uint32_t kb = 0; kb < nk; ++kb)
        for (int pr = 0; pr < nprod; ++pr) {
          const uint64_t da = tc_smem_desc(smem_u32(A + pa[pr] * nk * kATile + kb * kATile));
          const uint64_t db = tc_smem_desc(smem_u32(Bm + pb[pr] * nk * kBTile + kb * kBTile));
          tc_mma_bf16(tmem, da, db, kIdesc, acc);
          acc = 1;
        }
      tc_commit(mb + 2);
    }
    const int timed_out = __syncthreads_or(tc_mbar_wait(mb + 2, phm, 1u << 24) ? 0 : 1);
    phm ^= 1u;
    if (timed_out) {
      if (tid == 0) atomicOr(status, ST_ITER);
      ok = false;
    }
    tc_fence_after();
    if (warp < 4) {  // warp w reads TMEM lanes 32w..32w+31 (pixels)
      float x, y, z, pad;
      tc_tmem_ld4(tmem + ((warp * 32u) << 16), x, y, z, pad);
      const uint32_t r = warp * 32u + lane;
      if (ok && r < rows) {
        float* o = xyz + 3 * (p0 + r);
        o[0] = x;
        o[1] = y;
        o[2] = z;
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  // after an early exit, wait (bounded) for the copies still in flight
  if (!ok && tid == 0)
    for (uint32_t h = 0; h < 2u; ++h)
      if (inflight[h]) tc_mbar_wait(mb + h, ph[h], 1u << 24);
  tc_fence_after();
  if (warp == 0) tc_tmem_dealloc(tmem, kTmemCols);
}

size_t xyz_tma_smem(uint32_t band_count) {
  const uint32_t nk = (band_count + 15) / 16;
  return 2ull * kHalf * band_count * 8ull + 3ull * nk * kATile + 3ull * nk * kBTile + 64;
}

}  // namespace

size_t xyz_tc_smem(uint32_t band_count) {
  const uint32_t nk = (band_count + 15) / 16;
  return 3ull * nk * kATile + 3ull * nk * kBTile + 16;
}

void launch_xyz(const double* spectral, uint64_t n_pixels, const XyzWeights& w, uint32_t spp, int mode, float* xyz,
                cudaStream_t st, uint32_t* status, int sms) {
  if (n_pixels == 0) return;
  if (mode == 2) {
    int block = (int)(49152 / (8 * (size_t)w.band_count));
    block = block > 256 ? 256 : (block < 1 ? 1 : block);
    const uint64_t grid = (n_pixels + block - 1) / block;
    const size_t smem = (size_t)block * w.band_count * sizeof(double);
    k_xyz_fp64<<<(unsigned)grid, block, smem, st>>>(spectral, n_pixels, w.band_count, w.w32, 1.0 / (double)spp, xyz);
    return;
  }
  const uint32_t nk = (w.band_count + 15) / 16;
  const size_t tsmem = xyz_tma_smem(w.band_count);
  if (tsmem <= 227u * 1024u && ((uintptr_t)spectral & 15u) == 0) {
    cudaFuncSetAttribute(k_xyz_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem);
    const uint64_t ntiles = (n_pixels + kTileM - 1) / kTileM;
    uint64_t grid = (uint64_t)sms;
    if (grid > ntiles) grid = ntiles;
    k_xyz_tma<<<(unsigned)grid, kXyzTmaThreads, tsmem, st>>>(spectral, n_pixels, w.band_count, nk, w.w32,
                                                         1.0 / (double)spp, xyz, mode == 0 ? 3 : 1, status);
    return;
  }
  const size_t smem = xyz_tc_smem(w.band_count);
  cudaFuncSetAttribute(k_xyz_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const uint64_t ntiles = (n_pixels + kTileM - 1) / kTileM;
  int per_sm = (int)((227u * 1024u) / (smem + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > ntiles) grid = ntiles;
  const uint32_t inv_bc = (uint32_t)((0x100000000ull + w.band_count - 1) / w.band_count);
  k_xyz_tc<<<(unsigned)grid, kXyzThreads, smem, st>>>(spectral, n_pixels, w.band_count, nk, inv_bc, w.w32,
                                                      1.0 / (double)spp, xyz, mode == 0 ? 3 : 1, status);
}

}  // namespace srt

// Device-side building blocks of the spectral path tracer (sm_103a).
//
// FP32 geometry and optics; every formula is the paper's physics (section 3,
// Eq. 1 complex index; section 4, Eqs. 2-3) written for the GPU.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rt_internal.h"

namespace srt {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011).  Counter layout of the
// renderer: (global pixel, sample, band, 4 * vertex + call), key = seed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    if (i) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// top 24 bits -> [0, 1), exact in float
__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-8f; }

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 add(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 mul(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 madd(float3 p, float s, float3 d) {
  return make_float3(fmaf(s, d.x, p.x), fmaf(s, d.y, p.y), fmaf(s, d.z, p.z));
}
__device__ __forceinline__ float3 neg(float3 a) { return make_float3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float comp(float3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

// Orthonormal basis around a unit vector (Duff et al., "Building an
// orthonormal basis, revisited", JCGT 6(1), 2017).
__device__ __forceinline__ void onb(float3 n, float3& t1, float3& t2) {
  const float sign = copysignf(1.0f, n.z);
  const float a = -1.0f / (sign + n.z);
  const float b = n.x * n.y * a;
  t1 = make_float3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
  t2 = make_float3(b, sign + n.y * n.y * a, -n.y);
}

// ---------------------------------------------------------------------------
// optics, FP32
// ---------------------------------------------------------------------------

// Principal square root of zr + i zi, computed from the larger part first so
// that a tiny imaginary part is not lost to cancellation.
__device__ __forceinline__ void csqrt_principal(float zr, float zi, float& sr, float& si) {
  const float m = sqrtf(fmaf(zr, zr, zi * zi));
  if (zr >= 0.0f) {
    sr = sqrtf(0.5f * (m + zr));
    si = (sr > 0.0f) ? zi / (2.0f * sr) : 0.0f;
  } else {
    si = copysignf(sqrtf(0.5f * (m - zr)), zi);
    sr = fabsf(zi) / (2.0f * fabsf(si));
  }
}

// Unpolarised Fresnel reflectance from air into eta = n + i k (Eq. 1) at
// cos(theta_i) = c: s and p amplitude ratios with the complex cosine of the
// refracted angle, cos_t = sqrt(1 - sin^2 / eta^2).
__device__ __forceinline__ float fresnel_complex(float c, float n, float k) {
  const float s2 = fmaxf(0.0f, (1.0f - c) * (1.0f + c));
  const float er = (n - k) * (n + k), ei = 2.0f * n * k;  // eta^2
  const float inv = 1.0f / fmaf(er, er, ei * ei);
  const float zr = 1.0f - s2 * er * inv, zi = s2 * ei * inv;
  float ctr, cti;
  csqrt_principal(zr, zi, ctr, cti);
  // eta * cos_t
  const float pr = n * ctr - k * cti, pi = n * cti + k * ctr;
  const float rs = (((c - pr) * (c - pr)) + pi * pi) / (((c + pr) * (c + pr)) + pi * pi);
  // r_p = (eta c - cos_t) / (eta c + cos_t)
  const float ar = n * c - ctr, ai = k * c - cti;
  const float br = n * c + ctr, bi = k * c + cti;
  const float rp = (ar * ar + ai * ai) / (br * br + bi * bi);
  return 0.5f * (rs + rp);
}

// Thin sheet: faces reflect R, the interior transmits Ti = exp(-alpha d /
// cos_t) with alpha d = 4 pi k d / lambda precomputed per (material, band);
// incoherent multiple reflections give R_s and T_s.
__device__ __forceinline__ void thin_sheet(float c, float n, float k, float alpha_d, float& Rs, float& Ts) {
  const float R = fresnel_complex(c, n, k);
  const float s2 = fmaxf(0.0f, (1.0f - c) * (1.0f + c));
  const float ct = sqrtf(fmaxf(0.0f, 1.0f - s2 / (n * n)));
  const float Ti = expf(-alpha_d / ct);
  const float RT = R * Ti;
  const float den = 1.0f / (1.0f - RT * RT);
  const float omr2 = (1.0f - R) * (1.0f - R);
  Rs = R + omr2 * R * Ti * Ti * den;
  Ts = omr2 * Ti * den;
}

// ---------------------------------------------------------------------------
// Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2(1), 2013).  The
// edge functions are formed without FMA contraction so that the two
// triangles of a shared edge compute exactly opposite values; an edge value
// of exactly zero counts as inside.
// ---------------------------------------------------------------------------
struct RayW {
  float3 o;
  int kx, ky, kz;
  float Sx, Sy, Sz;
};

__device__ __forceinline__ RayW ray_prep(float3 o, float3 d) {
  RayW r;
  r.o = o;
  const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  r.kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
  r.kx = r.kz == 2 ? 0 : r.kz + 1;
  r.ky = r.kx == 2 ? 0 : r.kx + 1;
  const float dz = comp(d, r.kz);
  if (dz < 0.0f) {
    const int t = r.kx;
    r.kx = r.ky;
    r.ky = t;
  }
  r.Sx = __fdiv_rn(comp(d, r.kx), dz);
  r.Sy = __fdiv_rn(comp(d, r.ky), dz);
  r.Sz = __fdiv_rn(1.0f, dz);
  return r;
}

// returns t (> 0) or -1
__device__ __forceinline__ float tri_hit(const RayW& r, float3 va, float3 vb, float3 vc) {
  const float3 A = sub(va, r.o), B = sub(vb, r.o), C = sub(vc, r.o);
  const float Akz = comp(A, r.kz), Bkz = comp(B, r.kz), Ckz = comp(C, r.kz);
  const float Ax = __fsub_rn(comp(A, r.kx), __fmul_rn(r.Sx, Akz));
  const float Ay = __fsub_rn(comp(A, r.ky), __fmul_rn(r.Sy, Akz));
  const float Bx = __fsub_rn(comp(B, r.kx), __fmul_rn(r.Sx, Bkz));
  const float By = __fsub_rn(comp(B, r.ky), __fmul_rn(r.Sy, Bkz));
  const float Cx = __fsub_rn(comp(C, r.kx), __fmul_rn(r.Sx, Ckz));
  const float Cy = __fsub_rn(comp(C, r.ky), __fmul_rn(r.Sy, Ckz));
  const float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  const float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  const float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return -1.0f;
  const float det = U + V + W;
  if (det == 0.0f) return -1.0f;
  const float T = U * (r.Sz * Akz) + V * (r.Sz * Bkz) + W * (r.Sz * Ckz);
  const float t = __fdiv_rn(T, det);
  return t > 0.0f ? t : -1.0f;
}

// ---------------------------------------------------------------------------
// wavefront helpers shared by the path and guide kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t mix_sig(uint32_t h, uint32_t v) { return (h ^ v) * 16777619u; }

__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }

// Two adjacent float4 (32 bytes, 32-byte aligned) in one read-only 256-bit
// load (sm_100 and later).
__device__ __forceinline__ void ldg8(const float4* p, float4& a, float4& b) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}

// Warp-aggregated append of one element per lane with want = true; every lane
// of the warp must call it (converged).  Returns the slot of this lane.
__device__ __forceinline__ uint32_t warp_append(uint32_t* counter, bool want) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t mask = __ballot_sync(0xffffffffu, want);
  uint32_t base = 0;
  const int leader = __ffs(mask) - 1;
  if (mask != 0u && (int)lane == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader < 0 ? 0 : leader);
  return base + (uint32_t)__popc(mask & ((1u << lane) - 1u));
}

// Path identity from the wave-local id: in-sample index r, sample s,
// pixel, band index j.
struct PathId {
  uint32_t r, s, pix, j;
};

__device__ __forceinline__ PathId path_id(const WaveParams& w, uint32_t pid) {
  PathId p;
  p.r = w.r0 + pid;
  p.s = w.s0;
  if (p.r >= w.PB) {
    p.r -= w.PB;
    p.s += 1;
  }
  p.pix = p.r / w.band_count;
  p.j = p.r - p.pix * w.band_count;
  return p;
}

__device__ __forceinline__ void finalize(const WaveParams& w, const PathId& id, float L, uint32_t sg, double* accum,
                                         const Probe& probe, bool record) {
  if (L != 0.0f) accum[(size_t)id.pix * w.acc_stride + w.acc_off + id.j] += (double)L;
  if (record && probe.map != nullptr) {
    const uint32_t slot = probe.map[id.pix];
    if (slot != 0xFFFFFFFFu) {
      const size_t q = ((size_t)slot * w.spp + (id.s - w.s_base)) * w.acc_stride + w.acc_off + id.j;
      probe.L[q] = L;
      probe.sig[q] = sg;
    }
  }
}

// Bands carried by four-band path unit j: j + q G for q = 0..3 (G =
// band_count = ceil(B / 4) units per pixel), those below B.
__device__ __forceinline__ uint32_t four_band_count(const WaveParams& w, uint32_t j) {
  return min(4u, (w.B - j + w.band_count - 1u) / w.band_count);
}

// Termination of a path that carries four bands: each existing band adds
// its radiance to its own (pixel, band) slot, as four one-band paths would.
__device__ __forceinline__ void finalize4(const WaveParams& w, const PathId& id, const float (&L)[4], uint32_t sg,
                                          double* accum, const Probe& probe, bool record) {
  const uint32_t G = w.band_count;
  const uint32_t nv = four_band_count(w, id.j);
  const size_t base = (size_t)id.pix * w.B + id.j;
#pragma unroll
  for (uint32_t q = 0; q < 4u; ++q)
    if (q < nv && L[q] != 0.0f) accum[base + q * G] += (double)L[q];
  if (record && probe.map != nullptr) {
    const uint32_t slot = probe.map[id.pix];
    if (slot != 0xFFFFFFFFu) {
      const size_t r = ((size_t)slot * w.spp + (id.s - w.s_base)) * w.B + id.j;
#pragma unroll
      for (uint32_t q = 0; q < 4u; ++q)
        if (q < nv) {
          probe.L[r + q * G] = L[q];
          probe.sig[r + q * G] = sg;
        }
    }
  }
}

}  // namespace srt

// Wavefront path-tracing kernels (sm_103a).
//
// One wave holds up to C spectral paths (view, pixel, sample, band).  For each
// vertex k = 1..depth the host enqueues three kernels:
//   k_trace  - closest hit of every queued ray (four-wide BVH by default; the
//              binary, eight-wide and 8-bit-quantised trees as options;
//              watertight FP32 test), persistent warps refilling idle lanes
//              from the queue, leaf batching;
//   k_shade  - material event at the hit (section 4: Eq. 2 by cosine sampling
//              for stone, thin-glass/conductor Fresnel events with the complex
//              index of Eq. 1), next-event estimate of the sun cone (Eq. 3),
//              continuation ray appended to the next queue;
//   k_shadow - transmittance of the sun rays (0 behind stone, product of the
//              thin-glass T_s otherwise), added to the path's radiance.
// Each path owns one output slot (pixel, band) in the wave, so the FP64
// accumulation into the spectral image needs no atomics: different samples
// of a slot are in different waves, which run in sample order.
#include <algorithm>
#include <cstdio>

#include "rt_device.cuh"

// 1: four-wide node boxes read with 256-bit loads
#ifndef SRT_NODE_LD256
#define SRT_NODE_LD256 1
#endif

namespace srt {

namespace {

// ---------------------------------------------------------------------------
// BVH traversal as a resumable per-lane state machine.  One call of a step
// function visits one interior node (both children tested, the far one
// pushed) or one leaf, then pops if needed; it returns true when the ray is
// finished.  The persistent kernels below interleave steps with refills of
// idle lanes, so a warp never waits for its longest ray with most lanes idle.
//
// FMA selects the box test: false = (plane - o) * inv (any origin); true =
// fma(plane, inv, -o * inv), valid for origins within the scene bounds
// because rt_load_scene pads every node box by 2^-22 (max |coordinate| + eps),
// which covers the rounding of o * inv; the far distance is widened by
// 1 + 2^-21 for the relative rounding of both distances.
// ---------------------------------------------------------------------------
struct Trav {
  RayW rw;
  float3 inv, oinv;
  float best_t;
  uint32_t best_id;
  int best_leaf;
  uint32_t ref, cnt;
  int sp;
  uint32_t iter;
  uint32_t oct;  // four-wide nodes: bit a set when the ray runs towards -axis a
};

template <bool FMA>
__device__ __forceinline__ float box_t(const Trav& tv, float4 lo, float4 hi, float tmax) {
  float tx0, tx1, ty0, ty1, tz0, tz1;
  if (FMA) {
    tx0 = fmaf(lo.x, tv.inv.x, -tv.oinv.x);
    tx1 = fmaf(hi.x, tv.inv.x, -tv.oinv.x);
    ty0 = fmaf(lo.y, tv.inv.y, -tv.oinv.y);
    ty1 = fmaf(hi.y, tv.inv.y, -tv.oinv.y);
    tz0 = fmaf(lo.z, tv.inv.z, -tv.oinv.z);
    tz1 = fmaf(hi.z, tv.inv.z, -tv.oinv.z);
  } else {
    // oinv holds the origin itself in this mode
    tx0 = __fmul_rn(__fsub_rn(lo.x, tv.oinv.x), tv.inv.x);
    tx1 = __fmul_rn(__fsub_rn(hi.x, tv.oinv.x), tv.inv.x);
    ty0 = __fmul_rn(__fsub_rn(lo.y, tv.oinv.y), tv.inv.y);
    ty1 = __fmul_rn(__fsub_rn(hi.y, tv.oinv.y), tv.inv.y);
    tz0 = __fmul_rn(__fsub_rn(lo.z, tv.oinv.z), tv.inv.z);
    tz1 = __fmul_rn(__fsub_rn(hi.z, tv.oinv.z), tv.inv.z);
  }
  const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
  const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
  return (tn <= tf * 1.0000005f) ? tn : -1.0f;
}

// Starts a ray; returns false if it misses the root box (finished).
template <bool FMA>
__device__ __forceinline__ bool trav_init(Trav& tv, const DevScene& S, float3 o, float3 d) {
  tv.rw = ray_prep(o, d);
  const float tiny = 1e-20f;
  tv.inv.x = 1.0f / (fabsf(d.x) > tiny ? d.x : copysignf(tiny, d.x));
  tv.inv.y = 1.0f / (fabsf(d.y) > tiny ? d.y : copysignf(tiny, d.y));
  tv.inv.z = 1.0f / (fabsf(d.z) > tiny ? d.z : copysignf(tiny, d.z));
  tv.oinv = FMA ? make_float3(o.x * tv.inv.x, o.y * tv.inv.y, o.z * tv.inv.z) : o;
  tv.best_t = INFINITY;
  tv.best_id = 0xFFFFFFFFu;
  tv.best_leaf = -1;
  tv.sp = 0;
  tv.iter = 0;
  const float4 rlo = ldg4(S.nodes + 2), rhi = ldg4(S.nodes + 3);
  tv.ref = __float_as_uint(rlo.w);
  tv.cnt = __float_as_uint(rhi.w);
  return box_t<FMA>(tv, rlo, rhi, INFINITY) >= 0.0f;
}

// Interior node: test both children of pair ref, descend into the nearer,
// push the farther.  Returns false if neither child is entered.
template <bool FMA, bool COUNT>
__device__ __forceinline__ bool trav_interior(Trav& tv, uint2* stack, const DevScene& S, float tmax, uint32_t* status,
                                              uint32_t& n_nodes) {
  const float4* c = S.nodes + 2u * tv.ref;
  const float4 alo = ldg4(c), ahi = ldg4(c + 1), blo = ldg4(c + 2), bhi = ldg4(c + 3);
  if (COUNT) n_nodes += 2;
  const float ta = box_t<FMA>(tv, alo, ahi, tmax);
  const float tb = box_t<FMA>(tv, blo, bhi, tmax);
  // branch-free: descend into the nearer entered child; the farther one is
  // written to the stack unconditionally and kept only when both are entered
  const bool ha = ta >= 0.0f, hb = tb >= 0.0f;
  const bool an = ha && (!hb || ta <= tb);
  const bool both = ha && hb;
  if (both && tv.sp >= kStack) {
    atomicOr(status, ST_STACK);
    tv.sp = 0;
    return false;
  }
  const uint32_t fref = __float_as_uint(an ? blo.w : alo.w), fcnt = __float_as_uint(an ? bhi.w : ahi.w);
  stack[min(tv.sp, kStack - 1)] = make_uint2((fref << 3) | fcnt, __float_as_uint(an ? tb : ta));
  tv.sp += both ? 1 : 0;
  tv.ref = __float_as_uint(an ? alo.w : blo.w);
  tv.cnt = __float_as_uint(an ? ahi.w : bhi.w);
  return ha || hb;
}

// Pops the next stack entry whose entry distance is within tmax; false when
// the stack is empty (traversal finished).
__device__ __forceinline__ bool trav_pop(Trav& tv, const uint2* stack, float tmax) {
  while (tv.sp > 0) {
    const uint2 e = stack[--tv.sp];
    if (__uint_as_float(e.y) <= tmax) {
      tv.ref = e.x >> 3;
      tv.cnt = e.x & 7u;
      return true;
    }
  }
  return false;
}

// ---------------------------------------------------------------------------
// Four-wide BVH (node = 8 float4: lo.x, hi.x, lo.y, hi.y, lo.z, hi.z of the
// four children, then the children packed as ref << 3 | count, then padding).  Per axis the ray's direction
// sign picks the entry plane (lo for a positive direction) and the exit
// plane, so one slab test per child needs no min/max of the plane pair and an
// empty child slot (lo = +inf, hi = -inf) is never entered.  The box test
// rounds as box_t above.
// ---------------------------------------------------------------------------
template <bool FMA>
__device__ __forceinline__ void trav_init4(Trav& tv, float3 o, float3 d) {
  tv.rw = ray_prep(o, d);
  const float tiny = 1e-20f;
  tv.inv.x = 1.0f / (fabsf(d.x) > tiny ? d.x : copysignf(tiny, d.x));
  tv.inv.y = 1.0f / (fabsf(d.y) > tiny ? d.y : copysignf(tiny, d.y));
  tv.inv.z = 1.0f / (fabsf(d.z) > tiny ? d.z : copysignf(tiny, d.z));
  tv.oinv = FMA ? make_float3(o.x * tv.inv.x, o.y * tv.inv.y, o.z * tv.inv.z) : o;
  tv.best_t = INFINITY;
  tv.best_id = 0xFFFFFFFFu;
  tv.best_leaf = -1;
  tv.sp = 0;
  tv.iter = 0;
  tv.ref = 0;
  tv.cnt = 0;
  tv.oct = (tv.inv.x < 0.0f ? 1u : 0u) | (tv.inv.y < 0.0f ? 2u : 0u) | (tv.inv.z < 0.0f ? 4u : 0u);
}

template <bool FMA>
__device__ __forceinline__ float slab(float plane, float inv, float oinv) {
  // robust mode: oinv holds the origin itself
  return FMA ? fmaf(plane, inv, -oinv) : __fmul_rn(__fsub_rn(plane, oinv), inv);
}

template <bool FMA>
__device__ __forceinline__ float child_t(const Trav& tv, float nx, float fx, float ny, float fy, float nz, float fz,
                                         float tmax) {
  const float tn = fmaxf(fmaxf(slab<FMA>(nx, tv.inv.x, tv.oinv.x), slab<FMA>(ny, tv.inv.y, tv.oinv.y)),
                         fmaxf(slab<FMA>(nz, tv.inv.z, tv.oinv.z), 0.0f));
  const float tf = fminf(fminf(slab<FMA>(fx, tv.inv.x, tv.oinv.x), slab<FMA>(fy, tv.inv.y, tv.oinv.y)),
                         fminf(slab<FMA>(fz, tv.inv.z, tv.oinv.z), tmax));
  return tn <= tf * 1.0000005f ? tn : INFINITY;
}

__device__ __forceinline__ void cswap(float& ta, uint32_t& pa, float& tb, uint32_t& pb) {
  const bool sw = tb < ta;
  const float t = sw ? tb : ta;
  const uint32_t p = sw ? pb : pa;
  tb = sw ? ta : tb;
  pb = sw ? pa : pb;
  ta = t;
  pa = p;
}

// Interior node: test the four children, descend into the nearest entered
// one and push the others, the nearer ones last (popped first); with ANY
// (sun rays, which need every crossed sheet or one opaque hit, in any order)
// visit the entered children in slot order: descend into the first and push
// the others with the next one on top.  Slot order is set by k_sun_order4
// (farthest along the sun first).  Returns false if no child is entered.
template <bool FMA, bool COUNT, bool ANY = false>
__device__ __forceinline__ bool trav_interior4(Trav& tv, uint2* stack, const DevScene& S, float tmax,
                                               uint32_t* status, uint32_t& n_nodes) {
  const float4* nd = S.nodes4 + 8u * tv.ref;
#if SRT_NODE_LD256
  // each axis's plane pair in one 256-bit load (4 instead of 7 loads per
  // node: the kernel is bound by L1 wavefronts of scattered lanes)
  float4 lx, hx, ly, hy, lz, hz;
  ldg8(nd, lx, hx);
  ldg8(nd + 2, ly, hy);
  ldg8(nd + 4, lz, hz);
  const bool sx = tv.oct & 1u, sy = tv.oct & 2u, sz = tv.oct & 4u;
  const float4 nx = sx ? hx : lx, fx = sx ? lx : hx;
  const float4 ny = sy ? hy : ly, fy = sy ? ly : hy;
  const float4 nz = sz ? hz : lz, fz = sz ? lz : hz;
#else
  const uint32_t ox = tv.oct & 1u, oy = (tv.oct >> 1) & 1u, oz = (tv.oct >> 2) & 1u;
  const float4 nx = ldg4(nd + ox), fx = ldg4(nd + (ox ^ 1u));
  const float4 ny = ldg4(nd + 2u + oy), fy = ldg4(nd + 2u + (oy ^ 1u));
  const float4 nz = ldg4(nd + 4u + oz), fz = ldg4(nd + 4u + (oz ^ 1u));
#endif
  const uint4 pk = __ldg((const uint4*)(nd + 6));  // children: ref << 3 | count
  if (COUNT) n_nodes += 4;
  float t0 = child_t<FMA>(tv, nx.x, fx.x, ny.x, fy.x, nz.x, fz.x, tmax);
  float t1 = child_t<FMA>(tv, nx.y, fx.y, ny.y, fy.y, nz.y, fz.y, tmax);
  float t2 = child_t<FMA>(tv, nx.z, fx.z, ny.z, fy.z, nz.z, fz.z, tmax);
  float t3 = child_t<FMA>(tv, nx.w, fx.w, ny.w, fy.w, nz.w, fz.w, tmax);
  uint32_t p0 = pk.x, p1 = pk.y, p2 = pk.z, p3 = pk.w;
  const int nh = (t0 < INFINITY) + (t1 < INFINITY) + (t2 < INFINITY) + (t3 < INFINITY);
  if (nh == 0) return false;
  if (ANY) {
    if (tv.sp + nh - 1 > kStack) {
      atomicOr(status, ST_STACK);
      tv.sp = 0;
      return false;
    }
    const float tt[4] = {t0, t1, t2, t3};
    const uint32_t pp[4] = {p0, p1, p2, p3};
    // entered child j >= 1 (in slot order) goes to stack[sp + nh - 1 - j]
    const int top = tv.sp + nh - 2;
    int j = -1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (tt[i] < INFINITY) {
        if (j < 0) {
          tv.ref = pp[i] >> 3;
          tv.cnt = pp[i] & 7u;
        } else {
          stack[top - j] = make_uint2(pp[i], 0u);
        }
        ++j;
      }
    }
    tv.sp += nh - 1;
    return true;
  }
  // sorting network of four (missed children, at +inf, end up last)
  cswap(t0, p0, t1, p1);
  cswap(t2, p2, t3, p3);
  cswap(t0, p0, t2, p2);
  cswap(t1, p1, t3, p3);
  cswap(t1, p1, t2, p2);
  if (tv.sp + nh - 1 > kStack) {
    atomicOr(status, ST_STACK);
    tv.sp = 0;
    return false;
  }
  // entries 1 .. nh-1 go to stack[sp + nh - 1 - j] (entry 1 on top)
  const int top = tv.sp + nh - 2;
  if (nh > 1) stack[top] = make_uint2(p1, __float_as_uint(t1));
  if (nh > 2) stack[top - 1] = make_uint2(p2, __float_as_uint(t2));
  if (nh > 3) stack[top - 2] = make_uint2(p3, __float_as_uint(t3));
  tv.sp += nh - 1;
  tv.ref = p0 >> 3;
  tv.cnt = p0 & 7u;
  return true;
}

// ---------------------------------------------------------------------------
// Four-wide BVH with 8-bit child boxes (node = 4 float4, 64 bytes: {origin,
// bits(e_x | e_y << 8 | e_z << 16)}, {lo x, hi x, lo y, hi y} and {lo z,
// hi z} as one byte per child, then the children packed as in the float
// node).  Plane q of axis a lies at origin_a + q 2^e_a; the byte becomes the
// float 2^23 + q by a byte permute, and t = fma(2^23 + q, 2^e inv,
// b - 2^23 2^e inv) with b = (origin - o) inv: the subtraction rounds by
// at most half a cell, inside the cell of margin the builder leaves around
// every child box.  Same children, same order, half the bytes per node
// visit of the float node (the closest-hit kernel is bound by L1
// throughput).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float qplane(uint32_t word, uint32_t sel) {
  return __uint_as_float(__byte_perm(word, 0x4B000000u, sel));
}

template <bool FMA>
__device__ __forceinline__ float qslab_base(float origin, float inv, float oinv) {
  return FMA ? fmaf(origin, inv, -oinv) : __fmul_rn(__fsub_rn(origin, oinv), inv);
}

template <bool FMA, bool COUNT>
__device__ __forceinline__ bool trav_interior4q(Trav& tv, uint2* stack, const DevScene& S, float tmax,
                                                uint32_t* status, uint32_t& n_nodes) {
  const float4* nd = S.nodes4q + 4u * tv.ref;
  const float4 h = ldg4(nd), pa = ldg4(nd + 1), pb = ldg4(nd + 2);
  const uint4 pk = __ldg((const uint4*)(nd + 3));
  if (COUNT) n_nodes += 4;
  const uint32_t eb = __float_as_uint(h.w);
  // per axis: cell size times 1/d, and the offset of plane 2^23 + q
  const float sx = __uint_as_float(((eb & 0xFFu) + 127u - ((eb & 0x80u) << 1)) << 23) * tv.inv.x;
  const float sy = __uint_as_float((((eb >> 8) & 0xFFu) + 127u - (((eb >> 8) & 0x80u) << 1)) << 23) * tv.inv.y;
  const float sz = __uint_as_float((((eb >> 16) & 0xFFu) + 127u - (((eb >> 16) & 0x80u) << 1)) << 23) * tv.inv.z;
  const float bx = fmaf(-8388608.0f, sx, qslab_base<FMA>(h.x, tv.inv.x, tv.oinv.x));
  const float by = fmaf(-8388608.0f, sy, qslab_base<FMA>(h.y, tv.inv.y, tv.oinv.y));
  const float bz = fmaf(-8388608.0f, sz, qslab_base<FMA>(h.z, tv.inv.z, tv.oinv.z));
  // near planes: lo when the ray runs towards +axis
  const uint32_t wlx = __float_as_uint(pa.x), whx = __float_as_uint(pa.y);
  const uint32_t wly = __float_as_uint(pa.z), why = __float_as_uint(pa.w);
  const uint32_t wlz = __float_as_uint(pb.x), whz = __float_as_uint(pb.y);
  const uint32_t nx = (tv.oct & 1u) ? whx : wlx, fx = (tv.oct & 1u) ? wlx : whx;
  const uint32_t ny = (tv.oct & 2u) ? why : wly, fy = (tv.oct & 2u) ? wly : why;
  const uint32_t nz = (tv.oct & 4u) ? whz : wlz, fz = (tv.oct & 4u) ? wlz : whz;
  float t[4];
#pragma unroll
  for (uint32_t i = 0; i < 4; ++i) {
    const uint32_t sel = 0x7540u | i;
    const float tn = fmaxf(fmaxf(fmaf(qplane(nx, sel), sx, bx), fmaf(qplane(ny, sel), sy, by)),
                           fmaxf(fmaf(qplane(nz, sel), sz, bz), 0.0f));
    const float tf = fminf(fminf(fmaf(qplane(fx, sel), sx, bx), fmaf(qplane(fy, sel), sy, by)),
                           fminf(fmaf(qplane(fz, sel), sz, bz), tmax));
    t[i] = tn <= tf * 1.0000005f ? tn : INFINITY;
  }
  float t0 = t[0], t1 = t[1], t2 = t[2], t3 = t[3];
  uint32_t p0 = pk.x, p1 = pk.y, p2 = pk.z, p3 = pk.w;
  const int nh = (t0 < INFINITY) + (t1 < INFINITY) + (t2 < INFINITY) + (t3 < INFINITY);
  if (nh == 0) return false;
  cswap(t0, p0, t1, p1);
  cswap(t2, p2, t3, p3);
  cswap(t0, p0, t2, p2);
  cswap(t1, p1, t3, p3);
  cswap(t1, p1, t2, p2);
  if (tv.sp + nh - 1 > kStack) {
    atomicOr(status, ST_STACK);
    tv.sp = 0;
    return false;
  }
  const int top = tv.sp + nh - 2;
  if (nh > 1) stack[top] = make_uint2(p1, __float_as_uint(t1));
  if (nh > 2) stack[top - 1] = make_uint2(p2, __float_as_uint(t2));
  if (nh > 3) stack[top - 2] = make_uint2(p3, __float_as_uint(t3));
  tv.sp += nh - 1;
  tv.ref = p0 >> 3;
  tv.cnt = p0 & 7u;
  return true;
}

// ---------------------------------------------------------------------------
// Eight-wide BVH (node = 14 float4: per axis the lo planes of children 0-3
// and 4-7, then their hi planes, then the eight children packed as
// ref << 3 | count).  The builder puts in slot s the child that lies towards
// the corner ((s & 1) ? +x : -x, (s & 2) ? +y : -y, (s & 4) ? +z : -z) of the
// node, so visiting the entered children in the order s = i ^ oct meets the
// corner nearest to the ray first without a per-ray sort: the first entered
// child in that order is descended into, the others pushed with the next one
// on top.  Half a node (children 0-3, then 4-7) is tested at a time.
// ---------------------------------------------------------------------------
template <bool FMA, bool COUNT>
__device__ __forceinline__ bool trav_interior8(Trav& tv, uint2* stack, const DevScene& S, float tmax,
                                               uint32_t* status, uint32_t& n_nodes) {
  const float4* nd = S.nodes8 + 14u * tv.ref;
  const uint32_t ox = (tv.oct & 1u) << 1, oy = tv.oct & 2u, oz = (tv.oct >> 1) & 2u;
  if (COUNT) n_nodes += 8;
  float t[8];
#pragma unroll
  for (uint32_t h = 0; h < 2; ++h) {
    const float4 nx = ldg4(nd + ox + h), fx = ldg4(nd + (ox ^ 2u) + h);
    const float4 ny = ldg4(nd + 4u + oy + h), fy = ldg4(nd + 4u + (oy ^ 2u) + h);
    const float4 nz = ldg4(nd + 8u + oz + h), fz = ldg4(nd + 8u + (oz ^ 2u) + h);
    t[4 * h] = child_t<FMA>(tv, nx.x, fx.x, ny.x, fy.x, nz.x, fz.x, tmax);
    t[4 * h + 1] = child_t<FMA>(tv, nx.y, fx.y, ny.y, fy.y, nz.y, fz.y, tmax);
    t[4 * h + 2] = child_t<FMA>(tv, nx.z, fx.z, ny.z, fy.z, nz.z, fz.z, tmax);
    t[4 * h + 3] = child_t<FMA>(tv, nx.w, fx.w, ny.w, fy.w, nz.w, fz.w, tmax);
  }
  uint32_t m = 0;
#pragma unroll
  for (int s = 0; s < 8; ++s) m |= (t[s] < INFINITY ? 1u : 0u) << s;
  if (m == 0u) return false;
  const int nh = __popc(m);
  if (tv.sp + nh - 1 > kStack) {
    atomicOr(status, ST_STACK);
    tv.sp = 0;
    return false;
  }
  const uint4 pa = __ldg((const uint4*)(nd + 12)), pb = __ldg((const uint4*)(nd + 13));
  const uint32_t p[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
  // the entered slots in visit order: bit i of v is slot i ^ oct
  uint32_t v = m;
  if (tv.oct & 1u) v = ((v & 0x55u) << 1) | ((v >> 1) & 0x55u);
  if (tv.oct & 2u) v = ((v & 0x33u) << 2) | ((v >> 2) & 0x33u);
  if (tv.oct & 4u) v = ((v & 0x0Fu) << 4) | ((v >> 4) & 0x0Fu);
  // visit rank r >= 1 goes to stack[top - r], rank 1 on top
  const int top = tv.sp + nh - 1;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    if (t[s] < INFINITY) {
      const uint32_t i = (uint32_t)s ^ tv.oct;
      const int r = __popc(v & ((1u << i) - 1u));
      if (r == 0) {
        tv.ref = p[s] >> 3;
        tv.cnt = p[s] & 7u;
      } else {
        stack[top - r] = make_uint2(p[s], __float_as_uint(t[s]));
      }
    }
  }
  tv.sp += nh - 1;
  return true;
}

template <bool W4, bool FMA, bool COUNT, bool ANY = false>
__device__ __forceinline__ bool interior_w(Trav& tv, uint2* stack, const DevScene& S, float tmax, uint32_t* status,
                                           uint32_t& n_nodes) {
  return W4 ? trav_interior4<FMA, COUNT, ANY>(tv, stack, S, tmax, status, n_nodes)
            : trav_interior<FMA, COUNT>(tv, stack, S, tmax, status, n_nodes);
}

// Starts a ray; false if it misses the binary tree's root box.
template <bool W4, bool FMA>
__device__ __forceinline__ bool init_w(Trav& tv, const DevScene& S, float3 o, float3 d) {
  if (W4) {
    trav_init4<FMA>(tv, o, d);
    return true;
  }
  return trav_init<FMA>(tv, S, o, d);
}

__device__ __forceinline__ void closest_leaf(Trav& tv, const DevScene& S, uint32_t& n_tris, bool count) {
  for (uint32_t t = tv.ref; t < tv.ref + tv.cnt; ++t) {
    const float4* tr = S.tris + 3u * t;
    const float4 v0 = ldg4(tr), v1 = ldg4(tr + 1), v2 = ldg4(tr + 2);
    if (count) ++n_tris;
    const float th = tri_hit(tv.rw, f3(v0), f3(v1), f3(v2));
    const uint32_t id = __float_as_uint(v0.w);
    if (th > 0.0f && (th < tv.best_t || (th == tv.best_t && id < tv.best_id))) {
      tv.best_t = th;
      tv.best_leaf = (int)t;
      tv.best_id = id;
    }
  }
}

// One closest-hit step (t > 0; ties in t go to the lower input id).  With WW
// (Aila and Laine's while-while form) the step runs interior nodes until the
// lane reaches a leaf, then that leaf, so that a warp's lanes execute the same
// phase together.
template <bool FMA, bool COUNT, bool WW>
__device__ __forceinline__ bool closest_step(Trav& tv, uint2* stack, const DevScene& S, uint32_t cap,
                                             uint32_t* status, uint32_t& n_nodes, uint32_t& n_tris) {
  if (WW) {
    while (tv.cnt == 0u) {
      if (++tv.iter > cap) {
        atomicOr(status, ST_ITER);
        return true;
      }
      if (!trav_interior<FMA, COUNT>(tv, stack, S, tv.best_t, status, n_nodes) && !trav_pop(tv, stack, tv.best_t))
        return true;
    }
    closest_leaf(tv, S, n_tris, COUNT);
    return !trav_pop(tv, stack, tv.best_t);
  }
  if (++tv.iter > cap) {
    atomicOr(status, ST_ITER);
    return true;
  }
  if (tv.cnt == 0u) {
    if (trav_interior<FMA, COUNT>(tv, stack, S, tv.best_t, status, n_nodes)) return false;
  } else {
    closest_leaf(tv, S, n_tris, COUNT);
  }
  return !trav_pop(tv, stack, tv.best_t);
}

// Sun-ray leaf: product of thin-glass T_s over every crossed sheet; returns
// true at the first opaque triangle (T = 0, n_glass = 0xFFFFFFFF).
__device__ __forceinline__ bool shadow_leaf(Trav& tv, const DevScene& S, const DevSpectra& P, float3 d, uint32_t band,
                                            float& T, uint32_t& ng, uint32_t& n_tris, bool count) {
  for (uint32_t t = tv.ref; t < tv.ref + tv.cnt; ++t) {
    const float4* tr = S.tris + 3u * t;
    const float4 v0 = ldg4(tr), v1 = ldg4(tr + 1), v2 = ldg4(tr + 2);
    if (count) ++n_tris;
    const float th = tri_hit(tv.rw, f3(v0), f3(v1), f3(v2));
    if (th > 0.0f) {
      const uint32_t mat = __float_as_uint(v1.w);
      if (__ldg(P.mtype + mat) != 1) {
        T = 0.0f;
        ng = 0xFFFFFFFFu;
        return true;
      }
      const float4 nr = ldg4(S.nrm + t);
      const float c = fabsf(dot(d, f3(nr)));
      const float4 m = ldg4(P.mb + mat * P.n_bands + band);
      float Rs, Ts;
      thin_sheet(c, m.x, m.y, __ldg(P.ad + mat * P.n_bands + band), Rs, Ts);
      T *= Ts;
      ++ng;
    }
  }
  return false;
}

// Sun-ray leaf for a path that carries bands band0 + q G, q < nv: the
// product of thin-glass T_s per band.
__device__ __forceinline__ bool shadow_leaf4(Trav& tv, const DevScene& S, const DevSpectra& P, float3 d,
                                             uint32_t band0, uint32_t G, uint32_t nv, float (&T)[4], uint32_t& ng,
                                             uint32_t& n_tris, bool count) {
  for (uint32_t t = tv.ref; t < tv.ref + tv.cnt; ++t) {
    const float4* tr = S.tris + 3u * t;
    const float4 v0 = ldg4(tr), v1 = ldg4(tr + 1), v2 = ldg4(tr + 2);
    if (count) ++n_tris;
    const float th = tri_hit(tv.rw, f3(v0), f3(v1), f3(v2));
    if (th > 0.0f) {
      const uint32_t mat = __float_as_uint(v1.w);
      if (__ldg(P.mtype + mat) != 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q) T[q] = 0.0f;
        ng = 0xFFFFFFFFu;
        return true;
      }
      const float4 nr = ldg4(S.nrm + t);
      const float c = fabsf(dot(d, f3(nr)));
#pragma unroll
      for (uint32_t q = 0; q < 4u; ++q)
        if (q < nv) {
          const uint32_t mb = mat * P.n_bands + band0 + q * G;
          const float4 m = ldg4(P.mb + mb);
          float Rs, Ts;
          thin_sheet(c, m.x, m.y, __ldg(P.ad + mb), Rs, Ts);
          T[q] *= Ts;
        }
      ++ng;
    }
  }
  return false;
}

// One sun-ray step (WW as for closest_step).
template <bool FMA, bool COUNT, bool WW>
__device__ __forceinline__ bool shadow_step(Trav& tv, uint2* stack, const DevScene& S, const DevSpectra& P, float3 d,
                                            uint32_t band, float& T, uint32_t& ng, uint32_t cap, uint32_t* status,
                                            uint32_t& n_nodes, uint32_t& n_tris) {
  if (WW) {
    while (tv.cnt == 0u) {
      if (++tv.iter > cap) {
        atomicOr(status, ST_ITER);
        return true;
      }
      if (!trav_interior<FMA, COUNT>(tv, stack, S, INFINITY, status, n_nodes) && !trav_pop(tv, stack, INFINITY))
        return true;
    }
    if (shadow_leaf(tv, S, P, d, band, T, ng, n_tris, COUNT)) return true;
    return !trav_pop(tv, stack, INFINITY);
  }
  if (++tv.iter > cap) {
    atomicOr(status, ST_ITER);
    return true;
  }
  if (tv.cnt == 0u) {
    if (trav_interior<FMA, COUNT>(tv, stack, S, INFINITY, status, n_nodes)) return false;
  } else {
    if (shadow_leaf(tv, S, P, d, band, T, ng, n_tris, COUNT)) return true;
  }
  return !trav_pop(tv, stack, INFINITY);
}

__device__ __forceinline__ uint32_t trav_cap(const DevScene& S) {
  return S.iter_cap ? S.iter_cap : 4u * S.n_nodes + 64u;
}

// Whole-ray helpers for the single-step entry points (any origin).
__device__ __forceinline__ void closest_hit(const DevScene& S, float3 o, float3 d, float& best_t, int& best_leaf,
                                            uint32_t* status) {
  Trav tv;
  uint2 stack[kStack];
  uint32_t a = 0, b = 0;
  trav_init4<false>(tv, o, d);
  const uint32_t cap = trav_cap(S);
  for (;;) {
    if (++tv.iter > cap) {
      atomicOr(status, ST_ITER);
      break;
    }
    if (tv.cnt == 0u) {
      if (trav_interior4<false, false>(tv, stack, S, tv.best_t, status, a)) continue;
    } else {
      closest_leaf(tv, S, b, false);
    }
    if (!trav_pop(tv, stack, tv.best_t)) break;
  }
  best_t = tv.best_t;
  best_leaf = tv.best_leaf;
}

__device__ __forceinline__ float shadow_T(const DevScene& S, const DevSpectra& P, float3 o, float3 d, uint32_t band,
                                          uint32_t& n_glass, uint32_t* status) {
  Trav tv;
  uint2 stack[kStack];
  uint32_t a = 0, b = 0;
  float T = 1.0f;
  uint32_t ng = 0;
  trav_init4<false>(tv, o, d);
  const uint32_t cap = trav_cap(S);
  for (;;) {
    if (++tv.iter > cap) {
      atomicOr(status, ST_ITER);
      break;
    }
    if (tv.cnt == 0u) {
      if (trav_interior4<false, false>(tv, stack, S, INFINITY, status, a)) continue;
    } else if (shadow_leaf(tv, S, P, d, band, T, ng, b, false)) {
      break;
    }
    if (!trav_pop(tv, stack, INFINITY)) break;
  }
  n_glass = ng;
  return T;
}

// Exclusive prefix sum of the bins: each block of 1024 threads scans one
// chunk of 1024 bins in place and writes the chunk total; the chunk totals
// (kCellSortBins / 1024 of them) are then scanned by one block, and the
// scatter adds the chunk's offset.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums, uint32_t& total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (uint32_t o = 1; o < 32u; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31u) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nw ? warp_sums[lane] : 0u;
#pragma unroll
    for (uint32_t o = 1; o < 32u; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) warp_sums[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  total = warp_sums[nw - 1];
  const uint32_t before = warp == 0 ? 0u : warp_sums[warp - 1];
  return before + x - v;
}

__global__ void __launch_bounds__(1024) k_cell_scan_chunks(uint32_t* __restrict__ bins, uint32_t* __restrict__ totals) {
  __shared__ uint32_t ws[32];
  const uint32_t i = blockIdx.x * 1024u + threadIdx.x;
  uint32_t tot;
  const uint32_t ex = block_exclusive_scan(bins[i], ws, tot);
  bins[i] = ex;
  if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_cell_scan_totals(uint32_t* __restrict__ totals) {
  __shared__ uint32_t ws[32];
  uint32_t tot;
  const uint32_t ex = block_exclusive_scan(totals[threadIdx.x], ws, tot);
  __syncthreads();
  totals[threadIdx.x] = ex;
}

// ---------------------------------------------------------------------------
// Cell sort of a ray queue (counting sort, 2^18 keys): vertex >= 2 rays by
// the Morton cell of their origin on a 32^3 grid over the scene box and
// their direction octant, sun rays (all nearly parallel) by the Morton cell
// on a 64^3 grid.  Rays of one warp then start close together and share the
// nodes they fetch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z, uint32_t bits) {
  uint32_t r = 0;
  for (uint32_t b = 0; b < bits; ++b)
    r |= (((x >> b) & 1u) << (3u * b)) | (((y >> b) & 1u) << (3u * b + 1u)) | (((z >> b) & 1u) << (3u * b + 2u));
  return r;
}

__device__ __forceinline__ uint32_t cell_of(const DevScene& S, float3 o, uint32_t bits) {
  const float n = (float)(1u << bits);
  const uint32_t m = (1u << bits) - 1u;
  const uint32_t x = min((uint32_t)fmaxf((o.x - S.blo[0]) * S.binv[0] * n, 0.0f), m);
  const uint32_t y = min((uint32_t)fmaxf((o.y - S.blo[1]) * S.binv[1] * n, 0.0f), m);
  const uint32_t z = min((uint32_t)fmaxf((o.z - S.blo[2]) * S.binv[2] * n, 0.0f), m);
  return morton3(x, y, z, bits);
}

template <bool SUN>
__global__ void k_rsort_hist(DevScene S, const float4* __restrict__ q, const Counters* __restrict__ cnt, uint32_t k,
                             uint32_t cap, uint32_t* __restrict__ key, uint32_t* __restrict__ bins) {
  const uint32_t count = min(SUN ? cnt[k].s_count : cnt[k].q_count, cap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const float4 a = __ldg(q + 2 * i);
    uint32_t kk;
    if (SUN) {
      kk = cell_of(S, f3(a), 6u);
    } else {
      const float4 b = __ldg(q + 2 * i + 1);
      const uint32_t oct = (b.x < 0.0f ? 1u : 0u) | (b.y < 0.0f ? 2u : 0u) | (b.z < 0.0f ? 4u : 0u);
      kk = cell_of(S, f3(a), 5u) | (oct << 15);
    }
    key[i] = kk;
    atomicAdd(bins + kk, 1u);
  }
}

template <bool SUN>
__global__ void k_rsort_scatter(const Counters* __restrict__ cnt, uint32_t k, uint32_t cap,
                                const uint32_t* __restrict__ key, uint32_t* __restrict__ bins,
                                uint32_t* __restrict__ perm) {
  const uint32_t count = min(SUN ? cnt[k].s_count : cnt[k].q_count, cap);
  const uint32_t* totals = bins + kCellSortBins;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const uint32_t kk = key[i];
    perm[__ldg(totals + (kk >> 10)) + atomicAdd(bins + kk, 1u)] = i;
  }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_camera(const DevCam* __restrict__ cams, uint32_t n_cams, WaveParams w,
                                                float4* __restrict__ q, float* __restrict__ L,
                                                uint32_t* __restrict__ sig, Counters* cnt, bool record,
                                                float4* __restrict__ L4, float4* __restrict__ T4, uint32_t cap,
                                                uint32_t* status) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cnt[1].q_count = w.n;
    if (w.n > cap) atomicOr(status, ST_QUEUE);  // a wave larger than its ray queue
  }
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += stride) {
    const PathId id = path_id(w, i);
    uint32_t v = 0;
    while (v + 1 < n_cams && cams[v + 1].offset <= id.pix) ++v;
    const DevCam& C = cams[v];
    const uint32_t local = id.pix - C.offset;
    const uint32_t y = local / C.W, x = local - y * C.W;
    const uint4 u = philox4x32_10(make_uint4(id.pix, id.s, w.band_first + id.j, 0u), w.key0, w.key1);
    const float sx = (2.0f * ((float)x + u01(u.x)) / (float)C.W - 1.0f) * C.tha;
    const float sy = (1.0f - 2.0f * ((float)y + u01(u.y)) / (float)C.H) * C.th;
    float3 dir = make_float3(C.f.x + sx * C.r.x + sy * C.u.x, C.f.y + sx * C.r.y + sy * C.u.y,
                             C.f.z + sx * C.r.z + sy * C.u.z);
    const float inv = 1.0f / sqrtf(dot(dir, dir));
    dir = mul(inv, dir);
    q[2 * i] = make_float4(C.pos.x, C.pos.y, C.pos.z, __uint_as_float(i));
    q[2 * i + 1] = make_float4(dir.x, dir.y, dir.z, 1.0f);
    if (w.nb == 4u) {
      // bands past the render's range carry nothing
      const uint32_t nv = four_band_count(w, id.j);
      L4[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      T4[i] = make_float4(1.0f, nv > 1u ? 1.0f : 0.0f, nv > 2u ? 1.0f : 0.0f, nv > 3u ? 1.0f : 0.0f);
    } else {
      L[i] = 0.0f;
    }
    if (record) sig[i] = 2166136261u;
  }
}

constexpr uint32_t kNoRay = 0xFFFFFFFFu;
// closest-hit kernel: blocks of at most 128 threads, launch bound 8 blocks
// per SM (<= 64 registers; the closest-hit kernel compiles to 56 and the
// launch takes the occupancy limit, 9 blocks, the one-band sun-ray kernel to
// 61 and 8 blocks).  With the 256-bit node loads, measured per render of the
// nave / the 2M-triangle nave, closest hit: bound 8 1372 / 2141 ms, bound 9
// 1384 / 2160, 7 and 6 about 1408 / 2200, 10 and 12 (spilled) 27% and 40%
// slower: more warps thrash the L1 that serves the node fetches
#ifndef SRT_TRACE_MIN_BLOCKS
#define SRT_TRACE_MIN_BLOCKS 8
#endif
constexpr int kTraceMaxThreads = 128, kTraceMinBlocks = SRT_TRACE_MIN_BLOCKS;
// sun-ray kernel: one band per path with the closest-hit kernel's bound
// (402 / 633 ms against 410 / 645 at bound 9, 56 registers); four bands per
// path at least 4 blocks of 256 threads' worth (<= 64 registers)
#ifndef SRT_SHADOW_MIN_BLOCKS
#define SRT_SHADOW_MIN_BLOCKS 4
#endif
constexpr int kShadowMinBlocks = SRT_SHADOW_MIN_BLOCKS;
#ifndef SRT_SHADOW_SORTED
constexpr bool kShadowAnyOrder = true;
#else
constexpr bool kShadowAnyOrder = false;
#endif

// Persistent traversal loop: a warp refills its idle lanes from the queue
// once at least `refill` lanes are idle, and each lane with a ray runs up to
// `steps` traversal steps between refill checks (steps large and refill 32
// give one batch of 32 rays per warp at a time).

// MODE 0: each lane runs up to `steps` node-or-leaf steps; 1: while-while
// steps; 2: warp-synchronous phases - interior steps for the lanes at an
// interior node until at least `leaf_min` lanes wait at a leaf (or none can
// go on), then one leaf step for every waiting lane, so that the costly
// triangle tests run with most of their lanes busy; 3 (the default, render
// option trace_variant 0): as 2 over the four-wide BVH; 4 (trace_variant 4):
// as 2 over the eight-wide BVH.  Modes 0-2 traverse the binary BVH.
template <bool FMA, bool COUNT, int MODE>
__global__ void __launch_bounds__(kTraceMaxThreads, kTraceMinBlocks) k_trace(DevScene S, const float4* __restrict__ q, float2* __restrict__ hit,
                                               Counters* cnt, uint32_t k, uint32_t cap, Totals* tot,
                                               uint32_t* status, int steps, int refill, int leaf_min,
                                               const uint32_t* __restrict__ perm) {
  const uint32_t count = min(cnt[k].q_count, cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&tot->ext_rays, (unsigned long long)count);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t icap = trav_cap(S);
  uint32_t nn = 0, nt = 0;
  Trav tv;
  uint2 stack[kStack];
  uint32_t ray = kNoRay;
  bool drained = count == 0u;
  for (;;) {
    const uint32_t idle = __ballot_sync(0xffffffffu, ray == kNoRay);
    if (!drained && (int)__popc(idle) >= refill) {
      const uint32_t n = __popc(idle);
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&cnt[k].q_fetch, n);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base + n >= count) drained = true;
      if (ray == kNoRay) {
        const uint32_t slot = base + __popc(idle & lt);
        if (slot < count) {
          const uint32_t ri = perm ? __ldg(perm + slot) : slot;
          const float4 a = __ldcs(q + 2 * ri), b = __ldcs(q + 2 * ri + 1);
          if (init_w<MODE >= 3, FMA>(tv, S, f3(a), f3(b))) {
            ray = ri;
          } else {
            __stcs(hit + ri, make_float2(-1.0f, __int_as_float(-1)));
          }
        }
      }
    }
    if (!__any_sync(0xffffffffu, ray != kNoRay)) {
      if (drained) break;
      continue;
    }
    if (MODE >= 2) {
      bool done = false;
      for (int i = 0; i < steps; ++i) {
        const bool act = ray != kNoRay && !done;
        const bool at_leaf = act && tv.cnt != 0u;
        const uint32_t ml = __ballot_sync(0xffffffffu, at_leaf);
        const uint32_t mi = __ballot_sync(0xffffffffu, act && !at_leaf);
        if ((ml | mi) == 0u) break;
        const bool leaf_phase = mi == 0u || (int)__popc(ml) >= leaf_min;
        if (act && at_leaf == leaf_phase) {
          if (++tv.iter > icap) {
            atomicOr(status, ST_ITER);
            done = true;
          } else if (leaf_phase) {
            closest_leaf(tv, S, nt, COUNT);
            done = !trav_pop(tv, stack, tv.best_t);
          } else if (!(MODE == 5   ? trav_interior4q<FMA, COUNT>(tv, stack, S, tv.best_t, status, nn)
                       : MODE == 4 ? trav_interior8<FMA, COUNT>(tv, stack, S, tv.best_t, status, nn)
                                   : interior_w<MODE == 3, FMA, COUNT>(tv, stack, S, tv.best_t, status, nn))) {
            done = !trav_pop(tv, stack, tv.best_t);
          }
        }
      }
      if (ray != kNoRay && done) {
        __stcs(hit + ray, make_float2(tv.best_leaf < 0 ? -1.0f : tv.best_t, __int_as_float(tv.best_leaf)));
        ray = kNoRay;
      }
    } else if (ray != kNoRay) {
      bool done = false;
      for (int i = 0; i < steps && !done; ++i)
        done = closest_step<FMA, COUNT, MODE == 1>(tv, stack, S, icap, status, nn, nt);
      if (done) {
        __stcs(hit + ray, make_float2(tv.best_leaf < 0 ? -1.0f : tv.best_t, __int_as_float(tv.best_leaf)));
        ray = kNoRay;
      }
    }
  }
  if (COUNT) {
    atomicAdd(&tot->nodes, (unsigned long long)nn);
    atomicAdd(&tot->tris, (unsigned long long)nt);
  }
}

// Spatial hash of an integer cell (three large odd multipliers, xor).
__device__ __forceinline__ uint32_t photon_cell_hash(int ix, int iy, int iz, uint32_t hbits) {
  const uint32_t h = ((uint32_t)ix * 73856093u) ^ ((uint32_t)iy * 19349663u) ^ ((uint32_t)iz * 83492791u);
  return h & ((1u << hbits) - 1u);
}

// Kernel-weighted flux of the photons of band j in map `map` within distance
// r of x, weight 1 - d^2 / r^2 (Epanechnikov): the (at most 8) cells of edge
// 2 r that the ball touches, duplicates of a hashed key skipped.
__device__ __forceinline__ float photon_gather(const PhotonMaps& M, uint32_t map, uint32_t j, float3 x) {
  const float ic = M.inv_cell[map];
  const float r = sqrtf(M.r2[map]);
  const int lx = (int)floorf((x.x - r) * ic), hx = (int)floorf((x.x + r) * ic);
  const int ly = (int)floorf((x.y - r) * ic), hy = (int)floorf((x.y + r) * ic);
  const int lz = (int)floorf((x.z - r) * ic), hz = (int)floorf((x.z + r) * ic);
  const uint32_t base = (map * M.Bc + j) << M.hbits;
  uint32_t seen[8];
  int ns = 0;
  float sum = 0.0f;
  for (int ix = lx; ix <= hx; ++ix)
    for (int iy = ly; iy <= hy; ++iy)
      for (int iz = lz; iz <= hz; ++iz) {
        const uint32_t key = base | photon_cell_hash(ix, iy, iz, M.hbits);
        bool dup = false;
        for (int q = 0; q < ns; ++q) dup |= seen[q] == key;
        if (dup || ns >= 8) continue;
        seen[ns++] = key;
        const uint32_t e = __ldg(M.end + key);
        for (uint32_t q = __ldg(M.start + key); q < e; ++q) {
          const float4 ph = ldg4(M.rec + q);
          const float dx = ph.x - x.x, dy = ph.y - x.y, dz = ph.z - x.z;
          const float d2 = dx * dx + dy * dy + dz * dz;
          if (d2 < M.r2[map]) sum += ph.w * (1.0f - d2 / M.r2[map]);
        }
      }
  return sum;
}

// PM: photon-mapping camera pass -- at the first Lambertian vertex the path
// adds (rho / pi) x the photon irradiance of both maps of pm and ends (its
// sun ray, if any, finishes it).
// three blocks of 256 per SM (<= 85 registers, no spills; unbounded, the
// one-band shading took 102 registers and two blocks): measured 291 instead
// of 304 ms per guided pass of the 2M-triangle nave, 375 instead of 377 ms
// per render of the nave; four blocks (64 registers, spilled) were slower
#ifndef SRT_SHADE_MIN_BLOCKS
#define SRT_SHADE_MIN_BLOCKS 3
#endif
template <bool RECORD, bool GUIDED, bool PM = false>
__global__ void __launch_bounds__(256, SRT_SHADE_MIN_BLOCKS) k_shade(DevScene S, DevSpectra P, WaveParams w, uint32_t k,
                                               const float4* __restrict__ qin, const float2* __restrict__ hit,
                                               float4* __restrict__ qout, float4* __restrict__ sq,
                                               float* __restrict__ Lbuf, uint32_t* __restrict__ sigbuf,
                                               Counters* cnt, uint32_t cap, double* __restrict__ accum,
                                               Probe probe, uint32_t* status, GuideWave gw, PhotonMaps pm) {
  const uint32_t count = min(cnt[k].q_count, cap);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < count; base += stride) {
    const uint32_t i = base + lane;
    bool emit_next = false, emit_shadow = false, emit_guide = false;
    float4 n0 = make_float4(0, 0, 0, 0), n1 = n0, s0 = n0, s1 = n0;
    float g_rho = 0.0f;
    if (i < count) {
      const float4 a = __ldcs(qin + 2 * i), b = __ldcs(qin + 2 * i + 1);
      const float2 h = __ldcs(hit + i);
      const uint32_t bits = __float_as_uint(a.w);
      const uint32_t pid = bits & kPidMask;
      const bool covered = (bits & kFlagCovered) != 0u;
      const float T = b.w;
      const float3 o = f3(a), d = f3(b);
      const PathId id = path_id(w, pid);
      const uint32_t band = w.band_first + id.j;
      float Lp = Lbuf[pid];
      uint32_t sg = RECORD ? sigbuf[pid] : 0u;
      // training slot of the previous (guided) vertex: radiance gathered so far
      if (GUIDED && gw.collect != 0u && k >= 2u && k - 1u <= gw.depth && pid % gw.collect == 0u)
        ((float*)(gw.raw + kRawF4 * ((k - 2u) * gw.slots_per_vertex + pid / gw.collect) + 1u))[3] = Lp;
      const int leaf = __float_as_int(h.y);
      bool terminate = false;
      if (leaf < 0) {
        if (RECORD) sg = mix_sig(sg, 0xFFFFFFFFu);
        if (dot(d, P.sun) >= P.cos_max) {
          if (!covered) Lp += T * __ldg(P.sunL + band);
          else if (GUIDED && (bits & kFlagGuidedEsc)) Lp += T * __ldg(P.sunL + band) * gw.wesc[pid];
        }
        terminate = true;
      } else {
        const float3 p = madd(o, h.x, d);
        const float4 nr = ldg4(S.nrm + leaf);
        const uint32_t mat = __float_as_uint(nr.w);
        if (RECORD) sg = mix_sig(sg, __float_as_uint(S.tris[3 * leaf].w));
        const float3 ng = f3(nr);
        const float3 n = dot(ng, d) < 0.0f ? ng : neg(ng);
        const float cos_i = -dot(d, n);
        const float4 m = ldg4(P.mb + mat * P.n_bands + band);
        const int type = __ldg(P.mtype + mat);
        const uint4 u = philox4x32_10(make_uint4(id.pix, id.s, band, 4u * k), w.key0, w.key1);
        if (type == 0 || type == 3) {
          if (type == 3) Lp += T * m.w;
          // next-event estimate: uniform direction in the sun cone
          const float om = u01(u.x) * P.one_minus_cos;
          const float ct = 1.0f - om;
          const float st = sqrtf(fmaxf(0.0f, om * (2.0f - om)));
          float sp_, cp_;
          sincospif(2.0f * u01(u.y), &sp_, &cp_);
          float3 t1, t2;
          onb(P.sun, t1, t2);
          const float3 wd = make_float3(st * cp_ * t1.x + st * sp_ * t2.x + ct * P.sun.x,
                                        st * cp_ * t1.y + st * sp_ * t2.y + ct * P.sun.y,
                                        st * cp_ * t1.z + st * sp_ * t2.z + ct * P.sun.z);
          const float c = dot(n, wd);
          const float3 po = madd(p, S.eps, n);
          if (c > 0.0f) {
            emit_shadow = true;
            const uint32_t fl = pid | ((PM || k == w.depth) ? kFlagTerm : 0u);
            s0 = make_float4(po.x, po.y, po.z, __uint_as_float(fl));
            s1 = make_float4(wd.x, wd.y, wd.z, T * m.z * c * __ldg(P.sunL + band) * 2.0f * P.one_minus_cos);
          }
          if (PM) {
            const float E = photon_gather(pm, 0u, id.j, p) * pm.norm[0] + photon_gather(pm, 1u, id.j, p) * pm.norm[1];
            Lp += T * m.z * (1.0f / 3.14159265358979f) * E;
            terminate = true;
          } else if (k == w.depth) {
            terminate = true;
          } else if (GUIDED && k <= gw.depth) {
            // the continuation is sampled by the guide kernel (one-sample MIS)
            emit_guide = true;
            n0 = make_float4(po.x, po.y, po.z, __uint_as_float(pid | kFlagCovered));
            n1 = make_float4(n.x, n.y, n.z, T);
            g_rho = m.z;
          } else {
            // cosine-weighted continuation, weight rho
            const float rr = sqrtf(u01(u.z));
            const float zz = sqrtf(fmaxf(0.0f, 1.0f - u01(u.z)));
            float s2, c2;
            sincospif(2.0f * u01(u.w), &s2, &c2);
            float3 b1, b2;
            onb(n, b1, b2);
            const float3 nd = make_float3(rr * c2 * b1.x + rr * s2 * b2.x + zz * n.x,
                                          rr * c2 * b1.y + rr * s2 * b2.y + zz * n.y,
                                          rr * c2 * b1.z + rr * s2 * b2.z + zz * n.z);
            emit_next = true;
            n0 = make_float4(po.x, po.y, po.z, __uint_as_float(pid | kFlagCovered));
            n1 = make_float4(nd.x, nd.y, nd.z, T * m.z);
          }
        } else if (type == 1) {
          float Rs, Ts;
          thin_sheet(cos_i, m.x, m.y, __ldg(P.ad + mat * P.n_bands + band), Rs, Ts);
          if (k == w.depth) {
            terminate = true;
          } else {
            const uint4 u1 = philox4x32_10(make_uint4(id.pix, id.s, band, 4u * k + 1u), w.key0, w.key1);
            emit_next = true;
            if (u01(u1.x) < Rs / (Rs + Ts)) {
              const float3 rd = madd(d, -2.0f * dot(d, n), n);
              const float3 po = madd(p, S.eps, n);
              n0 = make_float4(po.x, po.y, po.z, __uint_as_float(pid));
              n1 = make_float4(rd.x, rd.y, rd.z, T * (Rs + Ts));
            } else {
              const float3 po = madd(p, -S.eps, n);
              n0 = make_float4(po.x, po.y, po.z, __uint_as_float(pid | (bits & (kFlagCovered | kFlagGuidedEsc))));
              n1 = make_float4(d.x, d.y, d.z, T * (Rs + Ts));
            }
          }
        } else if (type == 4) {
          // solid refracting glass (section 3 Eq. 1): a segment that ends
          // here from inside crossed the medium, Beer-Lambert with alpha =
          // 4 pi k / lambda per metre; the face reflects with the Fresnel
          // reflectance of the relative index (n entering, 1/n leaving,
          // 1 past the critical angle), else refracts by Snell's law with
          // n(lambda).  The next ray starts a short step along itself so
          // that the distance crossed inside stays exact; the step's share
          // of the attenuation is taken now.
          const bool inside = dot(ng, d) > 0.0f;
          const float alpha = __ldg(P.ad + mat * P.n_bands + band);
          float Tn = inside ? T * expf(-alpha * h.x) : T;
          if (k == w.depth) {
            terminate = true;
          } else {
            const float eta = inside ? 1.0f / m.x : m.x;
            const float R = fresnel_complex(cos_i, eta, 0.0f);
            const float r = inside ? m.x : 1.0f / m.x;
            const float kk = 1.0f - r * r * (1.0f - cos_i * cos_i);
            const uint4 u1 = philox4x32_10(make_uint4(id.pix, id.s, band, 4u * k + 1u), w.key0, w.key1);
            float3 nd;
            if (u01(u1.x) < R || kk < 0.0f) {
              nd = madd(d, -2.0f * dot(d, n), n);
            } else {
              const float3 td = madd(make_float3(r * d.x, r * d.y, r * d.z), r * cos_i - sqrtf(kk), n);
              const float il = rsqrtf(dot(td, td));
              nd = make_float3(td.x * il, td.y * il, td.z * il);
            }
            const float step = S.eps / fmaxf(fabsf(dot(nd, n)), 0.0625f);
            if (dot(nd, ng) < 0.0f) Tn *= expf(-alpha * step);
            const float3 po = madd(p, step, nd);
            emit_next = true;
            n0 = make_float4(po.x, po.y, po.z, __uint_as_float(pid));
            n1 = make_float4(nd.x, nd.y, nd.z, Tn);
          }
        } else {
          const float R = fresnel_complex(cos_i, m.x, m.y);
          if (k == w.depth) {
            terminate = true;
          } else {
            const float3 rd = madd(d, -2.0f * dot(d, n), n);
            const float3 po = madd(p, S.eps, n);
            emit_next = true;
            n0 = make_float4(po.x, po.y, po.z, __uint_as_float(pid));
            n1 = make_float4(rd.x, rd.y, rd.z, T * R);
          }
        }
      }
      if (terminate && !emit_shadow) {
        finalize(w, id, Lp, sg, accum, probe, RECORD);
        if (GUIDED && gw.Lfinal) gw.Lfinal[pid] = Lp;
      } else {
        Lbuf[pid] = Lp;
        if (RECORD) sigbuf[pid] = sg;
      }
    }
    const uint32_t slot_n = warp_append(&cnt[k + 1].q_count, emit_next);
    const uint32_t slot_s = warp_append(&cnt[k].s_count, emit_shadow);
    if (GUIDED) {
      const uint32_t slot_g = warp_append(&cnt[k].g_count, emit_guide);
      if (emit_guide) {
        if (slot_g < cap) {
          gw.gq[3 * slot_g] = n0;
          gw.gq[3 * slot_g + 1] = n1;
          gw.gq[3 * slot_g + 2] =
              make_float4(g_rho, __uint_as_float(emit_shadow && slot_s < cap ? slot_s : 0xFFFFFFFFu), 0.0f, 0.0f);
        } else {
          atomicOr(status, ST_QUEUE);
        }
      }
    }
    if (emit_next) {
      if (slot_n < cap) {
        __stcs(qout + 2 * slot_n, n0);
        __stcs(qout + 2 * slot_n + 1, n1);
      } else {
        atomicOr(status, ST_QUEUE);
      }
    }
    if (emit_shadow) {
      if (slot_s < cap) {
        __stcs(sq + 2 * slot_s, s0);
        __stcs(sq + 2 * slot_s + 1, s1);
      } else {
        atomicOr(status, ST_QUEUE);
      }
    }
  }
}

// Shading for paths that carry four bands: path unit j of a pixel and
// sample carries bands band_first + j + q G, q = 0..3, G = ceil(B / 4) --
// spread over the spectrum like hero wavelengths, so that the bands of one
// path fall under different parts of the colour matching functions (four
// neighbouring bands would add their correlated noise into X, Y and Z
// almost undiluted); Philox counters are those of band j.  The bands share
// every direction until the first dispersive event:
//   Lambertian / emissive: one sun-ray direction and one cosine-sampled
//     continuation for all; per-band weights rho, emitted radiance, NEE;
//   thin glass: reflect with the mean over the carried bands of
//     R_s / (R_s + T_s), weights R_s / p or T_s / (1 - p) per band;
//   conductor: mirror, weight R per band;
//   solid glass: reflect with the mean Fresnel reflectance p, weight R / p;
//     else refraction bends each band differently, so one carried band,
//     chosen uniformly, continues with weight n_carried (1 - R) / (1 - p)
//     and the others stop (their radiance so far is kept).
// "Carried" = throughput != 0; with one band left every rule is the
// one-band rule of k_shade.  Each choice has the one-band expectation per
// band, so the four-band estimate of every band is unbiased.  Three blocks
// of 256 per SM (80 registers, a few bytes spilled) beat two blocks at 92.
template <bool RECORD>
__global__ void __launch_bounds__(256, 3) k_shade4(DevScene S, DevSpectra P, WaveParams w, uint32_t k,
                                                const float4* __restrict__ qin, const float2* __restrict__ hit,
                                                float4* __restrict__ qout, float4* __restrict__ sq,
                                                float4* __restrict__ L4, float4* __restrict__ T4,
                                                float4* __restrict__ C4, uint32_t* __restrict__ sigbuf,
                                                Counters* cnt, uint32_t cap, double* __restrict__ accum,
                                                Probe probe, uint32_t* status) {
  const uint32_t count = min(cnt[k].q_count, cap);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < count; base += stride) {
    const uint32_t i = base + lane;
    bool emit_next = false, emit_shadow = false;
    float4 n0 = make_float4(0, 0, 0, 0), n1 = n0, s0 = n0, s1 = n0;
    if (i < count) {
      const float4 a = __ldcs(qin + 2 * i), b = __ldcs(qin + 2 * i + 1);
      const float2 h = __ldcs(hit + i);
      const uint32_t bits = __float_as_uint(a.w);
      const uint32_t pid = bits & kPidMask;
      const bool covered = (bits & kFlagCovered) != 0u;
      const float3 o = f3(a), d = f3(b);
      const PathId id = path_id(w, pid);
      const uint32_t b0 = w.band_first + id.j, G = w.band_count;
      const uint32_t nv = four_band_count(w, id.j);
      const float4 t4 = T4[pid], l4 = L4[pid];
      float T[4] = {t4.x, t4.y, t4.z, t4.w}, L[4] = {l4.x, l4.y, l4.z, l4.w};
      uint32_t sg = RECORD ? sigbuf[pid] : 0u;
      const int leaf = __float_as_int(h.y);
      bool terminate = false;
      if (leaf < 0) {
        if (RECORD) sg = mix_sig(sg, 0xFFFFFFFFu);
        if (!covered && dot(d, P.sun) >= P.cos_max) {
#pragma unroll
          for (uint32_t q = 0; q < 4u; ++q)
            if (q < nv) L[q] += T[q] * __ldg(P.sunL + b0 + q * G);
        }
        terminate = true;
      } else {
        const float3 p = madd(o, h.x, d);
        const float4 nr = ldg4(S.nrm + leaf);
        const uint32_t mat = __float_as_uint(nr.w);
        if (RECORD) sg = mix_sig(sg, __float_as_uint(S.tris[3 * leaf].w));
        const float3 ng = f3(nr);
        const float3 n = dot(ng, d) < 0.0f ? ng : neg(ng);
        const float cos_i = -dot(d, n);
        const uint32_t mrow = mat * P.n_bands + b0;
        // material rows of the carried bands: each branch loads only the
        // fields it reads (n, k / rho, le), which keeps fewer registers live
        const float4* mr = P.mb + mrow;
        const int type = __ldg(P.mtype + mat);
        const uint4 u = philox4x32_10(make_uint4(id.pix, id.s, b0, 4u * k), w.key0, w.key1);
        // the bands still carried (throughput != 0), else every band of the path
        uint32_t act = 0;
#pragma unroll
        for (uint32_t q = 0; q < 4u; ++q)
          if (q < nv && T[q] != 0.0f) act |= 1u << q;
        if (act == 0u) act = (1u << nv) - 1u;
        const float na = (float)__popc(act);
        if (type == 0 || type == 3) {
          float rho[4];
#pragma unroll
          for (uint32_t q = 0; q < 4u; ++q) rho[q] = q < nv ? __ldg(&mr[q * G].z) : 0.0f;
          if (type == 3) {
#pragma unroll
            for (uint32_t q = 0; q < 4u; ++q)
              if (q < nv) L[q] += T[q] * __ldg(&mr[q * G].w);
          }
          const float om = u01(u.x) * P.one_minus_cos;
          const float ct = 1.0f - om;
          const float st = sqrtf(fmaxf(0.0f, om * (2.0f - om)));
          float sp_, cp_;
          sincospif(2.0f * u01(u.y), &sp_, &cp_);
          float3 t1, t2;
          onb(P.sun, t1, t2);
          const float3 wd = make_float3(st * cp_ * t1.x + st * sp_ * t2.x + ct * P.sun.x,
                                        st * cp_ * t1.y + st * sp_ * t2.y + ct * P.sun.y,
                                        st * cp_ * t1.z + st * sp_ * t2.z + ct * P.sun.z);
          const float c = dot(n, wd);
          const float3 po = madd(p, S.eps, n);
          if (c > 0.0f) {
            emit_shadow = true;
            float C[4];
#pragma unroll
            for (uint32_t q = 0; q < 4u; ++q)
              C[q] = q < nv ? T[q] * rho[q] * c * __ldg(P.sunL + b0 + q * G) * 2.0f * P.one_minus_cos : 0.0f;
            C4[pid] = make_float4(C[0], C[1], C[2], C[3]);
            const uint32_t fl = pid | (k == w.depth ? kFlagTerm : 0u);
            s0 = make_float4(po.x, po.y, po.z, __uint_as_float(fl));
            s1 = make_float4(wd.x, wd.y, wd.z, 0.0f);
          }
          if (k == w.depth) {
            terminate = true;
          } else {
            const float rr = sqrtf(u01(u.z));
            const float zz = sqrtf(fmaxf(0.0f, 1.0f - u01(u.z)));
            float s2, c2;
            sincospif(2.0f * u01(u.w), &s2, &c2);
            float3 b1, b2;
            onb(n, b1, b2);
            const float3 nd = make_float3(rr * c2 * b1.x + rr * s2 * b2.x + zz * n.x,
                                          rr * c2 * b1.y + rr * s2 * b2.y + zz * n.y,
                                          rr * c2 * b1.z + rr * s2 * b2.z + zz * n.z);
#pragma unroll
            for (int q = 0; q < 4; ++q) T[q] *= rho[q];
            emit_next = true;
            n0 = make_float4(po.x, po.y, po.z, __uint_as_float(pid | kFlagCovered));
            n1 = make_float4(nd.x, nd.y, nd.z, 0.0f);
          }
        } else if (type == 1) {
          float Rs[4], Ts[4];
#pragma unroll
          for (uint32_t q = 0; q < 4u; ++q) {
            Rs[q] = 0.0f;
            Ts[q] = 1.0f;
            if (q < nv) {
              const float2 nk = __ldg((const float2*)(mr + q * G));
              thin_sheet(cos_i, nk.x, nk.y, __ldg(P.ad + mrow + q * G), Rs[q], Ts[q]);
            }
          }
          if (k == w.depth) {
            terminate = true;
          } else {
            const uint4 u1 = philox4x32_10(make_uint4(id.pix, id.s, b0, 4u * k + 1u), w.key0, w.key1);
            float pr = 0.0f;
#pragma unroll
            for (uint32_t q = 0; q < 4u; ++q)
              if (act & (1u << q)) pr += Rs[q] / (Rs[q] + Ts[q]);
            pr /= na;
            emit_next = true;
            if (u01(u1.x) < pr) {
#pragma unroll
              for (int q = 0; q < 4; ++q) T[q] *= Rs[q] / pr;
              const float3 rd = madd(d, -2.0f * dot(d, n), n);
              const float3 po = madd(p, S.eps, n);
              n0 = make_float4(po.x, po.y, po.z, __uint_as_float(pid));
              n1 = make_float4(rd.x, rd.y, rd.z, 0.0f);
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q) T[q] *= Ts[q] / (1.0f - pr);
              const float3 po = madd(p, -S.eps, n);
              n0 = make_float4(po.x, po.y, po.z, __uint_as_float(pid | (bits & kFlagCovered)));
              n1 = make_float4(d.x, d.y, d.z, 0.0f);
            }
          }
        } else if (type == 4) {
          const bool inside = dot(ng, d) > 0.0f;
          float alpha[4];
#pragma unroll
          for (uint32_t q = 0; q < 4u; ++q) alpha[q] = q < nv ? __ldg(P.ad + mrow + q * G) : 0.0f;
          if (inside) {
#pragma unroll
            for (int q = 0; q < 4; ++q) T[q] *= expf(-alpha[q] * h.x);
          }
          if (k == w.depth) {
            terminate = true;
          } else {
            float R[4], nq[4];
#pragma unroll
            for (uint32_t q = 0; q < 4u; ++q) {
              nq[q] = q < nv ? __ldg(&mr[q * G].x) : 1.0f;
              R[q] = q < nv ? fresnel_complex(cos_i, inside ? 1.0f / nq[q] : nq[q], 0.0f) : 1.0f;
            }
            const uint4 u1 = philox4x32_10(make_uint4(id.pix, id.s, b0, 4u * k + 1u), w.key0, w.key1);
            float pr = 0.0f;
#pragma unroll
            for (uint32_t q = 0; q < 4u; ++q)
              if (act & (1u << q)) pr += R[q];
            pr /= na;
            float3 nd;
            if (u01(u1.x) < pr) {
#pragma unroll
              for (int q = 0; q < 4; ++q) T[q] *= R[q] / pr;
              nd = madd(d, -2.0f * dot(d, n), n);
            } else {
              // refraction is the dispersive event: one carried band goes on
              uint32_t pick = min((uint32_t)(u01(u1.y) * na), (uint32_t)na - 1u);
              uint32_t c = 0;
#pragma unroll
              for (uint32_t q = 0; q < 4u; ++q)
                if (act & (1u << q)) {
                  if (pick == 0u) c = q;
                  pick = pick == 0u ? 0xFFFFFFFFu : pick - 1u;
                }
              float Rc = R[0], nc = nq[0];
#pragma unroll
              for (uint32_t q = 1; q < 4u; ++q)
                if (q == c) {
                  Rc = R[q];
                  nc = nq[q];
                }
              const float wgt = na * (1.0f - Rc) / (1.0f - pr);
#pragma unroll
              for (uint32_t q = 0; q < 4u; ++q) T[q] = q == c ? T[q] * wgt : 0.0f;
              const float r = inside ? nc : 1.0f / nc;
              const float kk = 1.0f - r * r * (1.0f - cos_i * cos_i);
              if (kk < 0.0f) {
                nd = madd(d, -2.0f * dot(d, n), n);  // R = 1 there: the weight is already 0
              } else {
                const float3 td = madd(make_float3(r * d.x, r * d.y, r * d.z), r * cos_i - sqrtf(kk), n);
                const float il = rsqrtf(dot(td, td));
                nd = make_float3(td.x * il, td.y * il, td.z * il);
              }
            }
            const float step = S.eps / fmaxf(fabsf(dot(nd, n)), 0.0625f);
            if (dot(nd, ng) < 0.0f) {
#pragma unroll
              for (int q = 0; q < 4; ++q) T[q] *= expf(-alpha[q] * step);
            }
            const float3 po = madd(p, step, nd);
            emit_next = true;
            n0 = make_float4(po.x, po.y, po.z, __uint_as_float(pid));
            n1 = make_float4(nd.x, nd.y, nd.z, 0.0f);
          }
        } else {
          float R[4];
#pragma unroll
          for (uint32_t q = 0; q < 4u; ++q) {
            R[q] = 0.0f;
            if (q < nv) {
              const float2 nk = __ldg((const float2*)(mr + q * G));
              R[q] = fresnel_complex(cos_i, nk.x, nk.y);
            }
          }
          if (k == w.depth) {
            terminate = true;
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) T[q] *= R[q];
            const float3 rd = madd(d, -2.0f * dot(d, n), n);
            const float3 po = madd(p, S.eps, n);
            emit_next = true;
            n0 = make_float4(po.x, po.y, po.z, __uint_as_float(pid));
            n1 = make_float4(rd.x, rd.y, rd.z, 0.0f);
          }
        }
      }
      if (terminate && !emit_shadow) {
        finalize4(w, id, L, sg, accum, probe, RECORD);
      } else {
        L4[pid] = make_float4(L[0], L[1], L[2], L[3]);
        if (RECORD) sigbuf[pid] = sg;
      }
      if (emit_next) T4[pid] = make_float4(T[0], T[1], T[2], T[3]);
    }
    const uint32_t slot_n = warp_append(&cnt[k + 1].q_count, emit_next);
    const uint32_t slot_s = warp_append(&cnt[k].s_count, emit_shadow);
    if (emit_next) {
      if (slot_n < cap) {
        __stcs(qout + 2 * slot_n, n0);
        __stcs(qout + 2 * slot_n + 1, n1);
      } else {
        atomicOr(status, ST_QUEUE);
      }
    }
    if (emit_shadow) {
      if (slot_s < cap) {
        __stcs(sq + 2 * slot_s, s0);
        __stcs(sq + 2 * slot_s + 1, s1);
      } else {
        atomicOr(status, ST_QUEUE);
      }
    }
  }
}

// NB = 4: every sun ray belongs to a path that carries four bands; the ray
// gathers one transmittance per band and the contributions wait in C4.
template <bool RECORD, bool COUNT, int MODE, int NB = 1>
__global__ void __launch_bounds__(NB == 1 ? kTraceMaxThreads : 256, NB == 1 ? kTraceMinBlocks : kShadowMinBlocks)
    k_shadow(DevScene S, DevSpectra P, WaveParams w, uint32_t k,
                                                const float4* __restrict__ sq, float* __restrict__ Lbuf,
                                                uint32_t* __restrict__ sigbuf, Counters* cnt, uint32_t cap,
                                                double* __restrict__ accum, Probe probe, Totals* tot,
                                                uint32_t* status, int steps, int refill, float* Lfinal,
                                                GuideWave gw, int leaf_min, const uint32_t* __restrict__ perm,
                                                float4* __restrict__ L4, const float4* __restrict__ C4) {
  static_assert(NB == 1 || (NB == 4 && MODE >= 2), "four-band sun rays use the leaf-batched traversal");
  const bool rec_sun = gw.on && gw.collect != 0u && k <= gw.depth && k < w.depth;
  const uint32_t count = min(cnt[k].s_count, cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&tot->shadow_rays, (unsigned long long)count);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t icap = trav_cap(S);
  uint32_t nn = 0, nt = 0;
  Trav tv;
  uint2 stack[kStack];
  uint32_t ray = kNoRay, bits = 0, band = 0, ng = 0, nv = 1;
  float contrib = 0.0f, T[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) T[q] = 1.0f;
  float3 dir = make_float3(0.0f, 0.0f, 0.0f);
  bool drained = count == 0u;
  for (;;) {
    const uint32_t idle = __ballot_sync(0xffffffffu, ray == kNoRay);
    if (!drained && (int)__popc(idle) >= refill) {
      const uint32_t n = __popc(idle);
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&cnt[k].s_fetch, n);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base + n >= count) drained = true;
      if (ray == kNoRay) {
        const uint32_t slot = base + __popc(idle & lt);
        if (slot < count) {
          const uint32_t ri = perm ? __ldg(perm + slot) : slot;
          const float4 a = __ldcs(sq + 2 * ri), b = __ldcs(sq + 2 * ri + 1);
          ray = ri;
          bits = __float_as_uint(a.w);
          contrib = b.w;
          dir = f3(b);
          const uint32_t j = path_id(w, bits & kPidMask).j;
          band = w.band_first + j;
          if (NB == 4) nv = four_band_count(w, j);
#pragma unroll
          for (int q = 0; q < NB; ++q) T[q] = 1.0f;
          ng = 0;
          if (!init_w<MODE == 3, true>(tv, S, f3(a), dir)) tv.sp = -1;  // misses everything: finished
        }
      }
    }
    if (!__any_sync(0xffffffffu, ray != kNoRay)) {
      if (drained) break;
      continue;
    }
    bool done = false;
    if (MODE >= 2) {
      done = ray != kNoRay && tv.sp < 0;
      for (int i = 0; i < steps; ++i) {
        const bool act = ray != kNoRay && !done;
        const bool at_leaf = act && tv.cnt != 0u;
        const uint32_t ml = __ballot_sync(0xffffffffu, at_leaf);
        const uint32_t mi = __ballot_sync(0xffffffffu, act && !at_leaf);
        if ((ml | mi) == 0u) break;
        const bool leaf_phase = mi == 0u || (int)__popc(ml) >= leaf_min;
        if (act && at_leaf == leaf_phase) {
          if (++tv.iter > icap) {
            atomicOr(status, ST_ITER);
            done = true;
          } else if (leaf_phase) {
            bool opaque;
            if constexpr (NB == 4) opaque = shadow_leaf4(tv, S, P, dir, band, w.band_count, nv, T, ng, nt, COUNT);
            else opaque = shadow_leaf(tv, S, P, dir, band, T[0], ng, nt, COUNT);
            done = opaque || !trav_pop(tv, stack, INFINITY);
          } else if (!interior_w<MODE == 3, true, COUNT, kShadowAnyOrder>(tv, stack, S, INFINITY, status, nn)) {
            done = !trav_pop(tv, stack, INFINITY);
          }
        }
      }
    } else if (ray != kNoRay) {
      done = tv.sp < 0;
      for (int i = 0; i < steps && !done; ++i)
        done = shadow_step<true, COUNT, MODE == 1>(tv, stack, S, P, dir, band, T[0], ng, icap, status, nn, nt);
    }
    if constexpr (NB == 4) {
      if (done) {
        const uint32_t pid = bits & kPidMask;
        const float4 c4 = C4[pid], l4 = L4[pid];
        const float L[4] = {l4.x + c4.x * T[0], l4.y + c4.y * T[1], l4.z + c4.z * T[2], l4.w + c4.w * T[3]};
        uint32_t sg = 0;
        if (RECORD) sg = mix_sig(sigbuf[pid], ng);
        if (bits & kFlagTerm) {
          finalize4(w, path_id(w, pid), L, sg, accum, probe, RECORD);
        } else {
          L4[pid] = make_float4(L[0], L[1], L[2], L[3]);
          if (RECORD) sigbuf[pid] = sg;
        }
        ray = kNoRay;
      }
      continue;
    }
    if (done) {
      const uint32_t pid = bits & kPidMask;
      const PathId id = path_id(w, pid);
      const float Lp = Lbuf[pid] + contrib * T[0];
      if (rec_sun && pid % gw.collect == 0u)
        ((float*)(gw.raw + kRawF4 * ((k - 1u) * gw.slots_per_vertex + pid / gw.collect) + 5u))[0] =
            T[0] * __ldg(P.sunL + w.band_first + id.j);
      uint32_t sg = 0;
      if (RECORD) sg = mix_sig(sigbuf[pid], ng);
      if (bits & kFlagTerm) {
        finalize(w, id, Lp, sg, accum, probe, RECORD);
        if (Lfinal) Lfinal[pid] = Lp;
      } else {
        Lbuf[pid] = Lp;
        if (RECORD) sigbuf[pid] = sg;
      }
      ray = kNoRay;
    }
  }
  if (COUNT) {
    atomicAdd(&tot->snodes, (unsigned long long)nn);
    atomicAdd(&tot->stris, (unsigned long long)nt);
  }
}

// Streaming-read probe: every thread reads float4s of a buffer that fits in
// L2, `iters` passes; the sum goes to a sink so the loads are not removed.
__global__ void __launch_bounds__(512) k_l2_probe(const float4* __restrict__ buf, size_t n4, int iters,
                                                  float* __restrict__ sink) {
  float acc = 0.0f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int it = 0; it < iters; ++it)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);
      acc += v.x + v.y + v.z + v.w;
    }
  if (acc == 1.2345f) sink[0] = acc;
}

// ---- photon mapping (section 4) ----------------------------------------

// Photon pass: one thread per photon.  Emission from the disk tangent to the
// scene's bounding sphere on the sun's side, direction minus a uniform
// sample of the sun cone, flux L_sun cos Omega pi R_d^2 / N; then the path
// tracer's material rules, storing every Lambertian hit (direct: only
// thin-glass transmissions before it; caustic: a reflection or refraction
// before the first diffuse hit; indirect: after a diffuse hit).
__global__ void __launch_bounds__(128) k_photon_trace(DevScene S, DevSpectra P, PhotonPass pp,
                                                      float4* __restrict__ rec, uint32_t* __restrict__ keys,
                                                      uint32_t* __restrict__ vals, uint8_t* __restrict__ cls,
                                                      uint32_t* status) {
  const uint32_t total = pp.Bc * pp.N;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    const uint32_t j = g / pp.N, i = g - j * pp.N;
    const uint32_t b = pp.band0 + j;
    const size_t slot0 = (size_t)g * pp.depth;
    for (uint32_t q = 0; q < pp.depth; ++q) {
      keys[slot0 + q] = kPhotonEmpty;
      vals[slot0 + q] = (uint32_t)(slot0 + q);
      rec[slot0 + q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (cls) cls[slot0 + q] = 0;
    }
    const uint4 r0 = philox4x32_10(make_uint4(i, b, 0u, 0u), pp.key0, pp.key1);
    float3 o, d;
    float phi;
    if (pp.emission == 0u) {
      const float rad = pp.Rd * sqrtf(u01(r0.x));
      float sp, cp;
      sincospif(2.0f * u01(r0.y), &sp, &cp);
      o = make_float3(pp.c0.x + rad * (cp * pp.t1.x + sp * pp.t2.x), pp.c0.y + rad * (cp * pp.t1.y + sp * pp.t2.y),
                      pp.c0.z + rad * (cp * pp.t1.z + sp * pp.t2.z));
      const float om = u01(r0.z) * P.one_minus_cos;
      const float ct = 1.0f - om;
      const float st = sqrtf(fmaxf(0.0f, om * (2.0f - om)));
      float sp2, cp2;
      sincospif(2.0f * u01(r0.w), &sp2, &cp2);
      d = make_float3(-(st * cp2 * pp.t1.x + st * sp2 * pp.t2.x + ct * P.sun.x),
                      -(st * cp2 * pp.t1.y + st * sp2 * pp.t2.y + ct * P.sun.y),
                      -(st * cp2 * pp.t1.z + st * sp2 * pp.t2.z + ct * P.sun.z));
      phi = __ldg(P.sunL + b) * ct * pp.flux;
    } else {
      // portal emission: a thin-glass triangle by its share of A |s . n|
      // (the first whose cumulative share exceeds u0), a uniform point on
      // it, a direction of the cone; nothing when the direction grazes the
      // face from behind or the way back to the sun is blocked
      const float u0 = u01(r0.x);
      uint32_t lo = 0, hi = pp.n_portal - 1u;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(pp.cdf + mid) > u0) hi = mid;
        else lo = mid + 1u;
      }
      const float4 v0 = ldg4(pp.portal + 4u * lo), v1 = ldg4(pp.portal + 4u * lo + 1u),
                   v2 = ldg4(pp.portal + 4u * lo + 2u), pn = ldg4(pp.portal + 4u * lo + 3u);
      const float su = sqrtf(u01(r0.y)), u2 = u01(r0.z);
      const float wa = 1.0f - su, wb = su * (1.0f - u2), wc = su * u2;
      const float3 pg = make_float3(wa * v0.x + wb * v1.x + wc * v2.x, wa * v0.y + wb * v1.y + wc * v2.y,
                                    wa * v0.z + wb * v1.z + wc * v2.z);
      const uint4 r1 = philox4x32_10(make_uint4(i, b, 0u, 1u), pp.key0, pp.key1);
      const float om = u01(r1.x) * P.one_minus_cos;
      const float ct = 1.0f - om;
      const float st = sqrtf(fmaxf(0.0f, om * (2.0f - om)));
      float sp2, cp2;
      sincospif(2.0f * u01(r1.y), &sp2, &cp2);
      const float3 w = make_float3(st * cp2 * pp.t1.x + st * sp2 * pp.t2.x + ct * P.sun.x,
                                   st * cp2 * pp.t1.y + st * sp2 * pp.t2.y + ct * P.sun.y,
                                   st * cp2 * pp.t1.z + st * sp2 * pp.t2.z + ct * P.sun.z);
      const float3 pnv = f3(pn);
      const float wn = dot(w, pnv);
      if (!(wn > 0.0f)) continue;
      o = madd(pg, S.eps, pnv);
      float tb;
      int lb;
      closest_hit(S, o, w, tb, lb, status);
      if (lb >= 0) continue;
      d = neg(w);
      phi = __ldg(P.sunL + b) * wn * pp.flux * pn.w;
    }
    bool nee_path = true;
    uint32_t n_diff = 0;
    for (uint32_t k = 1; k <= pp.depth; ++k) {
      float t;
      int leaf;
      closest_hit(S, o, d, t, leaf, status);
      if (leaf < 0) break;
      const float3 p = madd(o, t, d);
      const float4 nr = ldg4(S.nrm + leaf);
      const uint32_t mat = __float_as_uint(nr.w);
      const float3 ng = f3(nr);
      const float3 n = dot(ng, d) < 0.0f ? ng : neg(ng);
      const float cos_i = -dot(d, n);
      const float4 m = ldg4(P.mb + mat * P.n_bands + b);
      const int type = __ldg(P.mtype + mat);
      const uint4 u = philox4x32_10(make_uint4(i, b, 0u, 4u * k), pp.key0, pp.key1);
      if (type == 0 || type == 3) {
        const uint32_t c = n_diff > 0u ? 3u : (nee_path ? 1u : 2u);
        const size_t slot = slot0 + n_diff;
        rec[slot] = make_float4(p.x, p.y, p.z, phi);
        if (cls) cls[slot] = (uint8_t)c;
        if (c != 1u) {
          const uint32_t map = c == 2u ? 0u : 1u;
          const float ic = pp.inv_cell[map];
          const uint32_t h = photon_cell_hash((int)floorf(p.x * ic), (int)floorf(p.y * ic), (int)floorf(p.z * ic),
                                              pp.hbits);
          keys[slot] = ((map * pp.Bc + j) << pp.hbits) | h;
        }
        ++n_diff;
        if (k == pp.depth) break;
        const float rr = sqrtf(u01(u.z));
        const float zz = sqrtf(fmaxf(0.0f, 1.0f - u01(u.z)));
        float s2, c2;
        sincospif(2.0f * u01(u.w), &s2, &c2);
        float3 b1, b2;
        onb(n, b1, b2);
        d = make_float3(rr * c2 * b1.x + rr * s2 * b2.x + zz * n.x, rr * c2 * b1.y + rr * s2 * b2.y + zz * n.y,
                        rr * c2 * b1.z + rr * s2 * b2.z + zz * n.z);
        o = madd(p, S.eps, n);
        phi *= m.z;
      } else if (type == 1) {
        float Rs, Ts;
        thin_sheet(cos_i, m.x, m.y, __ldg(P.ad + mat * P.n_bands + b), Rs, Ts);
        if (k == pp.depth) break;
        const uint4 u1 = philox4x32_10(make_uint4(i, b, 0u, 4u * k + 1u), pp.key0, pp.key1);
        if (u01(u1.x) < Rs / (Rs + Ts)) {
          d = madd(d, -2.0f * dot(d, n), n);
          o = madd(p, S.eps, n);
          nee_path = false;
        } else {
          o = madd(p, -S.eps, n);
        }
        phi *= Rs + Ts;
      } else if (type == 4) {
        const bool inside = dot(ng, d) > 0.0f;
        const float alpha = __ldg(P.ad + mat * P.n_bands + b);
        if (inside) phi *= expf(-alpha * t);
        if (k == pp.depth) break;
        const float eta = inside ? 1.0f / m.x : m.x;
        const float R = fresnel_complex(cos_i, eta, 0.0f);
        const float r = inside ? m.x : 1.0f / m.x;
        const float kk = 1.0f - r * r * (1.0f - cos_i * cos_i);
        const uint4 u1 = philox4x32_10(make_uint4(i, b, 0u, 4u * k + 1u), pp.key0, pp.key1);
        if (u01(u1.x) < R || kk < 0.0f) {
          d = madd(d, -2.0f * dot(d, n), n);
        } else {
          const float3 td = madd(make_float3(r * d.x, r * d.y, r * d.z), r * cos_i - sqrtf(kk), n);
          const float il = rsqrtf(dot(td, td));
          d = make_float3(td.x * il, td.y * il, td.z * il);
        }
        const float step = S.eps / fmaxf(fabsf(dot(d, n)), 0.0625f);
        if (dot(d, ng) < 0.0f) phi *= expf(-alpha * step);
        o = madd(p, step, d);
        nee_path = false;
      } else {
        const float R = fresnel_complex(cos_i, m.x, m.y);
        if (k == pp.depth) break;
        d = madd(d, -2.0f * dot(d, n), n);
        o = madd(p, S.eps, n);
        phi *= R;
        nee_path = false;
      }
    }
  }
}

// Record ranges per key of the sorted photon slots, and the records in key
// order.
__global__ void k_photon_bounds(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ sv, uint32_t n,
                                const float4* __restrict__ rec, float4* __restrict__ rs, uint32_t* __restrict__ start,
                                uint32_t* __restrict__ end) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const uint32_t key = sk[q];
    if (key == kPhotonEmpty) continue;
    rs[q] = rec[sv[q]];
    if (q == 0u || sk[q - 1] != key) start[key] = q;
    if (q + 1u == n || sk[q + 1] != key) end[key] = q + 1u;
  }
}

// ---- single-step kernels for parity tests --------------------------------

__global__ void k_philox(const uint4* __restrict__ ctr, uint4* __restrict__ out, uint64_t n, uint32_t k0, uint32_t k1) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = philox4x32_10(ctr[i], k0, k1);
}

__global__ void k_closest_rays(DevScene S, const float* __restrict__ o, const float* __restrict__ d, uint64_t n,
                               float* __restrict__ tout, int32_t* __restrict__ prim, uint32_t* status) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    float t;
    int leaf;
    closest_hit(S, make_float3(o[3 * i], o[3 * i + 1], o[3 * i + 2]), make_float3(d[3 * i], d[3 * i + 1], d[3 * i + 2]),
                t, leaf, status);
    tout[i] = leaf < 0 ? -1.0f : t;
    prim[i] = leaf < 0 ? -1 : (int32_t)__float_as_uint(S.tris[3 * leaf].w);
  }
}

__global__ void k_shadow_rays(DevScene S, DevSpectra P, const float* __restrict__ o, const float* __restrict__ d,
                              const uint32_t* __restrict__ band, uint64_t n, float* __restrict__ T,
                              uint32_t* __restrict__ ng, uint32_t* status) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t g;
    T[i] = shadow_T(S, P, make_float3(o[3 * i], o[3 * i + 1], o[3 * i + 2]), make_float3(d[3 * i], d[3 * i + 1], d[3 * i + 2]),
                    band[i], g, status);
    ng[i] = g;
  }
}

__global__ void k_optics(const float* __restrict__ c, const float* __restrict__ n, const float* __restrict__ k,
                         const float* __restrict__ lam, const float* __restrict__ dd, uint64_t count,
                         float* __restrict__ R, float* __restrict__ Rs, float* __restrict__ Ts) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
    R[i] = fresnel_complex(c[i], n[i], k[i]);
    if (lam != nullptr && dd != nullptr) {
      // alpha d in FP64 then rounded, as the spectra tables are prepared
      const float ad = (float)(4.0 * 3.14159265358979323846 * (double)k[i] * (double)dd[i] / ((double)lam[i] * 1e-9));
      float rs, ts;
      thin_sheet(c[i], n[i], k[i], ad, rs, ts);
      Rs[i] = rs;
      Ts[i] = ts;
    }
  }
}

int grid_for(uint64_t n, int block) {
  uint64_t g = (n + block - 1) / block;
  if (g > 65535ull * 8) g = 65535ull * 8;
  return (int)(g == 0 ? 1 : g);
}

template <bool FMA, bool COUNT, int MODE>
void trace_t(const LaunchCfg& lc, const DevScene& S, const float4* qin, const WaveBufs& b, uint32_t k, cudaStream_t st) {
  const uint32_t* perm = (lc.sort_rays && k >= 2 && b.rperm) ? b.rperm : nullptr;
  k_trace<FMA, COUNT, MODE><<<lc.grid_trace, lc.block_trace, 0, st>>>(S, qin, b.hit, b.cnt, k, b.cap, b.tot, b.status,
                                                                     lc.trace_steps, lc.trace_refill, lc.leaf_min,
                                                                     perm);
}

template <bool FMA, bool COUNT>
void trace_m(const LaunchCfg& lc, const DevScene& S, const float4* qin, const WaveBufs& b, uint32_t k,
             cudaStream_t st) {
  if (lc.variant == 5) trace_t<FMA, COUNT, 5>(lc, S, qin, b, k, st);
  else if (lc.variant == 4) trace_t<FMA, COUNT, 4>(lc, S, qin, b, k, st);
  else if (lc.variant == 3) trace_t<FMA, COUNT, 2>(lc, S, qin, b, k, st);
  else if (lc.variant == 2) trace_t<FMA, COUNT, 0>(lc, S, qin, b, k, st);
  else if (lc.variant == 1) trace_t<FMA, COUNT, 1>(lc, S, qin, b, k, st);
  else trace_t<FMA, COUNT, 3>(lc, S, qin, b, k, st);
}

void launch_trace(const LaunchCfg& lc, bool robust, const DevScene& S, const float4* qin, const WaveBufs& b, uint32_t k,
                  cudaStream_t st) {
  if (robust) {
    if (lc.counting) trace_m<false, true>(lc, S, qin, b, k, st);
    else trace_m<false, false>(lc, S, qin, b, k, st);
  } else {
    if (lc.counting) trace_m<true, true>(lc, S, qin, b, k, st);
    else trace_m<true, false>(lc, S, qin, b, k, st);
  }
}

template <bool RECORD, bool COUNT, int MODE, int NB = 1>
void shadow_t(const LaunchCfg& lc, const DevScene& S, const DevSpectra& P, const WaveParams& w, uint32_t k,
              const WaveBufs& b, double* accum, const Probe& probe, float* Lfinal, const GuideWave& gw,
              cudaStream_t st) {
  const uint32_t* perm = (lc.sort_rays && b.rperm) ? b.rperm : nullptr;
  k_shadow<RECORD, COUNT, MODE, NB><<<lc.grid_shadow, lc.block_trace, 0, st>>>(
      S, P, w, k, b.sq, b.L, b.sig, b.cnt, b.cap, accum, probe, b.tot, b.status, lc.shadow_steps, lc.shadow_refill,
      Lfinal, gw, lc.leaf_min, perm, b.L4, b.C4);
}

template <bool RECORD, bool COUNT>
void shadow_m(const LaunchCfg& lc, const DevScene& S, const DevSpectra& P, const WaveParams& w, uint32_t k,
              const WaveBufs& b, double* accum, const Probe& probe, float* Lf, const GuideWave& gw, cudaStream_t st) {
  // four bands per path: the four-wide tree with leaf batching (the host
  // refuses other traversal variants there)
  if (w.nb == 4u) shadow_t<RECORD, COUNT, 3, 4>(lc, S, P, w, k, b, accum, probe, Lf, gw, st);
  // (the eight-wide variant 4 changes the closest-hit traversal only)
  else if (lc.variant == 3) shadow_t<RECORD, COUNT, 2>(lc, S, P, w, k, b, accum, probe, Lf, gw, st);
  else if (lc.variant == 2) shadow_t<RECORD, COUNT, 0>(lc, S, P, w, k, b, accum, probe, Lf, gw, st);
  else if (lc.variant == 1) shadow_t<RECORD, COUNT, 1>(lc, S, P, w, k, b, accum, probe, Lf, gw, st);
  else shadow_t<RECORD, COUNT, 3>(lc, S, P, w, k, b, accum, probe, Lf, gw, st);
}

void launch_shadow(const LaunchCfg& lc, const DevScene& S, const DevSpectra& P, const WaveParams& w, uint32_t k,
                   const WaveBufs& b, double* accum, const Probe& probe, float* Lf, const GuideWave& gw,
                   cudaStream_t st) {
  if (lc.record) {
    if (lc.counting) shadow_m<true, true>(lc, S, P, w, k, b, accum, probe, Lf, gw, st);
    else shadow_m<true, false>(lc, S, P, w, k, b, accum, probe, Lf, gw, st);
  } else {
    if (lc.counting) shadow_m<false, true>(lc, S, P, w, k, b, accum, probe, Lf, gw, st);
    else shadow_m<false, false>(lc, S, P, w, k, b, accum, probe, Lf, gw, st);
  }
}

template <bool SUN>
void sort_queue(const DevScene& S, const float4* q, const WaveBufs& b, uint32_t k, cudaStream_t st, int sms) {
  const int g = sms > 0 ? sms * 8 : 1024;
  cudaMemsetAsync(b.rbins, 0, kCellSortBins * sizeof(uint32_t), st);
  k_rsort_hist<SUN><<<g, 256, 0, st>>>(S, q, b.cnt, k, b.cap, b.rkey, b.rbins);
  k_cell_scan_chunks<<<kCellSortBins / 1024u, 1024, 0, st>>>(b.rbins, b.rbins + kCellSortBins);
  k_cell_scan_totals<<<1, kCellSortBins / 1024u, 0, st>>>(b.rbins + kCellSortBins);
  k_rsort_scatter<SUN><<<g, 256, 0, st>>>(b.cnt, k, b.cap, b.rkey, b.rbins, b.rperm);
}

}  // namespace

void launch_cell_scan(uint32_t* bins, cudaStream_t st) { launch_scan(bins, kCellSortBins, st); }

void launch_scan(uint32_t* data, size_t n, cudaStream_t st) {
  k_cell_scan_chunks<<<(unsigned)(n / 1024u), 1024, 0, st>>>(data, data + n);
  k_cell_scan_totals<<<1, (unsigned)(n / 1024u), 0, st>>>(data + n);
}

void launch_wave(const LaunchCfg& lc, const DevScene& S, const DevSpectra& P, const DevCam* cams, uint32_t n_cams,
                 const WaveParams& w, const WaveBufs& b, double* accum, const Probe& probe, cudaStream_t st,
                 int* launches, StageTimer* tm, const GuideWave* gwp, const GuideDev* gdev, const void* gpack,
                 int sms, const PhotonMaps* pm) {
  GuideWave gw{};
  if (gwp) gw = *gwp;
  const bool guided = gw.on;
  const bool rec = lc.record;
  if (tm) tm->begin(STG_CAMERA, st);
  k_camera<<<grid_for(w.n, 256), 256, 0, st>>>(cams, n_cams, w, b.q[1], b.L, b.sig, b.cnt, rec, b.L4, b.T4, b.cap,
                                                b.status);
  if (tm) tm->end(STG_CAMERA, st);
  int nl = 1;
  for (uint32_t k = 1; k <= w.depth; ++k) {
    const float4* qin = b.q[k & 1];
    float4* qout = b.q[(k + 1) & 1];
    if (tm) tm->begin(STG_TRACE, st);
    if (lc.sort_rays && k >= 2 && b.rperm) {
      sort_queue<false>(S, qin, b, k, st, sms);
      nl += 4;
    }
    // vertex 1 starts at the cameras, which may lie anywhere: robust box
    // test; later origins are surface points inside the padded bounds
    launch_trace(lc, k == 1, S, qin, b, k, st);
    if (tm) tm->end(STG_TRACE, st);
    if (tm) tm->begin(STG_SHADE, st);
    if (w.nb == 4u) {
      if (rec)
        k_shade4<true><<<lc.grid_shade, lc.block_shade, 0, st>>>(S, P, w, k, qin, b.hit, qout, b.sq, b.L4, b.T4, b.C4,
                                                                 b.sig, b.cnt, b.cap, accum, probe, b.status);
      else
        k_shade4<false><<<lc.grid_shade, lc.block_shade, 0, st>>>(S, P, w, k, qin, b.hit, qout, b.sq, b.L4, b.T4,
                                                                  b.C4, b.sig, b.cnt, b.cap, accum, probe, b.status);
    } else if (pm) {
      if (rec)
        k_shade<true, false, true><<<lc.grid_shade, lc.block_shade, 0, st>>>(
            S, P, w, k, qin, b.hit, qout, b.sq, b.L, b.sig, b.cnt, b.cap, accum, probe, b.status, gw, *pm);
      else
        k_shade<false, false, true><<<lc.grid_shade, lc.block_shade, 0, st>>>(
            S, P, w, k, qin, b.hit, qout, b.sq, b.L, b.sig, b.cnt, b.cap, accum, probe, b.status, gw, *pm);
    } else if (guided) {
      if (rec)
        k_shade<true, true><<<lc.grid_shade, lc.block_shade, 0, st>>>(S, P, w, k, qin, b.hit, qout, b.sq, b.L, b.sig,
                                                                     b.cnt, b.cap, accum, probe, b.status, gw, PhotonMaps{});
      else
        k_shade<false, true><<<lc.grid_shade, lc.block_shade, 0, st>>>(S, P, w, k, qin, b.hit, qout, b.sq, b.L, b.sig,
                                                                      b.cnt, b.cap, accum, probe, b.status, gw, PhotonMaps{});
    } else {
      if (rec)
        k_shade<true, false><<<lc.grid_shade, lc.block_shade, 0, st>>>(S, P, w, k, qin, b.hit, qout, b.sq, b.L, b.sig,
                                                                      b.cnt, b.cap, accum, probe, b.status, gw, PhotonMaps{});
      else
        k_shade<false, false><<<lc.grid_shade, lc.block_shade, 0, st>>>(S, P, w, k, qin, b.hit, qout, b.sq, b.L,
                                                                       b.sig, b.cnt, b.cap, accum, probe, b.status, gw, PhotonMaps{});
    }
    if (tm) tm->end(STG_SHADE, st);
    if (guided && k <= gw.depth && k < w.depth) {
      if (tm) tm->begin(STG_GUIDE, st);
      launch_guide_sample(*gdev, gpack, P, w, k, gw, b, accum, probe, rec, sms, st);
      if (tm) tm->end(STG_GUIDE, st);
      nl += gw.perm ? 5 : 1;  // with the query sort: histogram, 2 scans, scatter
    }
    if (tm) tm->begin(STG_SHADOW, st);
    if (lc.sort_rays && b.rperm) {
      sort_queue<true>(S, b.sq, b, k, st, sms);
      nl += 4;
    }
    launch_shadow(lc, S, P, w, k, b, accum, probe, guided ? gw.Lfinal : nullptr, gw, st);
    if (tm) tm->end(STG_SHADOW, st);
    nl += 3;
  }
  if (launches) *launches += nl;
}

void launch_photon_trace(const DevScene& S, const DevSpectra& P, const PhotonPass& pp, float4* rec, uint32_t* keys,
                         uint32_t* vals, uint8_t* cls, uint32_t* status, int sms, cudaStream_t st) {
  const uint64_t n = (uint64_t)pp.Bc * pp.N;
  const unsigned g = (unsigned)std::min<uint64_t>((n + 127) / 128, (uint64_t)(sms > 0 ? sms : 1) * 64);
  k_photon_trace<<<g, 128, 0, st>>>(S, P, pp, rec, keys, vals, cls, status);
}

void launch_photon_maps(const uint32_t* sorted_keys, const uint32_t* sorted_vals, uint32_t n, const float4* rec,
                        float4* rec_sorted, uint32_t* start, uint32_t* end, int sms, cudaStream_t st) {
  k_photon_bounds<<<(sms > 0 ? sms : 1) * 8, 256, 0, st>>>(sorted_keys, sorted_vals, n, rec, rec_sorted, start, end);
}

void launch_philox(const uint32_t* ctr, uint32_t* out, uint64_t n, uint32_t k0, uint32_t k1, cudaStream_t st) {
  k_philox<<<grid_for(n, 256), 256, 0, st>>>((const uint4*)ctr, (uint4*)out, n, k0, k1);
}

void launch_trace_closest_rays(const DevScene& S, const float* o, const float* d, uint64_t n, float* t, int32_t* prim,
                               uint32_t* status, cudaStream_t st) {
  k_closest_rays<<<grid_for(n, 128), 128, 0, st>>>(S, o, d, n, t, prim, status);
}

void launch_trace_shadow_rays(const DevScene& S, const DevSpectra& P, const float* o, const float* d,
                              const uint32_t* band, uint64_t n, float* T, uint32_t* n_glass, uint32_t* status,
                              cudaStream_t st) {
  k_shadow_rays<<<grid_for(n, 128), 128, 0, st>>>(S, P, o, d, band, n, T, n_glass, status);
}

void launch_optics(const float* c, const float* n, const float* k, const float* lam, const float* d, uint64_t count,
                   float* R, float* Rs, float* Ts, cudaStream_t st) {
  k_optics<<<grid_for(count, 256), 256, 0, st>>>(c, n, k, lam, d, count, R, Rs, Ts);
}

// Orders the four children of every four-wide node by the position of
// their box centres along the sun direction s, farthest first; empty slots
// (packed reference 0) last, ties by the packed reference, so that the order
// depends only on the children and s.  Sun rays visit entered children in
// slot order and stop at the first opaque triangle: in an enclosed scene the
// occluder is most often the outer shell, which far-first order reaches
// sooner (nave: 5.2 instead of 8.0 node visits per sun ray, counted on the
// CPU).  Closest-hit traversal sorts children per ray and does not depend
// on slot order.
__global__ void k_sun_order4(float4* __restrict__ nodes4, uint32_t n, float3 s) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float* f = reinterpret_cast<float*>(nodes4 + 8 * (size_t)i);
    float x[28];
#pragma unroll
    for (int q = 0; q < 28; ++q) x[q] = f[q];
    float key[4];
    uint32_t pk[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      pk[c] = __float_as_uint(x[24 + c]);
      key[c] = pk[c] == 0u ? -INFINITY
                           : (x[c] + x[4 + c]) * s.x + (x[8 + c] + x[12 + c]) * s.y + (x[16 + c] + x[20 + c]) * s.z;
    }
    int rank[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int r = 0;
#pragma unroll
      for (int d = 0; d < 4; ++d)
        if (d != c && (key[d] > key[c] || (key[d] == key[c] && (pk[d] > pk[c] || (pk[d] == pk[c] && d < c))))) ++r;
      rank[c] = r;
    }
#pragma unroll
    for (int q = 0; q < 7; ++q)
#pragma unroll
      for (int c = 0; c < 4; ++c) f[4 * q + rank[c]] = x[4 * q + c];
  }
}

void launch_sun_order4(float4* nodes4, uint32_t n, float3 sun, int sms, cudaStream_t st) {
  if (n == 0) return;
  const uint32_t grid = std::min<uint32_t>((n + 255) / 256, (uint32_t)sms * 8);
  k_sun_order4<<<grid, 256, 0, st>>>(nodes4, n, sun);
}

void launch_l2_probe(const float4* buf, size_t n4, int iters, float* sink, cudaStream_t st, int sms) {
  k_l2_probe<<<sms * 4, 512, 0, st>>>(buf, n4, iters, sink);
}

int trace_blocks_per_sm(int block) {
  int a = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_trace<true, false, 3>, block, 0);
  return a > 0 ? a : 1;
}

int shadow_blocks_per_sm(int block) {
  int a = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_shadow<false, false, 3>, block, 0);
  return a > 0 ? a : 1;
}

int num_sms(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
  return v;
}

}  // namespace srt

// rt_render_static: the render entry point for callers that must not
// allocate device memory.
//
// Some host programs cannot call cudaMalloc while they render: an
// application whose framework has already reserved the device memory for its
// own pool, a process held to a fixed memory budget, or a latency-sensitive
// loop that cannot afford the implicit device synchronisation that
// cudaMalloc / cudaFree may cause.  This entry point computes exactly what
// rt_render computes, but takes every byte of working memory (ray queues,
// hit records, sun-ray queue, per-path radiance, counters, status word and
// camera table) from one fixed array compiled into the library, and calls no
// allocating routine.  The caller passes the inputs (through the context's
// scene and spectra) and the outputs.
//
// The array is a file-scope __device__ variable of kStaticBytes; every GPU
// that loads the library holds it until the process exits.  Host code cannot
// use the array's name as a device address, so the first call on each device
// looks the address up with cudaGetSymbolAddress (with that device current)
// and caches it.  Make that first call before any stream capture begins.
// All calls share the array and it keeps the previous call's contents; the
// counters and the status word are cleared at the start of every call.  Two
// calls whose work overlaps on the GPU (different streams, or different
// contexts on one device) race on the array and give wrong results.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/spectral_rt.h"
#include "rt_internal.h"

using namespace srt;

namespace {

// Paths in flight per wave when working from the static array.
constexpr uint32_t kStaticWave = 1u << 19;
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffQ0 = 0;
constexpr size_t kOffQ1 = kOffQ0 + align256((size_t)kStaticWave * 2 * sizeof(float4));
constexpr size_t kOffHit = kOffQ1 + align256((size_t)kStaticWave * 2 * sizeof(float4));
constexpr size_t kOffSq = kOffHit + align256((size_t)kStaticWave * sizeof(float2));
constexpr size_t kOffL = kOffSq + align256((size_t)kStaticWave * 2 * sizeof(float4));
constexpr size_t kOffSig = kOffL + align256((size_t)kStaticWave * sizeof(float));
constexpr size_t kOffCnt = kOffSig + align256((size_t)kStaticWave * sizeof(uint32_t));
constexpr size_t kOffTot = kOffCnt + align256(sizeof(Counters) * (kMaxDepth + 2));
constexpr size_t kOffStatus = kOffTot + align256(sizeof(Totals));
constexpr size_t kOffCams = kOffStatus + align256(sizeof(uint32_t));
constexpr size_t kStaticBytes = kOffCams + align256(sizeof(DevCam) * kMaxCams);
static_assert(kStaticBytes < (64ull << 20), "static scratch stays below 64 MiB");

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {nullptr};

// Device address of the array on `device` (current), looked up once.
cudaError_t scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_addr[device] = (unsigned char*)p;
  }
  *out = g_addr[device];
  return cudaSuccess;
}

rt_status err(rt_ctx* c, rt_status s, const std::string& m, bool fatal = false) {
  ctx_error(c, m.c_str(), fatal);
  return s;
}

}  // namespace

extern "C" rt_status rt_render_static(rt_ctx* c, const rt_camera* cams, uint32_t n_cams, uint32_t band_first,
                                      uint32_t band_count, uint32_t spp, uint32_t depth, uint64_t seed,
                                      uint32_t xyz_mode, double* spectral_dev, float* xyz_dev) {
  CtxView v;
  if (!c) return RT_ERR_ARG;
  if (!ctx_view(c, &v)) return RT_ERR_STATE;
  if (!v.has_scene || !v.has_spectra) return err(c, RT_ERR_STATE, "rt_render_static: scene and spectra must be set");
  if (!spectral_dev) return err(c, RT_ERR_ARG, "rt_render_static: spectral_dev (the FP64 accumulator) is required");
  if (!cams || n_cams == 0 || n_cams > (uint32_t)kMaxCams)
    return err(c, RT_ERR_ARG, "rt_render_static: 1..64 cameras (the camera table lives in the static array)");
  if (band_count == 0 || band_first + band_count > v.P.n_bands || band_first + band_count < band_first)
    return err(c, RT_ERR_ARG, "rt_render_static: band range outside the spectra");
  if (spp == 0) return err(c, RT_ERR_ARG, "rt_render_static: spp must be >= 1");
  if (depth == 0 || depth > (uint32_t)kMaxDepth)
    return err(c, RT_ERR_ARG, "rt_render_static: depth must be 1..64 (counter rows in the static array)");
  if (xyz_mode > 2) return err(c, RT_ERR_ARG, "rt_render_static: unknown xyz_mode");
  if (xyz_mode != 2 && band_count > kXyzMaxBandsTc)
    return err(c, RT_ERR_ARG, "rt_render_static: tensor-core XYZ takes at most 192 bands (use RT_XYZ_FP64)");
  if (((uintptr_t)spectral_dev & 15u) != 0)
    return err(c, RT_ERR_ARG, "rt_render_static: spectral_dev must be 16-byte aligned");
  uint64_t npix = 0;
  const char* why = "";
  if (!build_dev_cams(cams, n_cams, v.h_cams, &npix, &why)) return err(c, RT_ERR_ARG, std::string("rt_render_static: ") + why);
  const uint64_t PB64 = npix * band_count;
  if (PB64 >= (1ull << 32)) return err(c, RT_ERR_ARG, "rt_render_static: pixels x bands must be below 2^32");

  if (cudaSetDevice(v.device) != cudaSuccess) return err(c, RT_ERR_CUDA, "rt_render_static: cudaSetDevice", true);
  unsigned char* base = nullptr;
  cudaError_t ce = scratch_address(v.device, &base);
  if (ce != cudaSuccess)
    return err(c, RT_ERR_CUDA, std::string("rt_render_static: cudaGetSymbolAddress: ") + cudaGetErrorString(ce), true);
  const cudaStream_t st = v.stream;
  const uint32_t PB = (uint32_t)PB64;
  const uint32_t cap = PB < kStaticWave ? PB : kStaticWave;
  WaveBufs b{};
  b.q[0] = (float4*)(base + kOffQ0);
  b.q[1] = (float4*)(base + kOffQ1);
  b.hit = (float2*)(base + kOffHit);
  b.sq = (float4*)(base + kOffSq);
  b.L = (float*)(base + kOffL);
  b.sig = (uint32_t*)(base + kOffSig);
  b.cnt = (Counters*)(base + kOffCnt);
  b.tot = (Totals*)(base + kOffTot);
  b.status = (uint32_t*)(base + kOffStatus);
  b.cap = cap;
  DevCam* d_cams = (DevCam*)(base + kOffCams);

#define STATIC_TRY(call)                                                                              \
  do {                                                                                                \
    const cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                            \
      return err(c, RT_ERR_CUDA, std::string("rt_render_static: " #call ": ") + cudaGetErrorString(e_), true); \
  } while (0)

  STATIC_TRY(cudaMemcpyAsync(d_cams, v.h_cams, sizeof(DevCam) * n_cams, cudaMemcpyHostToDevice, st));
  STATIC_TRY(cudaMemsetAsync(spectral_dev, 0, PB64 * sizeof(double), st));
  STATIC_TRY(cudaMemsetAsync(b.status, 0, sizeof(uint32_t), st));
  STATIC_TRY(cudaMemsetAsync(b.tot, 0, sizeof(Totals), st));
  LaunchCfg lc;
  lc.block_trace = 128;
  lc.block_shade = 256;
  lc.grid_trace = v.sms * trace_blocks_per_sm(lc.block_trace);
  lc.grid_shadow = v.sms * shadow_blocks_per_sm(lc.block_trace);
  lc.grid_shade = v.sms * 8;
  lc.counting = false;
  lc.record = false;
  lc.variant = 0;
  lc.leaf_min = kDefaultLeafBatch;
  lc.sort_rays = false;  // the static scratch holds no sort buffers; ray order changes no result
  lc.trace_steps = kDefaultTraceSteps;
  lc.trace_refill = kDefaultTraceRefill;
  lc.shadow_steps = kDefaultShadowSteps;
  lc.shadow_refill = kDefaultShadowRefill;
  const Probe probe{nullptr, nullptr, nullptr};
  WaveParams w{};
  w.PB = PB;
  w.band_first = band_first;
  w.band_count = band_count;
  w.spp = spp;
  w.depth = depth;
  w.key0 = (uint32_t)seed;
  w.key1 = (uint32_t)(seed >> 32);
  w.nb = 1;
  w.B = band_count;
  w.acc_stride = band_count;
  w.acc_off = 0;
  const uint64_t total = PB64 * spp;
  for (uint64_t ws = 0; ws < total; ws += cap) {
    w.n = (uint32_t)((total - ws) < cap ? (total - ws) : cap);
    w.s0 = (uint32_t)(ws / PB);
    w.r0 = (uint32_t)(ws % PB);
    STATIC_TRY(cudaMemsetAsync(b.cnt, 0, sizeof(Counters) * (depth + 2), st));
    launch_wave(lc, v.S, v.P, d_cams, n_cams, w, b, spectral_dev, probe, st, nullptr, nullptr);
  }
  STATIC_TRY(cudaGetLastError());
  if (xyz_dev) {
    XyzWeights xw;
    xw.w32 = v.cmfw + 3 * (size_t)band_first;
    xw.band_count = band_count;
    xw.kpad = (band_count + 15) / 16 * 16;
    launch_xyz(spectral_dev, npix, xw, spp, (int)xyz_mode, xyz_dev, st, b.status, v.sms);
    STATIC_TRY(cudaGetLastError());
  }
  STATIC_TRY(cudaMemcpyAsync(v.h_status, b.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  STATIC_TRY(cudaStreamSynchronize(st));
#undef STATIC_TRY
  const uint32_t s = *v.h_status;
  if (s == 0) return RT_OK;
  if (s & ST_STACK) return err(c, RT_ERR_STACK, "rt_render_static: BVH traversal stack exhausted");
  if (s & ST_ITER) return err(c, RT_ERR_TIMEOUT, "rt_render_static: device loop reached its iteration cap");
  if (s & ST_QUEUE) return err(c, RT_ERR_QUEUE_OVERFLOW, "rt_render_static: device work queue overflow");
  return err(c, RT_ERR_CUDA, "rt_render_static: device range check failed");
}

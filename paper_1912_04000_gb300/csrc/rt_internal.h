// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/spectral_rt.h"

namespace srt {

// device status word bits (set by kernels, read by the host after a render)
enum : uint32_t {
  ST_STACK = 1u,      // traversal stack exhausted
  ST_QUEUE = 2u,      // work queue overflow
  ST_ITER = 4u,       // traversal iteration cap
  ST_RANGE = 8u       // index out of range caught by a device check
};

constexpr int kStack = 96;             // traversal stack entries per thread
constexpr uint32_t kPidBits = 24;      // path id bits in a queue entry
constexpr uint32_t kPidMask = (1u << kPidBits) - 1u;
constexpr uint32_t kFlagCovered = 1u << 31;  // direct sun already estimated by NEE
constexpr uint32_t kFlagTerm = 1u << 30;     // shadow ray: path ends at this vertex
constexpr uint32_t kFlagGuidedEsc = 1u << 29;  // sun reached by escape counts with MIS weight wesc[pid]
constexpr uint32_t kMaxWave = 1u << kPidBits;

// Scene on the device.
// nodes: 2 float4 per node {lo.xyz, bits(ref)}, {hi.xyz, bits(count)}; node 1
//   is the root; the children of an interior node sit at an even index pair
//   (ref, ref + 1), 64-byte aligned; a leaf has count in [1, 7] triangles
//   starting at triangle ref.
// tris: 3 float4 per triangle in leaf order {v0, bits(input id)},
//   {v1, bits(material)}, {v2, 0}.
// nrm: per leaf-order triangle {unit geometric normal (FP64-rounded),
//   bits(material)}.
struct DevScene {
  const float4* nodes;   // binary BVH: 2 float4 per node, node 1 the root
  const float4* nodes4;  // four-wide BVH: 8 float4 per node, node 0 the root
  const float4* nodes8;  // eight-wide BVH: 14 float4 per node, node 0 the root (host builds; else null)
  const float4* nodes4q;  // the four-wide BVH with 8-bit child boxes: 4 float4 per node (host builds; else null)
  const float4* tris;
  const float4* nrm;
  uint32_t n_nodes;
  uint32_t n_nodes4;
  uint32_t n_nodes8;
  uint32_t n_tris;
  float blo[3], binv[3];  // scene box: lower corner and 1 / extent per axis
  float eps;  // origin offset along the normal: 1e-4 x scene diagonal
  uint32_t iter_cap;  // traversal steps per ray before ST_ITER; 0 = 4 x binary nodes + 64
};

// Spectral tables on the device.
// mb: per (material, band) {n, k, rho, le}; ad: per (material, band)
// 4 pi k d / lambda (thin glass, FP64-rounded); mtype per material.
struct DevSpectra {
  const float4* mb;
  const float* ad;
  const int* mtype;
  const float* sunL;
  uint32_t n_bands;
  uint32_t n_mat;
  float3 sun;
  float cos_max;
  float one_minus_cos;  // 1 - cos(half angle), FP64-rounded
};

// One camera in device form (FP64-derived basis).
struct DevCam {
  float3 pos, f, r, u;
  float tha, th;        // tan(vfov/2) * aspect, tan(vfov/2)
  uint32_t W, H;
  uint32_t offset;      // first global pixel id of this view
  uint32_t pad;
};

constexpr int kMaxCams = 64;

// One wave: paths [wave_start, wave_start + n) of the index space
// g = s * PB + r, r = pixel * band_count + j, PB = pixels * band_count.
struct WaveParams {
  uint32_t n;          // paths in this wave
  uint32_t s0, r0;     // sample and in-sample index of the first path
  uint32_t PB;         // pixels * band_count
  uint32_t band_first, band_count;
  uint32_t spp, depth;
  uint32_t key0, key1;
  uint32_t s_base;     // first sample index of the render call (probe rows)
  uint32_t n_bands;    // bands of the spectra (guide band groups)
  // bands carried per path: 1, or 4 (band_count = G = ceil(B / 4) units
  // per pixel; unit j stands for bands band_first + j + q G, q = 0..3, those
  // below B, the render's band count); with 1, B = band_count
  uint32_t nb, B;
  // one-band paths add to accum[pixel * acc_stride + acc_off + j] (a band
  // chunk of a wider spectral image; acc_stride = band_count, acc_off = 0
  // for a whole render)
  uint32_t acc_stride, acc_off;
};

// Guided sampling of one wave (on == false: plain cosine sampling).
// gq: guide queries, 3 float4 each: {origin, bits(pid | flags)}, {normal,
//   throughput}, {rho, bits(sun-ray slot or 0xFFFFFFFF), 0, 0}.
// At a guided vertex the direct sun is estimated by two strategies combined
// with the balance heuristic: next-event sampling of the sun cone (weight
// p_cone / (p_cone + p_mix)) and the guided continuation escaping into the
// cone (weight p_mix / (p_cone + p_mix), kept per path in wesc).
// raw: training slots (collect != 0), one per (guided vertex v, path id with
//   pid % collect == 0) at (v - 1) * slots_per_vertex + pid / collect, 6
//   float4: {origin, group}, {normal, radiance before vertex v + 1},
//   {omega, MIS pdf}, {cos, throughput after v, valid, pid},
//   {sun sample direction, cos}, {sun radiance x transmittance, p_cone, valid, 0}.
constexpr uint32_t kRawF4 = 6;
struct GuideWave {
  bool on;
  uint32_t depth;
  float alpha;
  float4* gq;
  float* wesc;    // per path id: MIS weight of a sun escape after a guided vertex
  uint32_t collect;
  uint32_t slots_per_vertex;
  float4* raw;
  float* Lfinal;  // final radiance per path id (collect != 0)
  // spatial order of the queries (null: queue order): perm[j] = query index
  // of the j-th query in Morton order of a 64^3 grid over the scene box;
  // skey[i] = cell of query i; bins = per-cell counts, then cursors within
  // chunks of 1024 cells, followed by the chunks' offsets
  uint32_t* perm;
  uint32_t* skey;
  uint32_t* bins;
};
constexpr uint32_t kGuideSortBits = 6;  // cells per axis = 2^6
constexpr uint32_t kGuideSortBins = 1u << (3 * kGuideSortBits);
constexpr uint32_t kCellSortBins = kGuideSortBins;  // 2^18 keys for every cell sort
// Exclusive scan of kCellSortBins counts in place, chunk offsets after them
// (rt_kernels.cu).
void launch_cell_scan(uint32_t* bins, cudaStream_t st);
// The same for n counts (n a multiple of 32768, at most 2^20): data[i] becomes
// the exclusive prefix within its chunk of 1024, data[n + c] the exclusive
// prefix of chunk c's total.
void launch_scan(uint32_t* data, size_t n, cudaStream_t st);

// Device BVH builder (rt_lbvh.cu).
constexpr uint32_t kLbvhMaxTris = 1u << 24;
size_t lbvh_scratch_bytes(uint32_t n);
void launch_lbvh(const float* verts, const uint32_t* tri, uint32_t n, const float lo[3], const float hi[3], float pad,
                 const float4* tri_in, const float4* nrm_in, void* scratch, float4* nodes4, float4* tri_out,
                 float4* nrm_out, uint32_t** counts_out, int sms, cudaStream_t st);
constexpr int kLbvhLevels = 64;
// Stable LSD radix sort of (key, value) pairs by the low key_bits bits, 8
// bits per pass (rt_lbvh.cu): keys[0] / vals[0] in, the result in
// keys[r] / vals[r] for the returned r; n <= 2^24; hist holds
// radix_sort_hist_words(n) words.
size_t radix_sort_hist_words(uint32_t n);
int launch_radix_sort(uint32_t* keys[2], uint32_t* vals[2], uint32_t n, uint32_t key_bits, uint32_t* hist,
                      cudaStream_t st);
  // collapse levels launched (counts has 2 + kLbvhLevels entries)

// Per-wave device counters, one row per vertex k (0 .. depth).
struct Counters {
  uint32_t q_count;     // rays queued for vertex k
  uint32_t q_fetch;     // traversal work fetch
  uint32_t s_count;     // shadow rays emitted at vertex k
  uint32_t s_fetch;
  uint32_t g_count;     // guide queries emitted at vertex k
  uint32_t g_pad;
};

struct Totals {
  unsigned long long ext_rays, shadow_rays, nodes, tris, snodes, stris;
};

// Per-stage CUDA-event timing of a render (host side, optional).
enum Stage { STG_CAMERA = 0, STG_TRACE = 1, STG_SHADE = 2, STG_SHADOW = 3, STG_XYZ = 4, STG_GUIDE = 5, STG_TRAIN = 6,
             STG_N = 7 };
struct StageTimer {
  virtual void begin(int stage, cudaStream_t st) = 0;
  virtual void end(int stage, cudaStream_t st) = 0;
  virtual ~StageTimer() {}
};

// Work buffers of one wave (capacity C paths).
struct WaveBufs {
  float4* q[2];         // ray queues, 2 float4 each: {o, bits(pid|flags)}, {d, T}
  float2* hit;          // {t, bits(leaf-order triangle or -1)}
  float4* sq;           // shadow queue, 2 float4 each: {o, bits(pid|flags)}, {w, contrib}
  float* L;             // accumulated radiance per path id
  uint32_t* sig;        // event signature per path id (record mode)
  Counters* cnt;        // [kMaxDepth + 2]
  Totals* tot;
  uint32_t* status;
  uint32_t cap;
  // spatial order of the ray queues (null: queue order): rperm[j] = queue
  // slot of the j-th ray in cell order; rkey = cell per slot; rbins as the
  // guide-query bins (kCellSortBins counts, then kCellSortBins / 1024 offsets)
  uint32_t* rperm;
  uint32_t* rkey;
  uint32_t* rbins;
  // four bands per path: radiance, throughput and the pending sun-ray
  // contribution per path id and band
  float4* L4;
  float4* T4;
  float4* C4;
};

constexpr int kMaxDepth = 64;

struct Probe {
  const uint32_t* map;  // per global pixel: probe slot or 0xFFFFFFFF
  float* L;
  uint32_t* sig;
};

// Default traversal loop parameters (set from measurements on a GB300).
constexpr int kDefaultTraceSteps = 4, kDefaultTraceRefill = 8;
constexpr int kDefaultShadowSteps = 4, kDefaultShadowRefill = 12;
constexpr int kDefaultLeafBatch = 24;

// Launchers (rt_kernels.cu).
struct LaunchCfg {
  int grid_trace, block_trace;  // block_trace also sizes the sun-ray kernel's blocks
  int grid_shadow;
  int grid_shade, block_shade;
  bool counting;
  bool record;
  int variant;  // traversal: 0 = four-wide, leaf batching; binary: 1 = while-while, 2 = node-or-leaf steps,
                // 3 = leaf batching
  bool sort_rays;  // reorder the vertex >= 2 and sun-ray queues by cell (needs b.rperm)
  int leaf_min;  // variant 2: lanes waiting at a leaf that start a leaf phase
  int trace_steps, trace_refill;    // closest hit: steps between refill checks, refill threshold
  int shadow_steps, shadow_refill;  // sun rays: the same
};

struct GuideDev;
struct PhotonMaps;
// pm != nullptr: photon-mapping camera pass (paths end at their first
// Lambertian vertex with the sun's next-event estimate and the photon
// density estimates of pm)
void launch_wave(const LaunchCfg& lc, const DevScene& S, const DevSpectra& P, const DevCam* cams, uint32_t n_cams,
                 const WaveParams& w, const WaveBufs& b, double* accum, const Probe& probe,
                 cudaStream_t st, int* launches, StageTimer* timer, const GuideWave* gw = nullptr,
                 const GuideDev* gdev = nullptr, const void* gpack = nullptr, int sms = 0,
                 const PhotonMaps* pm = nullptr);
// Sorts the children of the n four-wide nodes far-to-near along the sun
// (the visit order of sun rays).
void launch_sun_order4(float4* nodes4, uint32_t n, float3 sun, int sms, cudaStream_t st);
void launch_l2_probe(const float4* buf, size_t n4, int iters, float* sink, cudaStream_t st, int sms);
void launch_philox(const uint32_t* ctr, uint32_t* out, uint64_t n, uint32_t k0, uint32_t k1, cudaStream_t st);
void launch_trace_closest_rays(const DevScene& S, const float* o, const float* d, uint64_t n, float* t,
                               int32_t* prim, uint32_t* status, cudaStream_t st);
void launch_trace_shadow_rays(const DevScene& S, const DevSpectra& P, const float* o, const float* d,
                              const uint32_t* band, uint64_t n, float* T, uint32_t* n_glass, uint32_t* status,
                              cudaStream_t st);
void launch_optics(const float* c, const float* n, const float* k, const float* lam, const float* d,
                   uint64_t count, float* R, float* Rs, float* Ts, cudaStream_t st);

// XYZ contraction (rt_xyz.cu).  The kernels split the FP32 weights into
// their BF16 operand tiles themselves.
struct XyzWeights {
  const float* w32;        // [band_count][3] float
  uint32_t band_count;
  uint32_t kpad;           // band_count rounded up to 16
};
// Tensor-core modes keep all K-slices of a 128-pixel tile in shared memory:
// at most kXyzMaxBandsTc bands.
constexpr uint32_t kXyzMaxBandsTc = 192;
void launch_xyz(const double* spectral, uint64_t n_pixels, const XyzWeights& w, uint32_t spp, int mode, float* xyz,
                cudaStream_t st, uint32_t* status, int sms);

int num_sms(int device);
// Photon mapping (section 4; rt_photon.cu, kernels in rt_kernels.cu).
// Photon pass over bands band0 .. band0 + Bc - 1, N photons per band: slot
// (j * N + i) * depth + n holds the n-th diffuse hit of photon i of band
// band0 + j as {x, y, z, flux}; its sort key is kPhotonEmpty, or for a
// caustic (map 0) or indirect (map 1) photon ((map * Bc + j) << hbits) |
// hash of its cell (cells of edge 2 r of the map).
constexpr uint32_t kPhotonEmpty = 0xFFFFFFFFu;
constexpr uint32_t kPhotonMaxSlots = 1u << 24;
struct PhotonPass {
  uint32_t band0, Bc, N, depth;
  uint32_t key0, key1;       // Philox key of the photon pass
  float3 c0, t1, t2;         // emission disk: centre and basis (t1, t2 span the disk)
  float Rd, flux;            // disk radius; Omega pi Rd^2 / N
  float inv_cell[2];         // 1 / (2 r) of the caustic and indirect maps
  uint32_t hbits;            // 2^hbits hash cells per (map, band)
  // emission 1: photons start on the thin-glass portals facing the sun:
  // portal[4 q ..] = {v0, v1, v2, (sun-side normal, 1 / (s . n))}, cdf the
  // cumulative share of A |s . n|; flux then holds Omega W / N
  uint32_t emission, n_portal;
  const float4* portal;
  const float* cdf;
};
// The maps after sorting: rec holds the records in key order; start / end
// the record range of each key (empty: start = end = 0).
struct PhotonMaps {
  const uint32_t* start;
  const uint32_t* end;
  const float4* rec;
  float r2[2], inv_cell[2], norm[2];  // r^2, 1 / (2 r), 2 / (pi r^2) per map (Epanechnikov kernel)
  uint32_t hbits, Bc;
};
void launch_photon_trace(const DevScene& S, const DevSpectra& P, const PhotonPass& pp, float4* rec, uint32_t* keys,
                         uint32_t* vals, uint8_t* cls, uint32_t* status, int sms, cudaStream_t st);
void launch_photon_maps(const uint32_t* sorted_keys, const uint32_t* sorted_vals, uint32_t n, const float4* rec,
                        float4* rec_sorted, uint32_t* start, uint32_t* end, int sms, cudaStream_t st);
int trace_blocks_per_sm(int block);
int shadow_blocks_per_sm(int block);

// Learned guide (rt_guide.cu).
// Hash grid: kGuideLevels levels of kGuideFeatures features per entry.
constexpr int kGuideLevels = 8, kGuideFeatures = 4;
struct GuideDev {
  const float* grid;      // [kGuideLevels][2^log2T][kGuideFeatures] FP32
  uint32_t log2T;
  uint32_t res[kGuideLevels];  // grid resolution per level
  uint32_t dense_mask;    // bit l: level l indexed densely
  float lo[3], inv_ext[3];
};
size_t guide_eval_smem();
size_t guide_train_smem();
uint32_t guide_wsize();
uint32_t guide_wpack_bytes();
void launch_guide_init(float* grid, uint64_t n_grid, float* W, uint64_t seed, cudaStream_t st);
void launch_guide_pack(const float* W, void* pack, cudaStream_t st);
void launch_guide_eval(const GuideDev& g, const void* pack, const float* rec, uint64_t n, float* Y, float* q,
                       uint32_t* status, int sms, cudaStream_t st);
// dWpart: sms x 15360 floats of per-CTA partial weight gradients (scratch)
void launch_guide_train(const GuideDev& g, const void* pack, const float* rec, uint64_t n, float* wsum, float* dW,
                        float* dWpart, float* dgrid, float* loss, uint32_t* status, int sms, cudaStream_t st);
void launch_adam(float* p, const float* g, float* m, float* v, uint64_t n, float lr, float b1, float b2, float eps,
                 float c1, float c2, cudaStream_t st);
void launch_guide_sample(const GuideDev& g, const void* pack, const DevSpectra& P, const WaveParams& w, uint32_t k,
                         const GuideWave& gw, const WaveBufs& b, double* accum, const Probe& probe, bool record,
                         int sms, cudaStream_t st);
// Two training records per slot (continuation, sun sample): 2 * n_slots.
void launch_guide_records(const GuideWave& gw, uint32_t n_slots, uint32_t perm_mul, float* train_rec, cudaStream_t st);
// rt_guide_sample_step: caller vertices (rt_guide_vertex, 64 B each) into the
// guide queries and sun samples of a wave; and the step's outputs gathered
// per vertex (rt_guide_step_out, 48 B each).
void launch_guide_step_pack(const void* v, uint32_t n, float4* gq, float4* sq, cudaStream_t st);
void launch_guide_step_gather(const void* v, uint32_t n, uint32_t k, const GuideWave& gw, const WaveBufs& b, void* out,
                              cudaStream_t st);

// Cameras in device form (basis derived in FP64) into out[0 .. n_cams);
// *npix = pixels over all views; false with the reason in *why on a bad
// camera (rt_api.cu).
bool build_dev_cams(const rt_camera* cams, uint32_t n_cams, DevCam* out, uint64_t* npix, const char** why);

// Read-only view of a context for entry points defined outside rt_api.cu.
struct CtxView {
  int device;
  cudaStream_t stream;
  bool has_scene, has_spectra;
  DevScene S;
  DevSpectra P;
  const float* cmfw;     // device [n_bands][3]
  int sms;
  DevCam* h_cams;        // pinned staging, kMaxCams entries
  uint32_t* h_status;    // pinned
};
}  // namespace srt
struct rt_ctx;
namespace srt {
// Fills *v; returns false for a null or poisoned context.
bool ctx_view(rt_ctx* c, CtxView* v);
// Records an error message on the context (and poisons it when fatal).
void ctx_error(rt_ctx* c, const char* msg, bool fatal);

}  // namespace srt

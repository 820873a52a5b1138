// C ABI of the spectral path tracer: context, scene and spectra upload,
// render orchestration (wave loop), single-step entry points.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/spectral_rt.h"
#include "rt_bvh.h"
#include "rt_internal.h"

using namespace srt;

struct rt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  bool poisoned = false;
  bool counting = false;
  int sms = 0;
  // diagnostic limits (rt_set_limits; 0 = off): ray-queue capacity, traversal
  // steps per ray, and the countdown to an injected CUDA failure
  uint32_t lim_queue = 0, lim_steps = 0, fail_countdown = 0;
  int occ_trace = 0;
  int occ_shade = 0;
  // scene
  float4* d_nodes = nullptr;
  float4* d_nodes4 = nullptr;
  float4* d_nodes8 = nullptr;
  float4* d_nodes4q = nullptr;  // four-wide nodes with 8-bit quantised child boxes (4 float4 each)
  float4* d_tris = nullptr;
  float4* d_nrm = nullptr;
  uint32_t n_nodes = 0, n_nodes4 = 0, n_nodes8 = 0, n_tris = 0, n_mat = 0;
  float eps = 0.0f;
  bool has_scene = false;
  uint32_t builder = 2;       // BVH builder for the next rt_load_scene: 0 host SAH, 1 device LBVH,
                              // 2 host SAH with spatial splits (default)
  uint32_t builder_used = 0;  // builder of the loaded scene
  float build_ms = 0.0f;      // its build time
  // spectra
  float4* d_mb = nullptr;
  float* d_ad = nullptr;
  int* d_mtype = nullptr;
  float* d_sunL = nullptr;
  float* d_cmfw = nullptr;
  DevSpectra sp{};
  std::vector<float> cmf_w;
  std::vector<int> mtype;
  std::vector<float> mthick;
  bool has_spectra = false;
  // per-render buffers
  WaveBufs wb{};
  uint32_t wave_alloc = 0;
  uint32_t four_band_alloc = 0;
  std::vector<float> glass;  // thin-glass triangles of the scene, 9 floats each, input order
  // sun direction and cone in FP64 (photon emission geometry)
  double sun_d[3] = {0.0, 0.0, 1.0};
  double cos_max_d = 1.0;
  // photon-mapping buffers: slot records, sort keys and values (two
  // copies), radix histogram, records in key order, per-key ranges
  struct {
    float4* rec = nullptr;
    float4* rec_sorted = nullptr;
    uint32_t* keys[2] = {nullptr, nullptr};
    uint32_t* vals[2] = {nullptr, nullptr};
    uint32_t* hist = nullptr;
    size_t slots = 0;
    uint32_t* start = nullptr;
    uint32_t* end = nullptr;
    size_t table = 0;
  } ph;
  DevCam* d_cams = nullptr;
  DevCam* h_cams = nullptr;  // pinned staging
  double* d_accum = nullptr;
  size_t accum_cap = 0;
  float* d_xyz = nullptr;
  size_t xyz_cap = 0;
  uint32_t* h_status = nullptr;  // pinned
  Totals* h_tot = nullptr;       // pinned
  uint32_t* d_status_aux = nullptr;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool timing = false;
  std::vector<cudaEvent_t> tpool;
  // captured render (rt_render_opts.use_graph)
  cudaStream_t gstream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  std::string graph_key;
  int graph_launches = 0;
  uint32_t graph_waves = 0;
  float lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};  // scene bounds
  // learned guide
  struct Guide {
    bool init = false;
    rt_guide_config cfg{};
    float *grid = nullptr, *W = nullptr, *mg = nullptr, *vg = nullptr, *mW = nullptr, *vW = nullptr;
    float *dgrid = nullptr, *dW = nullptr, *scratch = nullptr;  // scratch: wsum, loss
    float* dWpart = nullptr;  // per-CTA partial weight gradients, sms x weights
    void* pack = nullptr;
    uint64_t n_grid = 0;
    uint32_t step = 0;
    GuideDev dev{};
    // guided rendering buffers
    float4* gq = nullptr;
    float* wesc = nullptr;
    uint32_t* perm = nullptr;
    uint32_t* skey = nullptr;
    uint32_t* bins = nullptr;
    uint32_t gq_cap = 0;
    float4* raw = nullptr;
    float* Lfinal = nullptr;
    float* trec = nullptr;
    uint64_t raw_cap = 0;
  } guide;
};

namespace {

rt_status fail(rt_ctx* c, rt_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

// An injected failure (rt_set_limits) stands for the checked call, which is
// then not made.
bool injected_failure(rt_ctx* c) { return c->fail_countdown != 0 && --c->fail_countdown == 0; }

#define CUDA_TRY(ctx, call)                                                                    \
  do {                                                                                         \
    cudaError_t e_ = injected_failure(ctx) ? cudaErrorUnknown : (call);                        \
    if (e_ != cudaSuccess) {                                                                   \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                         \
      if (e_ != cudaErrorMemoryAllocation) (ctx)->poisoned = true;                             \
      return e_ == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA;                       \
    }                                                                                          \
  } while (0)

template <class T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// Frees a temporary device buffer when the scope ends, error paths included.
template <class T>
struct DevTemp {
  T* p = nullptr;
  ~DevTemp() { dfree(p); }
};

rt_status check_ctx(rt_ctx* c) {
  if (!c) return RT_ERR_ARG;
  if (c->poisoned) return fail(c, RT_ERR_STATE, "context unusable after a CUDA error: " + c->err);
  return RT_OK;
}

rt_status ensure_wave(rt_ctx* c, uint32_t cap) {
  if (c->wave_alloc >= cap) return RT_OK;
  WaveBufs& b = c->wb;
  dfree(b.q[0]);
  dfree(b.q[1]);
  dfree(b.hit);
  dfree(b.sq);
  dfree(b.L);
  dfree(b.sig);
  dfree(b.rperm);
  dfree(b.rkey);
  c->wave_alloc = 0;
  CUDA_TRY(c, cudaMalloc(&b.q[0], (size_t)cap * 2 * sizeof(float4)));
  CUDA_TRY(c, cudaMalloc(&b.q[1], (size_t)cap * 2 * sizeof(float4)));
  CUDA_TRY(c, cudaMalloc(&b.hit, (size_t)cap * sizeof(float2)));
  CUDA_TRY(c, cudaMalloc(&b.sq, (size_t)cap * 2 * sizeof(float4)));
  CUDA_TRY(c, cudaMalloc(&b.L, (size_t)cap * sizeof(float)));
  CUDA_TRY(c, cudaMalloc(&b.sig, (size_t)cap * sizeof(uint32_t)));
  CUDA_TRY(c, cudaMalloc(&b.rperm, (size_t)cap * sizeof(uint32_t)));
  CUDA_TRY(c, cudaMalloc(&b.rkey, (size_t)cap * sizeof(uint32_t)));
  if (!b.rbins)
    CUDA_TRY(c, cudaMalloc(&b.rbins, (size_t)(kCellSortBins + kCellSortBins / 1024u) * sizeof(uint32_t)));
  b.cap = cap;
  c->wave_alloc = cap;
  return RT_OK;
}

// Per-path four-band state (radiance, throughput, pending sun-ray
// contribution), allocated on the first render that asks for it.
rt_status ensure_four_band(rt_ctx* c, uint32_t cap) {
  if (c->four_band_alloc >= cap) return RT_OK;
  WaveBufs& b = c->wb;
  dfree(b.L4);
  dfree(b.T4);
  dfree(b.C4);
  c->four_band_alloc = 0;
  CUDA_TRY(c, cudaMalloc(&b.L4, (size_t)cap * sizeof(float4)));
  CUDA_TRY(c, cudaMalloc(&b.T4, (size_t)cap * sizeof(float4)));
  CUDA_TRY(c, cudaMalloc(&b.C4, (size_t)cap * sizeof(float4)));
  c->four_band_alloc = cap;
  return RT_OK;
}

DevScene dev_scene(const rt_ctx* c) {
  DevScene S;
  S.nodes = c->d_nodes;
  S.nodes4 = c->d_nodes4;
  S.nodes8 = c->d_nodes8;
  S.nodes4q = c->d_nodes4q;
  S.tris = c->d_tris;
  S.nrm = c->d_nrm;
  S.n_nodes = c->n_nodes;
  S.n_nodes4 = c->n_nodes4;
  S.n_nodes8 = c->n_nodes8;
  for (int a = 0; a < 3; ++a) {
    S.blo[a] = c->lo[a];
    const float ext = c->hi[a] - c->lo[a];
    S.binv[a] = ext > 0.0f ? 1.0f / ext : 0.0f;
  }
  S.n_tris = c->n_tris;
  S.eps = c->eps;
  S.iter_cap = c->lim_steps;
  return S;
}

rt_status status_to_rt(rt_ctx* c, uint32_t st) {
  if (st == 0) return RT_OK;
  if (st & ST_STACK) return fail(c, RT_ERR_STACK, "BVH traversal stack exhausted");
  if (st & ST_ITER) return fail(c, RT_ERR_TIMEOUT, "device loop reached its iteration cap");
  if (st & ST_QUEUE) return fail(c, RT_ERR_QUEUE_OVERFLOW, "device work queue overflow");
  return fail(c, RT_ERR_CUDA, "device range check failed");
}

bool finite3(const float* p) { return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]); }

// Brackets launches with events from the context's pool; sums per stage
// after the stream has been synchronised.
struct EvTimer : StageTimer {
  std::vector<cudaEvent_t>& pool;
  size_t used = 0;
  int open[STG_N] = {};
  struct Pair {
    int stage, a, b;
  };
  std::vector<Pair> pairs;
  explicit EvTimer(std::vector<cudaEvent_t>& p) : pool(p) {}
  int next() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return (int)used++;
  }
  void begin(int stage, cudaStream_t st) override {
    open[stage] = next();
    cudaEventRecord(pool[open[stage]], st);
  }
  void end(int stage, cudaStream_t st) override {
    const int i = next();
    cudaEventRecord(pool[i], st);
    pairs.push_back({stage, open[stage], i});
  }
  void collect(float* ms, uint32_t* n) {
    for (const Pair& p : pairs) {
      float e = 0.0f;
      cudaEventElapsedTime(&e, pool[p.a], pool[p.b]);
      ms[p.stage] += e;
      n[p.stage] += 1;
    }
  }
};

}  // namespace

namespace srt {

bool ctx_view(rt_ctx* c, CtxView* v) {
  if (!c || c->poisoned) return false;
  v->device = c->device;
  v->stream = c->stream;
  v->has_scene = c->has_scene;
  v->has_spectra = c->has_spectra;
  v->S = dev_scene(c);
  v->P = c->sp;
  v->cmfw = c->d_cmfw;
  v->sms = c->sms;
  v->h_cams = c->h_cams;
  v->h_status = c->h_status;
  return true;
}

void ctx_error(rt_ctx* c, const char* msg, bool fatal) {
  if (!c) return;
  c->err = msg;
  if (fatal) c->poisoned = true;
}

}  // namespace srt

extern "C" {

rt_status rt_create(int device, void* cuda_stream, rt_ctx** out) {
  if (!out) return RT_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return RT_ERR_ARG;
  rt_ctx* c = new rt_ctx();
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete c;
    return RT_ERR_CUDA;
  }
  c->sms = num_sms(device);
  if (cudaMalloc(&c->wb.cnt, sizeof(Counters) * (kMaxDepth + 2)) != cudaSuccess ||
      cudaMalloc(&c->wb.tot, sizeof(Totals)) != cudaSuccess ||
      cudaMalloc(&c->wb.status, sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&c->d_cams, sizeof(DevCam) * kMaxCams) != cudaSuccess ||
      cudaMallocHost(&c->h_cams, sizeof(DevCam) * kMaxCams) != cudaSuccess ||
      cudaMallocHost(&c->h_status, sizeof(uint32_t)) != cudaSuccess ||
      cudaMallocHost(&c->h_tot, sizeof(Totals)) != cudaSuccess) {
    rt_destroy(c);
    return RT_ERR_OOM;
  }
  for (auto& e : c->ev) cudaEventCreate(&e);
  cudaMemset(c->wb.status, 0, sizeof(uint32_t));
  *out = c;
  return RT_OK;
}

void rt_destroy(rt_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  dfree(c->d_nodes);
  dfree(c->d_nodes4);
  dfree(c->d_nodes4q);
  dfree(c->d_nodes8);
  dfree(c->d_tris);
  dfree(c->d_nrm);
  dfree(c->d_mb);
  dfree(c->d_ad);
  dfree(c->d_mtype);
  dfree(c->d_sunL);
  dfree(c->d_cmfw);
  WaveBufs& b = c->wb;
  dfree(b.q[0]);
  dfree(b.q[1]);
  dfree(b.hit);
  dfree(b.sq);
  dfree(b.L);
  dfree(b.sig);
  dfree(b.rperm);
  dfree(b.rkey);
  dfree(b.rbins);
  dfree(b.L4);
  dfree(b.T4);
  dfree(b.C4);
  dfree(c->ph.rec);
  dfree(c->ph.rec_sorted);
  for (int q = 0; q < 2; ++q) {
    dfree(c->ph.keys[q]);
    dfree(c->ph.vals[q]);
  }
  dfree(c->ph.hist);
  dfree(c->ph.start);
  dfree(c->ph.end);
  dfree(b.cnt);
  dfree(b.tot);
  dfree(b.status);
  dfree(c->d_cams);
  dfree(c->d_accum);
  dfree(c->d_xyz);
  dfree(c->guide.grid);
  dfree(c->guide.W);
  dfree(c->guide.mg);
  dfree(c->guide.vg);
  dfree(c->guide.mW);
  dfree(c->guide.vW);
  dfree(c->guide.dgrid);
  dfree(c->guide.dW);
  dfree(c->guide.dWpart);
  dfree(c->guide.scratch);
  dfree(c->guide.gq);
  dfree(c->guide.wesc);
  dfree(c->guide.perm);
  dfree(c->guide.skey);
  dfree(c->guide.bins);
  dfree(c->guide.raw);
  dfree(c->guide.Lfinal);
  dfree(c->guide.trec);
  if (c->guide.pack) cudaFree(c->guide.pack);
  if (c->h_cams) cudaFreeHost(c->h_cams);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->h_tot) cudaFreeHost(c->h_tot);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->tpool) cudaEventDestroy(e);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  delete c;
}

const char* rt_last_error(const rt_ctx* c) { return c ? c->err.c_str() : "null context"; }

rt_status rt_set_stream(rt_ctx* c, void* s) {
  if (rt_status e = check_ctx(c)) return e;
  c->stream = (cudaStream_t)s;
  return RT_OK;
}

rt_status rt_set_counting(rt_ctx* c, int enable) {
  if (rt_status e = check_ctx(c)) return e;
  c->counting = enable != 0;
  return RT_OK;
}

rt_status rt_set_limits(rt_ctx* c, uint32_t queue_capacity, uint32_t traversal_steps, uint32_t fail_cuda_call) {
  if (rt_status e = check_ctx(c)) return e;
  c->lim_queue = queue_capacity;
  c->lim_steps = traversal_steps;
  c->fail_countdown = fail_cuda_call;
  c->graph_key.clear();  // a captured render holds the old limits
  return RT_OK;
}

rt_status rt_set_bvh_builder(rt_ctx* c, uint32_t builder) {
  if (rt_status e = check_ctx(c)) return e;
  if (builder > 2)
    return fail(c, RT_ERR_ARG, "rt_set_bvh_builder: 0 (host SAH), 1 (device LBVH) or 2 (host SAH with spatial splits)");
  c->builder = builder;
  return RT_OK;
}

rt_status rt_get_scene_info(rt_ctx* c, rt_scene_info* info) {
  if (rt_status e = check_ctx(c)) return e;
  if (!info) return fail(c, RT_ERR_ARG, "rt_get_scene_info: info is required");
  if (!c->has_scene) return fail(c, RT_ERR_STATE, "rt_get_scene_info: no scene loaded");
  info->n_tris = c->n_tris;
  info->n_nodes4 = c->n_nodes4;
  info->builder = c->builder_used;
  info->build_ms = c->build_ms;
  return RT_OK;
}

rt_status rt_set_timing(rt_ctx* c, int enable) {
  if (rt_status e = check_ctx(c)) return e;
  c->timing = enable != 0;
  return RT_OK;
}

rt_status rt_load_scene(rt_ctx* c, const float* verts, uint32_t n_verts, const uint32_t* tris, uint32_t n_tris,
                        const uint32_t* mat_id, const int32_t* mat_type, const float* mat_thickness, uint32_t n_mat) {
  if (rt_status e = check_ctx(c)) return e;
  if (!verts || !tris || !mat_id || !mat_type || !mat_thickness || n_verts == 0 || n_tris == 0 || n_mat == 0)
    return fail(c, RT_ERR_ARG, "rt_load_scene: null array or zero size");
  if (n_tris > (1u << 28)) return fail(c, RT_ERR_ARG, "rt_load_scene: more than 2^28 triangles");
  for (uint32_t i = 0; i < n_verts; ++i)
    if (!finite3(verts + 3 * (size_t)i)) return fail(c, RT_ERR_SCENE, "vertex " + std::to_string(i) + " not finite");
  for (uint32_t m = 0; m < n_mat; ++m) {
    if (mat_type[m] < 0 || mat_type[m] > 4) return fail(c, RT_ERR_SCENE, "material " + std::to_string(m) + ": bad type");
    if (!(mat_thickness[m] >= 0.0f) || !std::isfinite(mat_thickness[m]))
      return fail(c, RT_ERR_SCENE, "material " + std::to_string(m) + ": bad thickness");
  }
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (uint32_t i = 0; i < n_verts; ++i)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], (double)verts[3 * (size_t)i + a]);
      hi[a] = std::max(hi[a], (double)verts[3 * (size_t)i + a]);
    }
  std::vector<float> nrm64(4 * (size_t)n_tris);
  for (uint32_t t = 0; t < n_tris; ++t) {
    for (int v = 0; v < 3; ++v)
      if (tris[3 * (size_t)t + v] >= n_verts)
        return fail(c, RT_ERR_SCENE, "triangle " + std::to_string(t) + ": vertex index out of range");
    if (mat_id[t] >= n_mat) return fail(c, RT_ERR_SCENE, "triangle " + std::to_string(t) + ": material out of range");
    const float* a = verts + 3 * (size_t)tris[3 * (size_t)t];
    const float* b = verts + 3 * (size_t)tris[3 * (size_t)t + 1];
    const float* cc = verts + 3 * (size_t)tris[3 * (size_t)t + 2];
    const double e1[3] = {(double)b[0] - a[0], (double)b[1] - a[1], (double)b[2] - a[2]};
    const double e2[3] = {(double)cc[0] - a[0], (double)cc[1] - a[1], (double)cc[2] - a[2]};
    const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(len > 0.0)) return fail(c, RT_ERR_SCENE, "triangle " + std::to_string(t) + " is degenerate");
    for (int a2 = 0; a2 < 3; ++a2) nrm64[4 * (size_t)t + a2] = (float)(n[a2] / len);
  }
  if (n_tris >= (1u << 28)) return fail(c, RT_ERR_SCENE, "at most 2^28 triangles");
  const bool dev_build = c->builder == 1;
  if (dev_build && n_tris > kLbvhMaxTris) return fail(c, RT_ERR_ARG, "device BVH builder: at most 2^24 triangles");
  // Node boxes are padded by 2^-22 (max |coordinate| + origin offset) so that
  // the traversal's FMA slab test, fma(plane, 1/d, -o/d), stays conservative
  // for every origin inside the scene bounds (the rounding of o/d moves a
  // plane by at most 2^-24 |o|).
  const double diag = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                (hi[2] - lo[2]) * (hi[2] - lo[2]));
  double mabs = 0.0;
  for (int a = 0; a < 3; ++a) mabs = std::max(mabs, std::max(std::fabs(lo[a]), std::fabs(hi[a])));
  const double pad = std::ldexp(mabs + 2e-4 * diag, -22);
  auto down = [&](float v) {
    const double x = (double)v - pad;
    float f = (float)x;
    while ((double)f > x) f = std::nextafter(f, -INFINITY);
    return f;
  };
  auto up = [&](float v) {
    const double x = (double)v + pad;
    float f = (float)x;
    while ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
  };
  const auto t_build0 = std::chrono::steady_clock::now();
  // host build: binned SAH (with spatial splits for builder 2, which may
  // list a triangle in several leaves -- never a thin-glass one, whose
  // sun-ray transmittance must count once), leaf order from the tree; device
  // build: the records go up in input order and are sorted there
  BvhOut bvh;
  if (c->builder == 2) {
    std::vector<uint8_t> split(n_tris);
    for (uint32_t t = 0; t < n_tris; ++t) split[t] = mat_type[mat_id[t]] != 1;
    build_sbvh(verts, tris, n_tris, split.data(), bvh);
  } else if (!dev_build) {
    build_bvh(verts, tris, n_tris, bvh);
  }
  const size_t n_leaf = dev_build ? n_tris : bvh.order.size();
  if (n_leaf >= (1u << 29)) return fail(c, RT_ERR_SCENE, "too many BVH references");
  std::vector<float4> tr(3 * n_leaf), nr(n_leaf);
  for (uint32_t i = 0; i < (uint32_t)n_leaf; ++i) {
    const uint32_t t = dev_build ? i : bvh.order[i];
    const float* v[3];
    for (int k = 0; k < 3; ++k) v[k] = verts + 3 * (size_t)tris[3 * (size_t)t + k];
    uint32_t mid = mat_id[t];
    float idf, matf, zero = 0.0f;
    std::memcpy(&idf, &t, 4);
    std::memcpy(&matf, &mid, 4);
    tr[3 * (size_t)i] = make_float4(v[0][0], v[0][1], v[0][2], idf);
    tr[3 * (size_t)i + 1] = make_float4(v[1][0], v[1][1], v[1][2], matf);
    tr[3 * (size_t)i + 2] = make_float4(v[2][0], v[2][1], v[2][2], zero);
    nr[i] = make_float4(nrm64[4 * (size_t)t], nrm64[4 * (size_t)t + 1], nrm64[4 * (size_t)t + 2], matf);
  }
  std::vector<float4> nd;
  std::vector<Bvh4Node> b4;
  std::vector<float4> d8;  // eight-wide nodes in device layout (14 float4 each)
  std::vector<float4> d4q;  // four-wide nodes with 8-bit child boxes (4 float4 each)
  if (!dev_build) {
    nd.resize(2 * bvh.nodes.size());
    for (size_t i = 0; i < bvh.nodes.size(); ++i) {
      const BvhNode& b = bvh.nodes[i];
      float rf, cf;
      std::memcpy(&rf, &b.ref, 4);
      std::memcpy(&cf, &b.count, 4);
      nd[2 * i] = make_float4(down(b.lo[0]), down(b.lo[1]), down(b.lo[2]), rf);
      nd[2 * i + 1] = make_float4(up(b.hi[0]), up(b.hi[1]), up(b.hi[2]), cf);
    }
    // four-wide nodes, padded the same way (empty slots keep their +-inf box)
    // device layout per node: the six plane float4s, then the children packed
    // as the traversal stack stores them (ref << 3 | count; 0 for an empty
    // slot, whose box is never entered), then 16 bytes of padding
    collapse_bvh4(bvh, b4, nullptr);
    for (Bvh4Node& n4 : b4)
      for (int i = 0; i < 4; ++i) {
        if (n4.cnt[i] != kEmpty4) {
          n4.lox[i] = down(n4.lox[i]);
          n4.loy[i] = down(n4.loy[i]);
          n4.loz[i] = down(n4.loz[i]);
          n4.hix[i] = up(n4.hix[i]);
          n4.hiy[i] = up(n4.hiy[i]);
          n4.hiz[i] = up(n4.hiz[i]);
          n4.ref[i] = (n4.ref[i] << 3) | n4.cnt[i];
        } else {
          n4.ref[i] = 0;
        }
        n4.cnt[i] = 0;
      }
    // four-wide nodes with 8-bit child boxes: per axis a power-of-two cell
    // 2^e >= extent / 250 and an origin two cells below the node's lowest
    // padded plane (a float, rounded down); each child's padded planes
    // rounded outward to the grid and one more cell out on each side, a
    // margin that covers the traversal's half-cell rounding of the decoded
    // planes.  Layout: {origin, bits(e_x | e_y << 8 | e_z << 16)}, {lo x of
    // children 0-3, hi x, lo y, hi y} as bytes, {lo z, hi z, 0, 0}, children.
    d4q.resize(4 * b4.size());
    for (size_t j = 0; j < b4.size(); ++j) {
      const Bvh4Node& n4 = b4[j];
      const float* plo[3] = {n4.lox, n4.loy, n4.loz};
      const float* phi[3] = {n4.hix, n4.hiy, n4.hiz};
      float org[3];
      uint32_t ebits = 0;
      uint32_t words[6] = {0, 0, 0, 0, 0, 0};  // lo x, hi x, lo y, hi y, lo z, hi z
      for (int a = 0; a < 3; ++a) {
        double L = INFINITY, H = -INFINITY;
        for (int i = 0; i < 4; ++i) {
          if (plo[a][i] > phi[a][i]) continue;  // empty slot (lo +inf, hi -inf)
          L = std::min(L, (double)plo[a][i]);
          H = std::max(H, (double)phi[a][i]);
        }
        if (!(L <= H)) L = H = 0.0;  // no child (cannot happen below the root of a non-empty scene)
        const double ext = std::max(H - L, 1e-30);
        int e = (int)std::ceil(std::log2(ext / 250.0));
        e = std::max(-120, std::min(120, e));
        const double scale = std::ldexp(1.0, e);
        const double o = L - 2.0 * scale;
        float of = (float)o;
        while ((double)of > o) of = std::nextafter(of, -INFINITY);
        org[a] = of;
        ebits |= ((uint32_t)(uint8_t)(int8_t)e) << (8 * a);
        for (int i = 0; i < 4; ++i) {
          uint32_t ql = 255u, qh = 0u;  // empty slot: never entered
          if (!(plo[a][i] > phi[a][i])) {
            const double fl = std::floor(((double)plo[a][i] - (double)of) / scale) - 1.0;
            const double fh = std::ceil(((double)phi[a][i] - (double)of) / scale) + 1.0;
            ql = (uint32_t)std::max(0.0, std::min(255.0, fl));
            qh = (uint32_t)std::max(0.0, std::min(255.0, fh));
          }
          words[2 * a] |= ql << (8 * i);
          words[2 * a + 1] |= qh << (8 * i);
        }
      }
      float4* o4 = &d4q[4 * j];
      float eb, w[6];
      std::memcpy(&eb, &ebits, 4);
      std::memcpy(w, words, 24);
      o4[0] = make_float4(org[0], org[1], org[2], eb);
      o4[1] = make_float4(w[0], w[1], w[2], w[3]);
      o4[2] = make_float4(w[4], w[5], 0.0f, 0.0f);
      std::memcpy(&o4[3], n4.ref, 16);
    }
    // eight-wide nodes, padded the same way: the plane float4s (per axis lo
    // of children 0-3, 4-7, hi of 0-3, 4-7), then the children packed
    std::vector<Bvh8Node> b8;
    collapse_bvh8(bvh, b8, nullptr);
    d8.resize(14 * b8.size());
    for (size_t j = 0; j < b8.size(); ++j) {
      Bvh8Node& n8 = b8[j];
      uint32_t pk[8];
      for (int i = 0; i < 8; ++i) {
        if (n8.cnt[i] != kEmpty4) {
          n8.lox[i] = down(n8.lox[i]);
          n8.loy[i] = down(n8.loy[i]);
          n8.loz[i] = down(n8.loz[i]);
          n8.hix[i] = up(n8.hix[i]);
          n8.hiy[i] = up(n8.hiy[i]);
          n8.hiz[i] = up(n8.hiz[i]);
          pk[i] = (n8.ref[i] << 3) | n8.cnt[i];
        } else {
          pk[i] = 0;
        }
      }
      float4* o = &d8[14 * j];
      const float* planes[6] = {n8.lox, n8.hix, n8.loy, n8.hiy, n8.loz, n8.hiz};
      for (int q = 0; q < 6; ++q) {
        o[2 * q] = make_float4(planes[q][0], planes[q][1], planes[q][2], planes[q][3]);
        o[2 * q + 1] = make_float4(planes[q][4], planes[q][5], planes[q][6], planes[q][7]);
      }
      std::memcpy(&o[12], pk, 32);
    }
  }
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  dfree(c->d_nodes);
  dfree(c->d_nodes4);
  dfree(c->d_nodes8);
  dfree(c->d_nodes4q);
  c->n_nodes8 = 0;
  dfree(c->d_tris);
  dfree(c->d_nrm);
  c->has_scene = false;
  CUDA_TRY(c, cudaMalloc(&c->d_tris, tr.size() * sizeof(float4)));
  CUDA_TRY(c, cudaMalloc(&c->d_nrm, nr.size() * sizeof(float4)));
  if (!dev_build) {
    CUDA_TRY(c, cudaMalloc(&c->d_nodes, nd.size() * sizeof(float4)));
    CUDA_TRY(c, cudaMalloc(&c->d_nodes4, b4.size() * sizeof(Bvh4Node)));
    CUDA_TRY(c, cudaMemcpy(c->d_nodes4, b4.data(), b4.size() * sizeof(Bvh4Node), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMalloc(&c->d_nodes4q, d4q.size() * sizeof(float4)));
    CUDA_TRY(c, cudaMemcpy(c->d_nodes4q, d4q.data(), d4q.size() * sizeof(float4), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMalloc(&c->d_nodes8, d8.size() * sizeof(float4)));
    CUDA_TRY(c, cudaMemcpy(c->d_nodes8, d8.data(), d8.size() * sizeof(float4), cudaMemcpyHostToDevice));
    c->n_nodes8 = (uint32_t)(d8.size() / 14);
    CUDA_TRY(c, cudaMemcpy(c->d_nodes, nd.data(), nd.size() * sizeof(float4), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->d_tris, tr.data(), tr.size() * sizeof(float4), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->d_nrm, nr.data(), nr.size() * sizeof(float4), cudaMemcpyHostToDevice));
    c->n_nodes = (uint32_t)bvh.nodes.size();
    c->n_nodes4 = (uint32_t)b4.size();
    c->build_ms = (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_build0).count();
  } else {
    // device build from the uploaded geometry and input-order records
    float *d_verts = nullptr;
    uint32_t* d_idx = nullptr;
    float4 *d_tr_in = nullptr, *d_nr_in = nullptr;
    void* scratch = nullptr;
    rt_status st = RT_OK;
    auto release = [&]() {
      dfree(d_verts);
      dfree(d_idx);
      dfree(d_tr_in);
      dfree(d_nr_in);
      dfree(scratch);
    };
    const size_t n4cap = std::max<size_t>(n_tris - 1, 1);
    cudaError_t e = cudaMalloc(&d_verts, 3 * (size_t)n_verts * sizeof(float));
    if (!e) e = cudaMalloc(&d_idx, 3 * (size_t)n_tris * sizeof(uint32_t));
    if (!e) e = cudaMalloc(&d_tr_in, tr.size() * sizeof(float4));
    if (!e) e = cudaMalloc(&d_nr_in, nr.size() * sizeof(float4));
    if (!e) e = cudaMalloc(&scratch, lbvh_scratch_bytes(n_tris));
    if (!e) e = cudaMalloc(&c->d_nodes4, n4cap * 8 * sizeof(float4));
    if (!e) e = cudaMemcpy(d_verts, verts, 3 * (size_t)n_verts * sizeof(float), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(d_idx, tris, 3 * (size_t)n_tris * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(d_tr_in, tr.data(), tr.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(d_nr_in, nr.data(), nr.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (e) {
      release();
      CUDA_TRY(c, e);
    }
    float padf = (float)pad;
    if ((double)padf < pad) padf = std::nextafter(padf, INFINITY);
    const float flo[3] = {(float)lo[0], (float)lo[1], (float)lo[2]}, fhi[3] = {(float)hi[0], (float)hi[1], (float)hi[2]};
    cudaStream_t bs = c->stream;
    uint32_t* d_counts = nullptr;
    cudaEventRecord(c->ev[0], bs);
    launch_lbvh(d_verts, d_idx, n_tris, flo, fhi, padf, d_tr_in, d_nr_in, scratch, (float4*)c->d_nodes4,
                (float4*)c->d_tris, (float4*)c->d_nrm, &d_counts, c->sms, bs);
    cudaEventRecord(c->ev[1], bs);
    uint32_t counts[2] = {0, 0};
    e = cudaGetLastError();
    if (!e) e = cudaMemcpyAsync(counts, d_counts, sizeof(uint32_t), cudaMemcpyDeviceToHost, bs);
    if (!e) e = cudaMemcpyAsync(counts + 1, d_counts + kLbvhLevels, sizeof(uint32_t), cudaMemcpyDeviceToHost, bs);
    if (!e) e = cudaStreamSynchronize(bs);
    float ms = 0.0f;
    if (!e) e = cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
    release();
    CUDA_TRY(c, e);
    if (counts[1] != 0u || counts[0] == 0u || counts[0] > n4cap)
      st = fail(c, RT_ERR_SCENE, "device BVH builder: tree deeper than the collapse levels");
    if (st != RT_OK) return st;
    c->d_nodes = nullptr;  // no binary tree: the binary-tree traversal variants are unavailable
    c->n_nodes = 2 * n_tris - 1;
    c->n_nodes4 = counts[0];
    c->build_ms = ms;
  }
  c->builder_used = c->builder;
  c->n_tris = n_tris;
  c->n_mat = n_mat;
  const double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
  c->eps = (float)(1e-4 * std::sqrt(dx * dx + dy * dy + dz * dz));
  c->mtype.assign(mat_type, mat_type + n_mat);
  // thin-glass triangles in input order (portals of the photon pass)
  c->glass.clear();
  for (uint32_t t = 0; t < n_tris; ++t)
    if (mat_type[mat_id[t]] == 1)
      for (int q = 0; q < 3; ++q)
        for (int a = 0; a < 3; ++a) c->glass.push_back(verts[3 * (size_t)tris[3 * (size_t)t + q] + a]);
  c->mthick.assign(mat_thickness, mat_thickness + n_mat);
  for (int a = 0; a < 3; ++a) {
    c->lo[a] = (float)lo[a];
    c->hi[a] = (float)hi[a];
  }
  c->guide.init = false;
  c->has_scene = true;
  c->has_spectra = false;  // tables are per material: set them again
  return RT_OK;
}

rt_status rt_set_spectra(rt_ctx* c, const float* lambda_nm, uint32_t n_bands, const float* sun_L,
                         const float sun_dir[3], float sun_half_angle, const float* n, const float* k, const float* rho,
                         const float* le, const float* cmf_w) {
  if (rt_status e = check_ctx(c)) return e;
  if (!c->has_scene) return fail(c, RT_ERR_STATE, "rt_set_spectra: load a scene first");
  if (!lambda_nm || !sun_L || !sun_dir || !n || !k || !rho || !cmf_w || n_bands == 0 || n_bands > 4096)
    return fail(c, RT_ERR_ARG, "rt_set_spectra: null array or bad band count");
  if (!finite3(sun_dir) || !(sun_half_angle > 0.0f) || sun_half_angle > 3.14159275f)
    return fail(c, RT_ERR_ARG, "rt_set_spectra: bad sun direction or half angle");
  const double sl = std::sqrt((double)sun_dir[0] * sun_dir[0] + (double)sun_dir[1] * sun_dir[1] +
                              (double)sun_dir[2] * sun_dir[2]);
  if (!(sl > 0.0)) return fail(c, RT_ERR_ARG, "rt_set_spectra: zero sun direction");
  const uint32_t M = c->n_mat;
  std::vector<float4> mb((size_t)M * n_bands);
  std::vector<float> ad((size_t)M * n_bands);
  for (uint32_t m = 0; m < M; ++m)
    for (uint32_t b = 0; b < n_bands; ++b) {
      const size_t i = (size_t)m * n_bands + b;
      if (!std::isfinite(n[i]) || !std::isfinite(k[i]) || !std::isfinite(rho[i]) || (le && !std::isfinite(le[i])) ||
          !(lambda_nm[b] > 0.0f))
        return fail(c, RT_ERR_ARG, "rt_set_spectra: non-finite table entry");
      mb[i] = make_float4(n[i], k[i], rho[i], le ? le[i] : 0.0f);
      // thin glass: alpha d for its thickness; solid glass: alpha per metre
      const double len = c->mtype[m] == 4 ? 1.0 : (double)c->mthick[m];
      ad[i] = (float)(4.0 * M_PI * (double)k[i] * len / ((double)lambda_nm[b] * 1e-9));
    }
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  dfree(c->d_mb);
  dfree(c->d_ad);
  dfree(c->d_mtype);
  dfree(c->d_sunL);
  dfree(c->d_cmfw);
  c->has_spectra = false;
  CUDA_TRY(c, cudaMalloc(&c->d_mb, mb.size() * sizeof(float4)));
  CUDA_TRY(c, cudaMalloc(&c->d_ad, ad.size() * sizeof(float)));
  CUDA_TRY(c, cudaMalloc(&c->d_mtype, M * sizeof(int)));
  CUDA_TRY(c, cudaMalloc(&c->d_sunL, n_bands * sizeof(float)));
  CUDA_TRY(c, cudaMalloc(&c->d_cmfw, (size_t)n_bands * 3 * sizeof(float)));
  CUDA_TRY(c, cudaMemcpy(c->d_mb, mb.data(), mb.size() * sizeof(float4), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->d_ad, ad.data(), ad.size() * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->d_mtype, c->mtype.data(), M * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->d_sunL, sun_L, n_bands * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->d_cmfw, cmf_w, (size_t)n_bands * 3 * sizeof(float), cudaMemcpyHostToDevice));
  c->cmf_w.assign(cmf_w, cmf_w + (size_t)n_bands * 3);
  DevSpectra& P = c->sp;
  P.mb = c->d_mb;
  P.ad = c->d_ad;
  P.mtype = c->d_mtype;
  P.sunL = c->d_sunL;
  P.n_bands = n_bands;
  P.n_mat = M;
  P.sun = make_float3((float)(sun_dir[0] / sl), (float)(sun_dir[1] / sl), (float)(sun_dir[2] / sl));
  P.cos_max = (float)std::cos((double)sun_half_angle);
  for (int a = 0; a < 3; ++a) c->sun_d[a] = sun_dir[a] / sl;
  c->cos_max_d = std::cos((double)sun_half_angle);
  P.one_minus_cos = (float)(1.0 - std::cos((double)sun_half_angle));
  // the sun-ray visit order of the four-wide tree's children
  if (c->d_nodes4 && c->n_nodes4) {
    launch_sun_order4(c->d_nodes4, c->n_nodes4, P.sun, c->sms, c->stream);
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  c->has_spectra = true;
  return RT_OK;
}

extern "C++" {
namespace srt {

// Checks the cameras and writes their device form (basis derived in FP64)
// into out[0 .. n_cams); *npix = pixels over all views.  On a bad camera
// returns false with the reason in *why.
bool build_dev_cams(const rt_camera* cams, uint32_t n_cams, DevCam* out, uint64_t* npix_out, const char** why) {
  uint64_t npix = 0;
  for (uint32_t v = 0; v < n_cams; ++v) {
    const rt_camera& cm = cams[v];
    if (cm.width == 0 || cm.height == 0) return (*why = "zero-sized view"), false;
    if (!finite3(cm.pos) || !finite3(cm.look) || !finite3(cm.up) || !(cm.vfov_deg > 0.0f && cm.vfov_deg < 180.0f))
      return (*why = "bad camera"), false;
    npix += (uint64_t)cm.width * cm.height;
  }
  if (npix >= (1ull << 32)) return (*why = "too many pixels"), false;
  uint64_t off = 0;
  for (uint32_t v = 0; v < n_cams; ++v) {
    const rt_camera& cm = cams[v];
    double f[3], r[3], u[3];
    double fl = 0, rl = 0;
    for (int a = 0; a < 3; ++a) {
      f[a] = (double)cm.look[a] - cm.pos[a];
      fl += f[a] * f[a];
    }
    fl = std::sqrt(fl);
    if (!(fl > 0)) return (*why = "camera look == pos"), false;
    for (int a = 0; a < 3; ++a) f[a] /= fl;
    r[0] = f[1] * cm.up[2] - f[2] * cm.up[1];
    r[1] = f[2] * cm.up[0] - f[0] * cm.up[2];
    r[2] = f[0] * cm.up[1] - f[1] * cm.up[0];
    for (int a = 0; a < 3; ++a) rl += r[a] * r[a];
    rl = std::sqrt(rl);
    if (!(rl > 1e-12)) return (*why = "camera up parallel to the view direction"), false;
    for (int a = 0; a < 3; ++a) r[a] /= rl;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    DevCam& d = out[v];
    d.pos = make_float3(cm.pos[0], cm.pos[1], cm.pos[2]);
    d.f = make_float3((float)f[0], (float)f[1], (float)f[2]);
    d.r = make_float3((float)r[0], (float)r[1], (float)r[2]);
    d.u = make_float3((float)u[0], (float)u[1], (float)u[2]);
    const double th = std::tan(0.5 * (double)cm.vfov_deg * M_PI / 180.0);
    d.th = (float)th;
    d.tha = (float)(th * (double)cm.width / (double)cm.height);
    d.W = cm.width;
    d.H = cm.height;
    d.offset = (uint32_t)off;
    d.pad = 0;
    off += (uint64_t)cm.width * cm.height;
  }
  *npix_out = npix;
  return true;
}

}  // namespace srt
}  // extern "C++"

// The cameras of a render in the pinned staging array.
static rt_status stage_cameras(rt_ctx* c, const rt_camera* cams, uint32_t n_cams, const char* who, uint64_t* npix_out) {
  const char* why = "";
  if (!build_dev_cams(cams, n_cams, c->h_cams, npix_out, &why)) return fail(c, RT_ERR_ARG, std::string(who) + ": " + why);
  return RT_OK;
}

static void guide_train_enqueue(rt_ctx* c, const float* rec, uint64_t n);

static rt_status render_impl(rt_ctx* c, const rt_camera* cams, uint32_t n_cams, uint32_t band_first,
                             uint32_t band_count, uint32_t spp, uint32_t depth, uint64_t seed,
                             const rt_render_opts* opts, double* spectral_dev, float* xyz_dev, rt_stats* stats) {
  if (!c->has_scene || !c->has_spectra) return fail(c, RT_ERR_STATE, "rt_render: scene and spectra must be set");
  if (!cams || n_cams == 0 || n_cams > (uint32_t)kMaxCams) return fail(c, RT_ERR_ARG, "rt_render: 1..64 cameras");
  if (band_count == 0 || band_first + band_count > c->sp.n_bands || band_first + band_count < band_first)
    return fail(c, RT_ERR_ARG, "rt_render: band range outside the spectra");
  if (spp == 0) return fail(c, RT_ERR_ARG, "rt_render: spp must be >= 1");
  if (depth == 0 || depth > (uint32_t)kMaxDepth) return fail(c, RT_ERR_ARG, "rt_render: depth must be 1..64");
  rt_render_opts o{};
  if (opts) o = *opts;
  if (o.xyz_mode > 2) return fail(c, RT_ERR_ARG, "rt_render: unknown xyz_mode");
  if (o.xyz_mode != 2 && band_count > kXyzMaxBandsTc)
    return fail(c, RT_ERR_ARG, "rt_render: tensor-core XYZ takes at most 192 bands (use RT_XYZ_FP64)");
  if (o.trace_variant > 5) return fail(c, RT_ERR_ARG, "rt_render: unknown trace_variant");
  if (o.trace_variant == 5 && !c->d_nodes4q)
    return fail(c, RT_ERR_ARG, "rt_render: the quantised tree needs a host-built BVH (builder 0 or 2)");
  if (o.trace_variant == 4 && !c->d_nodes8)
    return fail(c, RT_ERR_ARG, "rt_render: the eight-wide tree needs a host-built BVH (builder 0 or 2)");
  if (o.trace_variant != 0 && !c->d_nodes)
    return fail(c, RT_ERR_ARG, "rt_render: binary-tree traversal variants need the host-built BVH");
  if (o.leaf_batch > 32) return fail(c, RT_ERR_ARG, "rt_render: leaf_batch is 1..32");
  if (o.guide_order > 1) return fail(c, RT_ERR_ARG, "rt_render: guide_order is 0 or 1");
  if (o.ray_order > 1) return fail(c, RT_ERR_ARG, "rt_render: ray_order is 0 or 1");
  if (o.bands_per_path != 0 && o.bands_per_path != 1 && o.bands_per_path != 4)
    return fail(c, RT_ERR_ARG, "rt_render: bands_per_path is 1 or 4");
  const uint32_t nb = o.bands_per_path == 4 ? 4u : 1u;
  if (nb == 4 && o.guided) return fail(c, RT_ERR_ARG, "rt_render: four bands per path exclude guided sampling");
  if (nb == 4 && o.trace_variant != 0)
    return fail(c, RT_ERR_ARG, "rt_render: four bands per path use the four-wide tree (trace_variant 0)");
  if (o.trace_refill > 32 || o.shadow_refill > 32) return fail(c, RT_ERR_ARG, "rt_render: refill thresholds are 1..32");
  if (o.guided && !c->guide.init) return fail(c, RT_ERR_STATE, "rt_render: guided rendering needs rt_guide_init");
  if (o.guide_train_steps && !(o.guided && o.guide_collect))
    return fail(c, RT_ERR_ARG, "rt_render: guide training needs guided = 1 and guide_collect > 0");
  if ((uint64_t)o.sample_first + spp > 0xFFFFFFFFull) return fail(c, RT_ERR_ARG, "rt_render: sample range overflows");
  if (o.accumulate && !spectral_dev) return fail(c, RT_ERR_ARG, "rt_render: accumulate needs spectral_dev");
  if ((o.probe_map_dev != nullptr) != (o.probe_L_dev != nullptr) ||
      (o.probe_map_dev != nullptr) != (o.probe_sig_dev != nullptr))
    return fail(c, RT_ERR_ARG, "rt_render: probe_map, probe_L and probe_sig go together");
  uint64_t npix = 0;
  if (rt_status e = stage_cameras(c, cams, n_cams, "rt_render", &npix)) return e;
  // path units per pixel: one per band, or one per group of four bands
  const uint32_t units = nb == 4 ? (band_count + 3) / 4 : band_count;
  const uint64_t ACC64 = npix * band_count;  // spectral slots
  const uint64_t PB64 = npix * units;
  if (ACC64 >= (1ull << 32)) return fail(c, RT_ERR_ARG, "rt_render: pixels x bands must be below 2^32");
  cudaSetDevice(c->device);
  cudaStream_t st = c->stream;
  const uint32_t PB = (uint32_t)PB64;
  uint32_t cap = o.wave_capacity ? o.wave_capacity : (1u << 23);
  cap = std::min<uint32_t>(std::min<uint32_t>(cap, kMaxWave), PB);
  cap = std::max<uint32_t>(cap, 1u);
  if (rt_status e = ensure_wave(c, cap)) return e;
  if (nb == 4)
    if (rt_status e = ensure_four_band(c, cap)) return e;
  if (spectral_dev && ((uintptr_t)spectral_dev & 15u) != 0)
    return fail(c, RT_ERR_ARG, "rt_render: spectral_dev must be 16-byte aligned");
  double* accum = spectral_dev;
  if (!accum) {
    if (c->accum_cap < ACC64) {
      dfree(c->d_accum);
      c->accum_cap = 0;
      CUDA_TRY(c, cudaMalloc(&c->d_accum, ACC64 * sizeof(double)));
      c->accum_cap = ACC64;
    }
    accum = c->d_accum;
  }
  if (o.trace_block && (o.trace_block > 128 || o.trace_block % 32))
    return fail(c, RT_ERR_ARG, "rt_render: trace_block must be a multiple of 32 up to 128");
  LaunchCfg lc;
  lc.block_trace = o.trace_block ? (int)o.trace_block : 128;
  lc.block_shade = 256;
  lc.grid_trace = c->sms * (o.ctas_per_sm ? (int)o.ctas_per_sm : trace_blocks_per_sm(lc.block_trace));
  lc.grid_shadow = c->sms * (o.ctas_per_sm ? (int)o.ctas_per_sm : shadow_blocks_per_sm(lc.block_trace));
  lc.grid_shade = c->sms * 8;
  lc.counting = c->counting;
  lc.record = o.probe_map_dev != nullptr;
  lc.variant = (int)o.trace_variant;
  lc.leaf_min = o.leaf_batch ? (int)o.leaf_batch : kDefaultLeafBatch;
  lc.sort_rays = o.ray_order == 1;
  lc.trace_steps = o.trace_steps ? (int)o.trace_steps : kDefaultTraceSteps;
  lc.trace_refill = o.trace_refill ? (int)o.trace_refill : kDefaultTraceRefill;
  lc.shadow_steps = o.shadow_steps ? (int)o.shadow_steps : kDefaultShadowSteps;
  lc.shadow_refill = o.shadow_refill ? (int)o.shadow_refill : kDefaultShadowRefill;
  Probe probe{o.probe_map_dev, o.probe_L_dev, o.probe_sig_dev};
  WaveParams w{};
  w.PB = PB;
  w.band_first = band_first;
  w.band_count = units;
  w.nb = nb;
  w.B = band_count;
  w.acc_stride = band_count;
  w.acc_off = 0;
  w.spp = spp;
  w.depth = depth;
  w.key0 = (uint32_t)seed;
  w.key1 = (uint32_t)(seed >> 32);
  w.s_base = o.sample_first;
  w.n_bands = c->sp.n_bands;
  const uint64_t total = PB64 * spp;
  const DevScene S = dev_scene(c);
  // guided sampling buffers
  GuideWave gw{};
  uint32_t n_slots = 0, perm_mul = 1;
  if (o.guided) {
    auto& G = c->guide;
    gw.on = true;
    gw.depth = std::min<uint32_t>(G.cfg.guide_depth, depth);
    gw.alpha = G.cfg.mis_alpha;
    if (G.gq_cap < cap) {
      dfree(G.gq);
      dfree(G.wesc);
      dfree(G.perm);
      dfree(G.skey);
      G.gq_cap = 0;
      CUDA_TRY(c, cudaMalloc(&G.gq, (size_t)cap * 3 * sizeof(float4)));
      CUDA_TRY(c, cudaMalloc(&G.wesc, (size_t)cap * sizeof(float)));
      CUDA_TRY(c, cudaMalloc(&G.perm, (size_t)cap * sizeof(uint32_t)));
      CUDA_TRY(c, cudaMalloc(&G.skey, (size_t)cap * sizeof(uint32_t)));
      G.gq_cap = cap;
    }
    // bins, then the chunk totals of the scan
    if (!G.bins) CUDA_TRY(c, cudaMalloc(&G.bins, (size_t)(kGuideSortBins + kGuideSortBins / 1024u) * sizeof(uint32_t)));
    gw.gq = G.gq;
    gw.wesc = G.wesc;
    if (o.guide_order == 1) {
      gw.perm = G.perm;
      gw.skey = G.skey;
      gw.bins = G.bins;
    }
    if (o.guide_collect) {
      gw.collect = o.guide_collect;
      gw.slots_per_vertex = (cap + o.guide_collect - 1) / o.guide_collect;
      n_slots = gw.slots_per_vertex * gw.depth;
      if (G.raw_cap < n_slots || !G.Lfinal) {
        dfree(G.raw);
        dfree(G.trec);
        dfree(G.Lfinal);
        G.raw_cap = 0;
        CUDA_TRY(c, cudaMalloc(&G.raw, (size_t)n_slots * kRawF4 * sizeof(float4)));
        CUDA_TRY(c, cudaMalloc(&G.trec, (size_t)n_slots * 2 * 3 * sizeof(float4)));
        CUDA_TRY(c, cudaMalloc(&G.Lfinal, (size_t)kMaxWave * sizeof(float)));
        G.raw_cap = n_slots;
      }
      gw.raw = G.raw;
      gw.Lfinal = G.Lfinal;
      // odd multiplier coprime with n_slots: slot -> position is a bijection
      auto gcd = [](uint64_t a, uint64_t b2) {
        while (b2) {
          uint64_t t = a % b2;
          a = b2;
          b2 = t;
        }
        return a;
      };
      const uint64_t n_rec = 2ull * n_slots;
      perm_mul = (uint32_t)(2654435761ull % n_rec);
      if (perm_mul == 0) perm_mul = 1;
      while (gcd(perm_mul, n_rec) != 1) ++perm_mul;
    }
  }
  // the queues as the kernels see them (a diagnostic limit may make them
  // smaller than the wave; the buffers keep their size)
  WaveBufs wb = c->wb;
  if (c->lim_queue && c->lim_queue < wb.cap) wb.cap = c->lim_queue;
  int launches = 0;
  uint32_t waves = 0;
  EvTimer timer(c->tpool);
  StageTimer* tm = c->timing ? &timer : nullptr;
  const bool use_graph = o.use_graph != 0;
  if (use_graph && (tm || lc.counting || lc.record || o.guide_train_steps))
    return fail(c, RT_ERR_ARG, "rt_render: use_graph excludes timing, counting, probes and guide training");
  if (o.guide_records_dev && (!o.guided || o.guide_collect != 1 || use_graph))
    return fail(c, RT_ERR_ARG, "rt_render: guide_records_dev needs guided, guide_collect = 1 and no graph");
  // Everything one render enqueues, on stream `s`; with events the device
  // time of the path tracing and of the XYZ contraction is bracketed.
  auto enqueue = [&](cudaStream_t s, bool events) -> cudaError_t {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(c->d_cams, c->h_cams, sizeof(DevCam) * n_cams, cudaMemcpyHostToDevice, s))) return e;
    if (!o.accumulate && (e = cudaMemsetAsync(accum, 0, ACC64 * sizeof(double), s))) return e;
    if ((e = cudaMemsetAsync(c->wb.status, 0, sizeof(uint32_t), s))) return e;
    if ((e = cudaMemsetAsync(c->wb.tot, 0, sizeof(Totals), s))) return e;
    if (events && (e = cudaEventRecord(c->ev[0], s))) return e;
    for (uint64_t ws = 0; ws < total; ws += cap) {
      w.n = (uint32_t)std::min<uint64_t>(cap, total - ws);
      w.s0 = o.sample_first + (uint32_t)(ws / PB);
      w.r0 = (uint32_t)(ws % PB);
      if ((e = cudaMemsetAsync(c->wb.cnt, 0, sizeof(Counters) * (depth + 2), s))) return e;
      if (gw.collect && (e = cudaMemsetAsync(gw.raw, 0, (size_t)n_slots * kRawF4 * sizeof(float4), s))) return e;
      launch_wave(lc, S, c->sp, c->d_cams, n_cams, w, wb, accum, probe, s, &launches, tm, &gw, &c->guide.dev,
                  c->guide.pack, c->sms);
      if (o.guide_records_dev) {
        // the wave's records in path order: slot (v, p) -> records 2 (v spv + p) and + 1, copied to
        // path ws + p of vertex v
        launch_guide_records(gw, n_slots, 1u, c->guide.trec, s);
        ++launches;
        const size_t row = (size_t)2 * 12 * sizeof(float);
        if ((e = cudaMemcpy2DAsync(o.guide_records_dev + 24 * ws, row * total, c->guide.trec, row * gw.slots_per_vertex,
                                   row * w.n, gw.depth, cudaMemcpyDeviceToDevice, s)))
          return e;
      }
      if (gw.collect && o.guide_train_steps) {
        if (tm) tm->begin(STG_TRAIN, s);
        launch_guide_records(gw, n_slots, perm_mul, c->guide.trec, s);
        const uint32_t steps = o.guide_train_steps;
        const uint64_t n_rec = 2ull * n_slots;
        uint64_t batch =
            o.guide_batch ? std::min<uint64_t>(o.guide_batch, n_rec) : std::max<uint64_t>(1, n_rec / steps);
        for (uint32_t t = 0; t < steps; ++t) {
          const uint64_t off = ((uint64_t)t * batch) % n_rec;
          const uint64_t nb = std::min<uint64_t>(batch, n_rec - off);
          guide_train_enqueue(c, c->guide.trec + 12 * off, nb);
        }
        if (tm) tm->end(STG_TRAIN, s);
        launches += 1 + 5 * (int)steps;
      }
      ++waves;
    }
    if ((e = cudaGetLastError())) return e;
    if (events && (e = cudaEventRecord(c->ev[1], s))) return e;
    if (xyz_dev) {
      XyzWeights xw;
      xw.w32 = c->d_cmfw + 3 * (size_t)band_first;
      xw.band_count = band_count;
      xw.kpad = (band_count + 15) / 16 * 16;
      if (tm) tm->begin(STG_XYZ, s);
      launch_xyz(accum, npix, xw, o.spp_total ? o.spp_total : spp, (int)o.xyz_mode, xyz_dev, s, c->wb.status, c->sms);
      if (tm) tm->end(STG_XYZ, s);
      ++launches;
      if ((e = cudaGetLastError())) return e;
    }
    if (events && (e = cudaEventRecord(c->ev[2], s))) return e;
    return cudaSuccess;
  };
  if (!use_graph) {
    CUDA_TRY(c, enqueue(st, true));
  } else {
    // one captured graph per launch configuration, replayed on an internal
    // stream ordered after the caller's stream
    char kb[512];
    std::snprintf(kb, sizeof(kb), "%u|%llu|%u|%u|%u|%u|%llu|%u|%u|%u|%u|%p|%p|%p|%p|%d|%d|%d|%d|%d|%d|%d|%d|%u|%u|%u|%u|%g|%d",
                  n_cams, (unsigned long long)npix, band_first, band_count, spp, depth, (unsigned long long)seed,
                  o.sample_first, o.accumulate, o.spp_total, o.xyz_mode, (void*)accum, (void*)xyz_dev,
                  (void*)c->d_nodes, (void*)c->d_mb, lc.grid_trace, lc.block_trace, lc.variant, lc.trace_steps,
                  lc.trace_refill, lc.shadow_steps, lc.shadow_refill, (int)cap, o.guided, gw.depth, gw.collect,
                  o.wave_capacity, (double)gw.alpha,
                  (lc.leaf_min * 4 + (int)o.guide_order * 2 + (int)o.ray_order) * 8 + (int)nb);
    std::string key(kb);
    char pb[160];
    std::snprintf(pb, sizeof(pb), "|%p|%p|%p|%p|%p", (void*)c->wb.q[0], (void*)c->wb.sq, (void*)gw.gq,
                  (void*)c->guide.grid, c->guide.pack);
    key += pb;
    for (uint32_t v = 0; v < n_cams; ++v) key += "|" + std::to_string(cams[v].width) + "x" + std::to_string(cams[v].height);
    if (!c->gstream) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
    if (!c->graph_exec || key != c->graph_key) {
      if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
      }
      CUDA_TRY(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
      const cudaError_t ce = enqueue(c->gstream, false);
      cudaGraph_t g = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(c->gstream, &g);
      if (ce != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        CUDA_TRY(c, ce != cudaSuccess ? ce : ee);
      }
      const cudaError_t ie = cudaGraphInstantiate(&c->graph_exec, g, 0);
      cudaGraphDestroy(g);
      CUDA_TRY(c, ie);
      c->graph_key = key;
      c->graph_launches = launches;
      c->graph_waves = waves;
    }
    launches = c->graph_launches;
    waves = c->graph_waves;
    CUDA_TRY(c, cudaEventRecord(c->ev[0], st));
    CUDA_TRY(c, cudaStreamWaitEvent(c->gstream, c->ev[0], 0));
    CUDA_TRY(c, cudaGraphLaunch(c->graph_exec, c->gstream));
    CUDA_TRY(c, cudaEventRecord(c->ev[1], c->gstream));
    CUDA_TRY(c, cudaStreamWaitEvent(st, c->ev[1], 0));
    CUDA_TRY(c, cudaEventRecord(c->ev[2], st));
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->wb.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaMemcpyAsync(c->h_tot, c->wb.tot, sizeof(Totals), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->paths = ACC64 * spp;  // spectral (pixel, sample, band) estimates
    stats->ext_rays = c->h_tot->ext_rays;
    stats->shadow_rays = c->h_tot->shadow_rays;
    stats->nodes_visited = c->h_tot->nodes;
    stats->tris_tested = c->h_tot->tris;
    stats->shadow_nodes_visited = c->h_tot->snodes;
    stats->shadow_tris_tested = c->h_tot->stris;
    if (tm) timer.collect(stats->ms_stage, stats->launches_stage);
    stats->waves = waves;
    stats->kernel_launches = (uint32_t)launches;
    cudaEventElapsedTime(&stats->ms_render, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&stats->ms_xyz, c->ev[1], c->ev[2]);
  }
  return status_to_rt(c, *c->h_status);
}

rt_status rt_render(rt_ctx* c, const rt_camera* cams, uint32_t n_cams, uint32_t band_first, uint32_t band_count,
                    uint32_t spp, uint32_t depth, uint64_t seed, const rt_render_opts* opts, double* spectral_dev,
                    float* xyz_dev, rt_stats* stats) {
  if (rt_status e = check_ctx(c)) return e;
  return render_impl(c, cams, n_cams, band_first, band_count, spp, depth, seed, opts, spectral_dev, xyz_dev, stats);
}

rt_status rt_render_host(rt_ctx* c, const rt_camera* cams, uint32_t n_cams, uint32_t band_first, uint32_t band_count,
                         uint32_t spp, uint32_t depth, uint64_t seed, const rt_render_opts* opts, double* spectral_host,
                         float* xyz_host, rt_stats* stats) {
  if (rt_status e = check_ctx(c)) return e;
  if (!xyz_host) return fail(c, RT_ERR_ARG, "rt_render_host: xyz_host is required");
  if (!cams || n_cams == 0 || n_cams > (uint32_t)kMaxCams) return fail(c, RT_ERR_ARG, "rt_render_host: 1..64 cameras");
  uint64_t npix = 0;
  for (uint32_t v = 0; v < n_cams; ++v) npix += (uint64_t)cams[v].width * cams[v].height;
  cudaSetDevice(c->device);
  if (c->xyz_cap < npix * 3) {
    dfree(c->d_xyz);
    c->xyz_cap = 0;
    CUDA_TRY(c, cudaMalloc(&c->d_xyz, npix * 3 * sizeof(float)));
    c->xyz_cap = npix * 3;
  }
  rt_status s = render_impl(c, cams, n_cams, band_first, band_count, spp, depth, seed, opts, nullptr, c->d_xyz, stats);
  if (s != RT_OK) return s;
  CUDA_TRY(c, cudaMemcpyAsync(xyz_host, c->d_xyz, npix * 3 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  if (spectral_host)
    CUDA_TRY(c, cudaMemcpyAsync(spectral_host, c->d_accum, npix * band_count * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RT_OK;
}

rt_status rt_philox(rt_ctx* c, const uint32_t* ctr_dev, uint32_t* out_dev, uint64_t n, uint32_t key0, uint32_t key1) {
  if (rt_status e = check_ctx(c)) return e;
  if (!ctr_dev || !out_dev) return fail(c, RT_ERR_ARG, "rt_philox: null pointer");
  if (n == 0) return RT_OK;
  cudaSetDevice(c->device);
  launch_philox(ctr_dev, out_dev, n, key0, key1, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RT_OK;
}

rt_status rt_trace_closest(rt_ctx* c, const float* o_dev, const float* d_dev, uint64_t n, float* t_dev,
                           int32_t* prim_dev) {
  if (rt_status e = check_ctx(c)) return e;
  if (!c->has_scene) return fail(c, RT_ERR_STATE, "rt_trace_closest: no scene");
  if (!o_dev || !d_dev || !t_dev || !prim_dev) return fail(c, RT_ERR_ARG, "rt_trace_closest: null pointer");
  if (n == 0) return RT_OK;
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaMemsetAsync(c->wb.status, 0, sizeof(uint32_t), c->stream));
  launch_trace_closest_rays(dev_scene(c), o_dev, d_dev, n, t_dev, prim_dev, c->wb.status, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->wb.status, 4, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return status_to_rt(c, *c->h_status);
}

rt_status rt_trace_shadow(rt_ctx* c, const float* o_dev, const float* d_dev, const uint32_t* band_dev, uint64_t n,
                          float* T_dev, uint32_t* n_glass_dev) {
  if (rt_status e = check_ctx(c)) return e;
  if (!c->has_scene || !c->has_spectra) return fail(c, RT_ERR_STATE, "rt_trace_shadow: scene and spectra required");
  if (!o_dev || !d_dev || !band_dev || !T_dev || !n_glass_dev) return fail(c, RT_ERR_ARG, "rt_trace_shadow: null");
  if (n == 0) return RT_OK;
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaMemsetAsync(c->wb.status, 0, sizeof(uint32_t), c->stream));
  launch_trace_shadow_rays(dev_scene(c), c->sp, o_dev, d_dev, band_dev, n, T_dev, n_glass_dev, c->wb.status,
                           c->stream);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->wb.status, 4, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return status_to_rt(c, *c->h_status);
}

rt_status rt_optics_eval(rt_ctx* c, const float* cos_dev, const float* n_dev, const float* k_dev,
                         const float* lambda_nm_dev, const float* d_dev, uint64_t count, float* R_dev, float* Rs_dev,
                         float* Ts_dev) {
  if (rt_status e = check_ctx(c)) return e;
  if (!cos_dev || !n_dev || !k_dev || !R_dev) return fail(c, RT_ERR_ARG, "rt_optics_eval: null pointer");
  if ((lambda_nm_dev || d_dev) && (!lambda_nm_dev || !d_dev || !Rs_dev || !Ts_dev))
    return fail(c, RT_ERR_ARG, "rt_optics_eval: slab outputs need lambda, d, Rs and Ts");
  if (count == 0) return RT_OK;
  cudaSetDevice(c->device);
  launch_optics(cos_dev, n_dev, k_dev, lambda_nm_dev, d_dev, count, R_dev, Rs_dev, Ts_dev, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RT_OK;
}

rt_status rt_xyz(rt_ctx* c, const double* spectral_dev, uint64_t n_pixels, uint32_t band_first, uint32_t band_count,
                 uint32_t spp, uint32_t mode, float* xyz_dev) {
  if (rt_status e = check_ctx(c)) return e;
  if (!c->has_spectra) return fail(c, RT_ERR_STATE, "rt_xyz: spectra required");
  if (!spectral_dev || !xyz_dev || spp == 0 || band_count == 0 || band_first + band_count > c->sp.n_bands ||
      mode > 2)
    return fail(c, RT_ERR_ARG, "rt_xyz: bad argument");
  if (mode != 2 && band_count > kXyzMaxBandsTc)
    return fail(c, RT_ERR_ARG, "rt_xyz: tensor-core XYZ takes at most 192 bands (use RT_XYZ_FP64)");
  if (((uintptr_t)spectral_dev & 15u) != 0) return fail(c, RT_ERR_ARG, "rt_xyz: spectral_dev must be 16-byte aligned");
  if (n_pixels == 0) return RT_OK;
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaMemsetAsync(c->wb.status, 0, sizeof(uint32_t), c->stream));
  XyzWeights xw;
  xw.w32 = c->d_cmfw + 3 * (size_t)band_first;
  xw.band_count = band_count;
  xw.kpad = (band_count + 15) / 16 * 16;
  launch_xyz(spectral_dev, n_pixels, xw, spp, (int)mode, xyz_dev, c->stream, c->wb.status, c->sms);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->wb.status, 4, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return status_to_rt(c, *c->h_status);
}

namespace {

rt_status guide_ready(rt_ctx* c) {
  if (rt_status e = check_ctx(c)) return e;
  if (!c->guide.init) return fail(c, RT_ERR_STATE, "guide not initialised (rt_guide_init after rt_load_scene)");
  return RT_OK;
}

uint64_t guide_wcount() { return guide_wsize(); }

}  // namespace

rt_status rt_guide_init(rt_ctx* c, const rt_guide_config* cfg_in, uint64_t seed) {
  if (rt_status e = check_ctx(c)) return e;
  if (!c->has_scene) return fail(c, RT_ERR_STATE, "rt_guide_init: load a scene first");
  rt_guide_config cfg{};
  if (cfg_in) cfg = *cfg_in;
  if (!cfg.log2_table) cfg.log2_table = 19;
  if (cfg.n_min == 0.0f) cfg.n_min = 16.0f;
  if (cfg.n_max == 0.0f) cfg.n_max = 2048.0f;
  if (cfg.lr_grid == 0.0f) cfg.lr_grid = 1e-2f;
  if (cfg.lr_mlp == 0.0f) cfg.lr_mlp = 1e-3f;
  if (cfg.beta1 == 0.0f) cfg.beta1 = 0.9f;
  if (cfg.beta2 == 0.0f) cfg.beta2 = 0.99f;
  if (cfg.eps == 0.0f) cfg.eps = 1e-15f;
  if (cfg.mis_alpha == 0.0f) cfg.mis_alpha = 0.7f;
  if (!cfg.guide_depth) cfg.guide_depth = 2;
  if (cfg.log2_table < 10 || cfg.log2_table > 22 || !(cfg.n_min >= 1.0f) || !(cfg.n_max >= cfg.n_min) ||
      !(cfg.mis_alpha > 0.0f && cfg.mis_alpha < 1.0f) || cfg.guide_depth > (uint32_t)kMaxDepth)
    return fail(c, RT_ERR_ARG, "rt_guide_init: bad configuration");
  auto& G = c->guide;
  cudaSetDevice(c->device);
  const uint64_t T = 1ull << cfg.log2_table;
  const uint64_t ng = (uint64_t)kGuideLevels * T * kGuideFeatures;
  if (G.n_grid != ng) {
    dfree(G.grid);
    dfree(G.mg);
    dfree(G.vg);
    dfree(G.dgrid);
    G.n_grid = 0;
    CUDA_TRY(c, cudaMalloc(&G.grid, ng * 4));
    CUDA_TRY(c, cudaMalloc(&G.mg, ng * 4));
    CUDA_TRY(c, cudaMalloc(&G.vg, ng * 4));
    CUDA_TRY(c, cudaMalloc(&G.dgrid, ng * 4));
    G.n_grid = ng;
  }
  if (!G.W) {
    CUDA_TRY(c, cudaMalloc(&G.W, guide_wcount() * 4));
    CUDA_TRY(c, cudaMalloc(&G.mW, guide_wcount() * 4));
    CUDA_TRY(c, cudaMalloc(&G.vW, guide_wcount() * 4));
    CUDA_TRY(c, cudaMalloc(&G.dW, guide_wcount() * 4));
    CUDA_TRY(c, cudaMalloc(&G.dWpart, (size_t)c->sms * guide_wcount() * 4));
    CUDA_TRY(c, cudaMalloc(&G.scratch, 64));
    CUDA_TRY(c, cudaMalloc(&G.pack, guide_wpack_bytes()));
  }
  G.cfg = cfg;
  GuideDev& d = G.dev;
  d.grid = G.grid;
  d.log2T = cfg.log2_table;
  // resolutions n_min b^l, b = (n_max / n_min)^(1 / (levels - 1)); the
  // relative 1e-12 keeps a product that is an integer in exact arithmetic
  // (16 x 2^7 = 2048) from rounding down to the integer below
  const double b = std::exp((std::log((double)cfg.n_max) - std::log((double)cfg.n_min)) / (kGuideLevels - 1));
  d.dense_mask = 0;
  for (int l = 0; l < kGuideLevels; ++l) {
    d.res[l] = (uint32_t)std::floor((double)cfg.n_min * std::pow(b, l) * (1.0 + 1e-12));
    const uint64_t r1 = (uint64_t)d.res[l] + 1;
    if (r1 * r1 * r1 <= T) d.dense_mask |= 1u << l;
  }
  for (int a = 0; a < 3; ++a) {
    d.lo[a] = c->lo[a];
    const float ext = c->hi[a] - c->lo[a];
    d.inv_ext[a] = ext > 0.0f ? 1.0f / ext : 0.0f;
  }
  launch_guide_init(G.grid, ng, G.W, seed, c->stream);
  CUDA_TRY(c, cudaMemsetAsync(G.mg, 0, ng * 4, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(G.vg, 0, ng * 4, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(G.mW, 0, guide_wcount() * 4, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(G.vW, 0, guide_wcount() * 4, c->stream));
  launch_guide_pack(G.W, G.pack, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  G.step = 0;
  G.init = true;
  return RT_OK;
}

rt_status rt_guide_set_params(rt_ctx* c, const float* grid, const float* W) {
  if (rt_status e = guide_ready(c)) return e;
  auto& G = c->guide;
  cudaSetDevice(c->device);
  if (grid) CUDA_TRY(c, cudaMemcpy(G.grid, grid, G.n_grid * 4, cudaMemcpyHostToDevice));
  if (W) CUDA_TRY(c, cudaMemcpy(G.W, W, guide_wcount() * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemsetAsync(G.mg, 0, G.n_grid * 4, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(G.vg, 0, G.n_grid * 4, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(G.mW, 0, guide_wcount() * 4, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(G.vW, 0, guide_wcount() * 4, c->stream));
  launch_guide_pack(G.W, G.pack, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  G.step = 0;
  return RT_OK;
}

rt_status rt_guide_get_params(rt_ctx* c, float* grid, float* W) {
  if (rt_status e = guide_ready(c)) return e;
  auto& G = c->guide;
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (grid) CUDA_TRY(c, cudaMemcpy(grid, G.grid, G.n_grid * 4, cudaMemcpyDeviceToHost));
  if (W) CUDA_TRY(c, cudaMemcpy(W, G.W, guide_wcount() * 4, cudaMemcpyDeviceToHost));
  return RT_OK;
}

rt_status rt_guide_eval(rt_ctx* c, const float* rec_dev, uint64_t n, float* Y_dev, float* q_dev) {
  if (rt_status e = guide_ready(c)) return e;
  if (!rec_dev || !Y_dev || !q_dev) return fail(c, RT_ERR_ARG, "rt_guide_eval: null pointer");
  if (((uintptr_t)rec_dev & 15u) != 0) return fail(c, RT_ERR_ARG, "rt_guide_eval: records must be 16-byte aligned");
  if (n == 0) return RT_OK;
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaMemsetAsync(c->wb.status, 0, 4, c->stream));
  launch_guide_eval(c->guide.dev, c->guide.pack, rec_dev, n, Y_dev, q_dev, c->wb.status, c->sms, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->wb.status, 4, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return status_to_rt(c, *c->h_status);
}

// Gradient of one batch into G.dgrid / G.dW (enqueued, no synchronisation).
static void guide_grad_enqueue(rt_ctx* c, const float* rec_dev, uint64_t n) {
  auto& G = c->guide;
  cudaMemsetAsync(G.dgrid, 0, G.n_grid * 4, c->stream);
  cudaMemsetAsync(G.dW, 0, guide_wcount() * 4, c->stream);
  cudaMemsetAsync(G.scratch, 0, 64, c->stream);
  launch_guide_train(G.dev, G.pack, rec_dev, n, G.scratch, G.dW, G.dWpart, G.dgrid, G.scratch + 1, c->wb.status, c->sms,
                     c->stream);
}

// Adam step on the gradient in G.dgrid / G.dW, then repack the BF16 weights.
static void guide_update_enqueue(rt_ctx* c) {
  auto& G = c->guide;
  G.step += 1;
  const float c1 = (float)(1.0 / (1.0 - std::pow((double)G.cfg.beta1, (double)G.step)));
  const float c2 = (float)(1.0 / (1.0 - std::pow((double)G.cfg.beta2, (double)G.step)));
  launch_adam(G.grid, G.dgrid, G.mg, G.vg, G.n_grid, G.cfg.lr_grid, G.cfg.beta1, G.cfg.beta2, G.cfg.eps, c1, c2,
              c->stream);
  launch_adam(G.W, G.dW, G.mW, G.vW, guide_wcount(), G.cfg.lr_mlp, G.cfg.beta1, G.cfg.beta2, G.cfg.eps, c1, c2,
              c->stream);
  launch_guide_pack(G.W, G.pack, c->stream);
}

static void guide_train_enqueue(rt_ctx* c, const float* rec, uint64_t n) {
  guide_grad_enqueue(c, rec, n);
  guide_update_enqueue(c);
}

static rt_status guide_grad_impl(rt_ctx* c, const float* rec_dev, uint64_t n, float* loss_host) {
  auto& G = c->guide;
  CUDA_TRY(c, cudaMemsetAsync(c->wb.status, 0, 4, c->stream));
  guide_grad_enqueue(c, rec_dev, n);
  CUDA_TRY(c, cudaGetLastError());
  if (loss_host) CUDA_TRY(c, cudaMemcpyAsync(loss_host, G.scratch + 1, 4, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->wb.status, 4, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return status_to_rt(c, *c->h_status);
}

rt_status rt_guide_grad(rt_ctx* c, const float* rec_dev, uint64_t n, float* loss, float* dgrid_dev, float* dW_dev) {
  if (rt_status e = guide_ready(c)) return e;
  if (!rec_dev || n == 0) return fail(c, RT_ERR_ARG, "rt_guide_grad: no records");
  if (((uintptr_t)rec_dev & 15u) != 0) return fail(c, RT_ERR_ARG, "rt_guide_grad: records must be 16-byte aligned");
  cudaSetDevice(c->device);
  if (rt_status e = guide_grad_impl(c, rec_dev, n, loss)) return e;
  auto& G = c->guide;
  if (dgrid_dev) CUDA_TRY(c, cudaMemcpyAsync(dgrid_dev, G.dgrid, G.n_grid * 4, cudaMemcpyDeviceToDevice, c->stream));
  if (dW_dev) CUDA_TRY(c, cudaMemcpyAsync(dW_dev, G.dW, guide_wcount() * 4, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RT_OK;
}

rt_status rt_guide_train_step(rt_ctx* c, const float* rec_dev, uint64_t n, float* loss) {
  if (rt_status e = guide_ready(c)) return e;
  if (!rec_dev || n == 0) return fail(c, RT_ERR_ARG, "rt_guide_train_step: no records");
  if (((uintptr_t)rec_dev & 15u) != 0)
    return fail(c, RT_ERR_ARG, "rt_guide_train_step: records must be 16-byte aligned");
  cudaSetDevice(c->device);
  if (rt_status e = guide_grad_impl(c, rec_dev, n, loss)) return e;
  guide_update_enqueue(c);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RT_OK;
}

rt_status rt_guide_sample_step(rt_ctx* c, const rt_guide_vertex* v_dev, uint32_t n, uint32_t k, uint32_t sample,
                               uint32_t band_first, uint32_t band_count, uint64_t seed, rt_guide_step_out* out_dev) {
  if (rt_status e = guide_ready(c)) return e;
  if (!c->has_spectra) return fail(c, RT_ERR_STATE, "rt_guide_sample_step: set spectra first");
  if (!v_dev || !out_dev) return fail(c, RT_ERR_ARG, "rt_guide_sample_step: null pointer");
  if ((((uintptr_t)v_dev) | ((uintptr_t)out_dev)) & 15u)
    return fail(c, RT_ERR_ARG, "rt_guide_sample_step: buffers must be 16-byte aligned");
  if (band_count == 0 || band_first + band_count > c->sp.n_bands || n % band_count != 0 || n > (1u << 24))
    return fail(c, RT_ERR_ARG, "rt_guide_sample_step: bad band range or vertex count");
  if (k < 1 || k + 1 >= (uint32_t)kMaxDepth) return fail(c, RT_ERR_ARG, "rt_guide_sample_step: vertex index");
  if (n == 0) return RT_OK;
  cudaSetDevice(c->device);
  cudaStream_t st = c->stream;
  DevTemp<float4> gq, sq, qout, raw;
  DevTemp<float> L, wesc, Lfinal;
  DevTemp<uint32_t> sig, status;
  DevTemp<double> accum;
  DevTemp<Counters> cnt;
  CUDA_TRY(c, cudaMalloc(&gq.p, (size_t)n * 3 * sizeof(float4)));
  CUDA_TRY(c, cudaMalloc(&sq.p, (size_t)n * 2 * sizeof(float4)));
  CUDA_TRY(c, cudaMalloc(&qout.p, (size_t)n * 2 * sizeof(float4)));
  CUDA_TRY(c, cudaMalloc(&raw.p, (size_t)n * kRawF4 * sizeof(float4)));
  CUDA_TRY(c, cudaMalloc(&L.p, (size_t)n * sizeof(float)));
  CUDA_TRY(c, cudaMalloc(&wesc.p, (size_t)n * sizeof(float)));
  CUDA_TRY(c, cudaMalloc(&Lfinal.p, (size_t)n * sizeof(float)));
  CUDA_TRY(c, cudaMalloc(&sig.p, (size_t)n * sizeof(uint32_t)));
  CUDA_TRY(c, cudaMalloc(&status.p, sizeof(uint32_t)));
  CUDA_TRY(c, cudaMalloc(&accum.p, (size_t)n * sizeof(double)));
  CUDA_TRY(c, cudaMalloc(&cnt.p, (size_t)(k + 2) * sizeof(Counters)));
  std::vector<Counters> hc(k + 2);
  std::memset(hc.data(), 0, hc.size() * sizeof(Counters));
  hc[k].g_count = n;
  CUDA_TRY(c, cudaMemcpyAsync(cnt.p, hc.data(), hc.size() * sizeof(Counters), cudaMemcpyHostToDevice, st));
  CUDA_TRY(c, cudaMemsetAsync(raw.p, 0, (size_t)n * kRawF4 * sizeof(float4), st));
  CUDA_TRY(c, cudaMemsetAsync(L.p, 0, (size_t)n * sizeof(float), st));
  CUDA_TRY(c, cudaMemsetAsync(wesc.p, 0, (size_t)n * sizeof(float), st));
  CUDA_TRY(c, cudaMemsetAsync(accum.p, 0, (size_t)n * sizeof(double), st));
  CUDA_TRY(c, cudaMemsetAsync(status.p, 0, sizeof(uint32_t), st));
  // vertex i: path of pixel i / band_count, band band_first + i % band_count
  WaveParams w{};
  w.n = n;
  w.s0 = sample;
  w.r0 = 0;
  w.PB = n;
  w.band_first = band_first;
  w.band_count = band_count;
  w.spp = sample + 1;
  w.depth = k + 1;
  w.key0 = (uint32_t)seed;
  w.key1 = (uint32_t)(seed >> 32);
  w.n_bands = c->sp.n_bands;
  w.nb = 1;
  w.B = band_count;
  w.acc_stride = band_count;
  GuideWave gw{};
  gw.on = true;
  gw.depth = k;
  gw.alpha = c->guide.cfg.mis_alpha;
  gw.gq = gq.p;
  gw.wesc = wesc.p;
  gw.collect = 1;
  gw.slots_per_vertex = 0;  // the one slot of path i is raw[i] whatever k is
  gw.raw = raw.p;
  gw.Lfinal = Lfinal.p;
  WaveBufs b{};
  b.q[(k + 1) & 1] = qout.p;
  b.q[k & 1] = qout.p;
  b.sq = sq.p;
  b.L = L.p;
  b.sig = sig.p;
  b.cnt = cnt.p;
  b.status = status.p;
  b.cap = n;
  launch_guide_step_pack(v_dev, n, gq.p, sq.p, st);
  launch_guide_sample(c->guide.dev, c->guide.pack, c->sp, w, k, gw, b, accum.p, Probe{nullptr, nullptr, nullptr},
                      false, c->sms, st);
  launch_guide_step_gather(v_dev, n, k, gw, b, out_dev, st);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaMemcpyAsync(c->h_status, status.p, 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  return status_to_rt(c, *c->h_status);
}

rt_status rt_autotune(rt_ctx* c, const rt_camera* cams, uint32_t n_cams, uint32_t band_first, uint32_t band_count,
                      uint32_t spp_probe, uint32_t depth, rt_render_opts* opts, rt_autotune_report* report) {
  if (rt_status e = check_ctx(c)) return e;
  if (!opts) return fail(c, RT_ERR_ARG, "rt_autotune: opts is required");
  if (spp_probe == 0) spp_probe = 1;
  rt_render_opts base = *opts;
  base.probe_map_dev = nullptr;
  base.probe_L_dev = nullptr;
  base.probe_sig_dev = nullptr;
  base.use_graph = 0;
  base.accumulate = 0;
  base.guide_train_steps = 0;
  base.guide_collect = 0;
  const bool timing = c->timing, counting = c->counting;
  c->timing = false;
  c->counting = false;
  uint32_t trials = 0;
  float default_ms = 0.0f;
  auto run = [&](const rt_render_opts& o, float* ms) -> rt_status {
    rt_stats st;
    // warm-up render, then the timed one
    for (int rep = 0; rep < 2; ++rep) {
      rt_status e = render_impl(c, cams, n_cams, band_first, band_count, spp_probe, depth, 0x5eed, &o, nullptr,
                                nullptr, &st);
      if (e != RT_OK) return e;
    }
    *ms = st.ms_render;
    ++trials;
    return RT_OK;
  };
  float best_ms;
  rt_status e = run(base, &best_ms);
  if (e != RT_OK) {
    c->timing = timing;
    c->counting = counting;
    return e;
  }
  default_ms = best_ms;
  rt_render_opts best = base;
  auto try_opt = [&](rt_render_opts o) -> rt_status {
    float ms;
    rt_status e2 = run(o, &ms);
    if (e2 != RT_OK) return e2;
    if (ms < best_ms) {
      best_ms = ms;
      best = o;
    }
    return RT_OK;
  };
  // coordinate descent: paths in flight, leaf batch, closest-hit loop,
  // sun-ray loop, block
  const uint32_t waves[] = {1u << 21, 1u << 22, 1u << 23, 1u << 24};
  const uint32_t leaf[] = {12, 16, 32};
  const uint32_t tl[][2] = {{8, 8}, {2, 8}, {4, 4}, {4, 16}};
  const uint32_t sl[][2] = {{8, 12}, {2, 12}, {4, 4}, {4, 24}};
  const uint32_t blocks[] = {128, 64, 96};
  rt_render_opts o;
  for (uint32_t wv : waves) {
    o = best;
    o.wave_capacity = wv;
    if ((e = try_opt(o))) break;
  }
  for (size_t i = 0; e == RT_OK && base.trace_variant == 0 && i < sizeof(leaf) / sizeof(leaf[0]); ++i) {
    o = best;
    o.leaf_batch = leaf[i];
    e = try_opt(o);
  }
  for (size_t i = 0; e == RT_OK && i < sizeof(tl) / sizeof(tl[0]); ++i) {
    o = best;
    o.trace_steps = tl[i][0];
    o.trace_refill = tl[i][1];
    e = try_opt(o);
  }
  for (size_t i = 0; e == RT_OK && i < sizeof(sl) / sizeof(sl[0]); ++i) {
    o = best;
    o.shadow_steps = sl[i][0];
    o.shadow_refill = sl[i][1];
    e = try_opt(o);
  }
  for (size_t i = 0; e == RT_OK && i < sizeof(blocks) / sizeof(blocks[0]); ++i) {
    o = best;
    o.trace_block = blocks[i];
    e = try_opt(o);
  }
  c->timing = timing;
  c->counting = counting;
  if (e != RT_OK) return e;
  // keep the caller's own fields; copy the tuned ones
  opts->wave_capacity = best.wave_capacity;
  opts->trace_steps = best.trace_steps;
  opts->trace_refill = best.trace_refill;
  opts->shadow_steps = best.shadow_steps;
  opts->shadow_refill = best.shadow_refill;
  opts->trace_block = best.trace_block;
  opts->leaf_batch = best.leaf_batch;
  if (report) {
    report->trials = trials;
    report->best_ms = best_ms;
    report->default_ms = default_ms;
  }
  return RT_OK;
}

rt_status rt_probe_l2(rt_ctx* c, uint64_t bytes, uint32_t iters, float* gbs) {
  if (rt_status e = check_ctx(c)) return e;
  if (!gbs || bytes < 16 || bytes > (96ull << 20) || iters == 0) return fail(c, RT_ERR_ARG, "rt_probe_l2: bad argument");
  cudaSetDevice(c->device);
  const size_t n4 = bytes / 16;
  float4* buf = nullptr;
  float* sink = nullptr;
  CUDA_TRY(c, cudaMalloc(&buf, n4 * 16));
  CUDA_TRY(c, cudaMalloc(&sink, 16));
  CUDA_TRY(c, cudaMemsetAsync(buf, 0, n4 * 16, c->stream));
  launch_l2_probe(buf, n4, 2, sink, c->stream, c->sms);  // warm L2
  CUDA_TRY(c, cudaEventRecord(c->ev[0], c->stream));
  launch_l2_probe(buf, n4, (int)iters, sink, c->stream, c->sms);
  CUDA_TRY(c, cudaEventRecord(c->ev[1], c->stream));
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
  cudaFree(buf);
  cudaFree(sink);
  *gbs = (float)((double)n4 * 16.0 * iters / (ms * 1e-3) / 1e9);
  return RT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// photon mapping (section 4)
// ---------------------------------------------------------------------------

// Emission geometry of the photon pass (FP64 on the host): a disk
// perpendicular to the sun, tangent to the scene's bounding sphere (centre
// c, radius R) on the sun's side, radius R_d = R (tan a + 1 / cos a) so that
// every ray of the cone that meets the sphere starts on it; each of the N
// photons of a band carries L_sun cos Omega pi R_d^2 / N.
// Portal table for portal emission: the thin-glass triangles that face the
// sun, {v0, v1, v2, (sun-side unit normal, 1 / (s . n))}, and the cumulative
// share of A |s . n| (FP64 sums, stored as float, the last entry 1).
static rt_status photon_portals(rt_ctx* c, float4** d_portal, float** d_cdf, uint32_t* n_out, double* W_out) {
  std::vector<float4> tab;
  std::vector<double> cum;
  double W = 0.0;
  const double* s = c->sun_d;
  for (size_t t = 0; t + 9 <= c->glass.size(); t += 9) {
    const float* g = c->glass.data() + t;
    double e1[3], e2[3], n[3];
    for (int a = 0; a < 3; ++a) {
      e1[a] = (double)g[3 + a] - g[a];
      e2[a] = (double)g[6 + a] - g[a];
    }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double a2 = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(a2 > 0.0)) continue;
    for (int a = 0; a < 3; ++a) n[a] /= a2;
    double cs = n[0] * s[0] + n[1] * s[1] + n[2] * s[2];
    if (cs == 0.0) continue;
    if (cs < 0.0) {
      for (int a = 0; a < 3; ++a) n[a] = -n[a];
      cs = -cs;
    }
    tab.push_back(make_float4(g[0], g[1], g[2], 0.0f));
    tab.push_back(make_float4(g[3], g[4], g[5], 0.0f));
    tab.push_back(make_float4(g[6], g[7], g[8], 0.0f));
    tab.push_back(make_float4((float)n[0], (float)n[1], (float)n[2], (float)(1.0 / cs)));
    W += 0.5 * a2 * cs;
    cum.push_back(W);
  }
  if (tab.empty()) return fail(c, RT_ERR_ARG, "portal emission: no thin-glass triangle faces the sun");
  std::vector<float> cdf(cum.size());
  for (size_t q = 0; q < cum.size(); ++q) cdf[q] = (float)(cum[q] / W);
  cdf.back() = 1.0f;
  CUDA_TRY(c, cudaMalloc(d_portal, tab.size() * sizeof(float4)));
  CUDA_TRY(c, cudaMalloc(d_cdf, cdf.size() * sizeof(float)));
  CUDA_TRY(c, cudaMemcpy(*d_portal, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(*d_cdf, cdf.data(), cdf.size() * sizeof(float), cudaMemcpyHostToDevice));
  *n_out = (uint32_t)cum.size();
  *W_out = W;
  return RT_OK;
}

static void photon_setup(const rt_ctx* c, uint32_t N, uint64_t seed, PhotonPass& pp) {
  double ctr[3], R2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    ctr[a] = 0.5 * ((double)c->lo[a] + (double)c->hi[a]);
    const double e = (double)c->hi[a] - (double)c->lo[a];
    R2 += e * e;
  }
  const double R = 0.5 * std::sqrt(R2);
  const double cm = c->cos_max_d;
  const double sa = std::sqrt(std::max(0.0, 1.0 - cm * cm));
  const double Rd = R * (sa / cm + 1.0 / cm);
  const double omega = 2.0 * M_PI * (1.0 - cm);
  // orthonormal basis around the sun (the same construction as the kernels')
  const double* n = c->sun_d;
  const double sign = std::copysign(1.0, n[2]);
  const double aa = -1.0 / (sign + n[2]);
  const double bb = n[0] * n[1] * aa;
  pp.t1 = make_float3((float)(1.0 + sign * n[0] * n[0] * aa), (float)(sign * bb), (float)(-sign * n[0]));
  pp.t2 = make_float3((float)bb, (float)(sign + n[1] * n[1] * aa), (float)(-n[1]));
  pp.c0 = make_float3((float)(ctr[0] + R * n[0]), (float)(ctr[1] + R * n[1]), (float)(ctr[2] + R * n[2]));
  pp.Rd = (float)Rd;
  pp.flux = (float)(omega * M_PI * Rd * Rd / (double)N);
  pp.N = N;
  pp.key0 = (uint32_t)seed;
  pp.key1 = (uint32_t)(seed >> 32) ^ 0x50484F54u;
}

rt_status rt_photon_records(rt_ctx* c, uint32_t band_first, uint32_t band_count, uint32_t n_photons, uint32_t depth,
                            uint64_t seed, uint32_t emission, float* rec_dev, uint8_t* cls_dev) {
  if (rt_status e = check_ctx(c)) return e;
  if (!c->has_scene || !c->has_spectra) return fail(c, RT_ERR_STATE, "rt_photon_records: scene and spectra required");
  if (!rec_dev || ((uintptr_t)rec_dev & 15u)) return fail(c, RT_ERR_ARG, "rt_photon_records: rec_dev must be 16-byte aligned");
  if (band_count == 0 || band_first + band_count > c->sp.n_bands || band_first + band_count < band_first)
    return fail(c, RT_ERR_ARG, "rt_photon_records: band range outside the spectra");
  if (n_photons == 0 || depth == 0 || depth > (uint32_t)kMaxDepth)
    return fail(c, RT_ERR_ARG, "rt_photon_records: n_photons >= 1 and depth 1..64");
  const uint64_t slots = (uint64_t)band_count * n_photons * depth;
  if (slots > (1ull << 28)) return fail(c, RT_ERR_ARG, "rt_photon_records: more than 2^28 slots");
  if (!(c->cos_max_d > std::cos(1.0))) return fail(c, RT_ERR_ARG, "rt_photon_records: sun half angle must be below 1 rad");
  if (emission > 1) return fail(c, RT_ERR_ARG, "rt_photon_records: emission is 0 (disk) or 1 (portals)");
  cudaSetDevice(c->device);
  cudaStream_t st = c->stream;
  PhotonPass pp{};
  photon_setup(c, n_photons, seed, pp);
  DevTemp<float4> portal;
  DevTemp<float> cdf;
  if (emission == 1) {
    double W = 0.0;
    if (rt_status e = photon_portals(c, &portal.p, &cdf.p, &pp.n_portal, &W)) return e;
    pp.portal = portal.p;
    pp.cdf = cdf.p;
    pp.emission = 1;
    pp.flux = (float)(2.0 * M_PI * (1.0 - c->cos_max_d) * W / (double)n_photons);
  }
  DevTemp<uint32_t> kvt;
  CUDA_TRY(c, cudaMalloc(&kvt.p, slots * 2 * sizeof(uint32_t)));
  uint32_t* kv = kvt.p;
  pp.band0 = band_first;
  pp.Bc = band_count;
  pp.depth = depth;
  pp.inv_cell[0] = pp.inv_cell[1] = 1.0f;
  pp.hbits = 8;
  CUDA_TRY(c, cudaMemsetAsync(c->wb.status, 0, sizeof(uint32_t), st));
  launch_photon_trace(dev_scene(c), c->sp, pp, (float4*)rec_dev, kv, kv + slots, cls_dev, c->wb.status, c->sms, st);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->wb.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  return status_to_rt(c, *c->h_status);
}

rt_status rt_render_photons(rt_ctx* c, const rt_camera* cams, uint32_t n_cams, uint32_t band_first,
                            uint32_t band_count, uint32_t spp, uint32_t depth, uint64_t seed,
                            const rt_photon_opts* opts, double* spectral_dev, float* xyz_dev, rt_stats* stats) {
  if (rt_status e = check_ctx(c)) return e;
  if (!c->has_scene || !c->has_spectra) return fail(c, RT_ERR_STATE, "rt_render_photons: scene and spectra must be set");
  if (!cams || n_cams == 0 || n_cams > (uint32_t)kMaxCams) return fail(c, RT_ERR_ARG, "rt_render_photons: 1..64 cameras");
  if (band_count == 0 || band_first + band_count > c->sp.n_bands || band_first + band_count < band_first)
    return fail(c, RT_ERR_ARG, "rt_render_photons: band range outside the spectra");
  if (spp == 0) return fail(c, RT_ERR_ARG, "rt_render_photons: spp must be >= 1");
  if (depth == 0 || depth > (uint32_t)kMaxDepth) return fail(c, RT_ERR_ARG, "rt_render_photons: depth must be 1..64");
  rt_photon_opts o{};
  if (opts) o = *opts;
  const uint32_t N = o.n_photons ? o.n_photons : 65536u;
  const uint32_t pd = o.photon_depth ? o.photon_depth : 4u;
  const uint32_t hb = o.log2_cells ? o.log2_cells : 16u;
  if (pd > (uint32_t)kMaxDepth) return fail(c, RT_ERR_ARG, "rt_render_photons: photon_depth is 1..64");
  if ((uint64_t)N * pd > kPhotonMaxSlots) return fail(c, RT_ERR_ARG, "rt_render_photons: n_photons x photon_depth above 2^24");
  if (hb < 8 || hb > 20) return fail(c, RT_ERR_ARG, "rt_render_photons: log2_cells is 8..20");
  if (o.xyz_mode > 2) return fail(c, RT_ERR_ARG, "rt_render_photons: unknown xyz_mode");
  if (o.emission > 1) return fail(c, RT_ERR_ARG, "rt_render_photons: emission is 0 (disk) or 1 (portals)");
  if (o.xyz_mode != 2 && band_count > kXyzMaxBandsTc)
    return fail(c, RT_ERR_ARG, "rt_render_photons: tensor-core XYZ takes at most 192 bands (use RT_XYZ_FP64)");
  if (!(c->cos_max_d > std::cos(1.0)))
    return fail(c, RT_ERR_ARG, "rt_render_photons: photon emission needs a sun half angle below 1 rad");
  if ((o.probe_map_dev != nullptr) != (o.probe_L_dev != nullptr) ||
      (o.probe_map_dev != nullptr) != (o.probe_sig_dev != nullptr))
    return fail(c, RT_ERR_ARG, "rt_render_photons: probe_map, probe_L and probe_sig go together");
  double diag2 = 0.0;
  for (int a = 0; a < 3; ++a) diag2 += ((double)c->hi[a] - c->lo[a]) * ((double)c->hi[a] - c->lo[a]);
  const double rc = o.r_caustic > 0.0f ? (double)o.r_caustic : 0.005 * std::sqrt(diag2);
  const double rg = o.r_global > 0.0f ? (double)o.r_global : 0.02 * std::sqrt(diag2);
  if (!(rc > 0.0) || !(rg > 0.0) || !std::isfinite(rc) || !std::isfinite(rg))
    return fail(c, RT_ERR_ARG, "rt_render_photons: gather radii must be positive");
  uint64_t npix = 0;
  if (rt_status e = stage_cameras(c, cams, n_cams, "rt_render_photons", &npix)) return e;
  const uint64_t ACC64 = npix * band_count;
  if (ACC64 >= (1ull << 32)) return fail(c, RT_ERR_ARG, "rt_render_photons: pixels x bands must be below 2^32");
  // bands per chunk: the chunk's slots fit one sort, and its two key tables
  // (2 x Bc x 2^hb ranges) stay at 2^26 entries (keys far below the empty key)
  uint32_t Bc = (uint32_t)std::min<uint64_t>(band_count, kPhotonMaxSlots / ((uint64_t)N * pd));
  Bc = std::max<uint32_t>(1u, std::min<uint32_t>(Bc, 1u << (25 - hb)));
  const size_t slots = (size_t)Bc * N * pd;
  const size_t table = (size_t)2 * Bc << hb;
  cudaSetDevice(c->device);
  cudaStream_t st = c->stream;
  if (spectral_dev && ((uintptr_t)spectral_dev & 15u) != 0)
    return fail(c, RT_ERR_ARG, "rt_render_photons: spectral_dev must be 16-byte aligned");
  auto& B = c->ph;
  if (B.slots < slots) {
    dfree(B.rec);
    dfree(B.rec_sorted);
    for (int q = 0; q < 2; ++q) {
      dfree(B.keys[q]);
      dfree(B.vals[q]);
    }
    dfree(B.hist);
    B.slots = 0;
    CUDA_TRY(c, cudaMalloc(&B.rec, slots * sizeof(float4)));
    CUDA_TRY(c, cudaMalloc(&B.rec_sorted, slots * sizeof(float4)));
    for (int q = 0; q < 2; ++q) {
      CUDA_TRY(c, cudaMalloc(&B.keys[q], slots * sizeof(uint32_t)));
      CUDA_TRY(c, cudaMalloc(&B.vals[q], slots * sizeof(uint32_t)));
    }
    CUDA_TRY(c, cudaMalloc(&B.hist, radix_sort_hist_words((uint32_t)slots) * sizeof(uint32_t)));
    B.slots = slots;
  }
  if (B.table < table) {
    dfree(B.start);
    dfree(B.end);
    B.table = 0;
    CUDA_TRY(c, cudaMalloc(&B.start, table * sizeof(uint32_t)));
    CUDA_TRY(c, cudaMalloc(&B.end, table * sizeof(uint32_t)));
    B.table = table;
  }
  double* accum = spectral_dev;
  if (!accum) {
    if (c->accum_cap < ACC64) {
      dfree(c->d_accum);
      c->accum_cap = 0;
      CUDA_TRY(c, cudaMalloc(&c->d_accum, ACC64 * sizeof(double)));
      c->accum_cap = ACC64;
    }
    accum = c->d_accum;
  }
  PhotonPass pp{};
  photon_setup(c, N, seed, pp);
  DevTemp<float4> portal;
  DevTemp<float> cdf;
  if (o.emission == 1) {
    double W = 0.0;
    if (rt_status e = photon_portals(c, &portal.p, &cdf.p, &pp.n_portal, &W)) return e;
    pp.portal = portal.p;
    pp.cdf = cdf.p;
    pp.emission = 1;
    pp.flux = (float)(2.0 * M_PI * (1.0 - c->cos_max_d) * W / (double)N);
  }
  pp.depth = pd;
  pp.inv_cell[0] = (float)(1.0 / (2.0 * rc));
  pp.inv_cell[1] = (float)(1.0 / (2.0 * rg));
  pp.hbits = hb;
  PhotonMaps M{};
  M.start = B.start;
  M.end = B.end;
  M.rec = B.rec_sorted;
  M.r2[0] = (float)(rc * rc);
  M.r2[1] = (float)(rg * rg);
  M.inv_cell[0] = pp.inv_cell[0];
  M.inv_cell[1] = pp.inv_cell[1];
  // Epanechnikov kernel 1 - d^2 / r^2 over the disk of radius r: norm 2 / (pi r^2)
  M.norm[0] = (float)(2.0 / (M_PI * rc * rc));
  M.norm[1] = (float)(2.0 / (M_PI * rg * rg));
  M.hbits = hb;
  // camera pass: the wavefront kernels of rt_render (camera rays, closest
  // hit, shading that ends at the first Lambertian vertex, sun rays), one
  // band chunk at a time, into the chunk's columns of the spectral image
  const Probe probe{o.probe_map_dev, o.probe_L_dev, o.probe_sig_dev};
  uint32_t cap = (uint32_t)std::min<uint64_t>(std::min<uint64_t>(1u << 23, npix * Bc), kMaxWave);
  cap = std::max<uint32_t>(cap, 1u);
  if (rt_status e = ensure_wave(c, cap)) return e;
  LaunchCfg lc;
  lc.block_trace = 128;
  lc.block_shade = 256;
  lc.grid_trace = c->sms * trace_blocks_per_sm(lc.block_trace);
  lc.grid_shadow = c->sms * shadow_blocks_per_sm(lc.block_trace);
  lc.grid_shade = c->sms * 8;
  lc.counting = false;
  lc.record = o.probe_map_dev != nullptr;
  lc.variant = 0;
  lc.leaf_min = kDefaultLeafBatch;
  lc.sort_rays = false;
  lc.trace_steps = kDefaultTraceSteps;
  lc.trace_refill = kDefaultTraceRefill;
  lc.shadow_steps = kDefaultShadowSteps;
  lc.shadow_refill = kDefaultShadowRefill;
  WaveParams w{};
  w.spp = spp;
  w.depth = depth;
  w.key0 = (uint32_t)seed;
  w.key1 = (uint32_t)(seed >> 32);
  w.s_base = 0;
  w.n_bands = c->sp.n_bands;
  w.nb = 1;
  w.acc_stride = band_count;
  const DevScene S = dev_scene(c);
  struct Events {
    std::vector<cudaEvent_t> v;
    ~Events() {
      for (auto e : v) cudaEventDestroy(e);
    }
  } evs;
  std::vector<cudaEvent_t>& ev = evs.v;
  auto mark = [&]() {
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, st);
    ev.push_back(e);
  };
  int launches = 0;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_cams, c->h_cams, sizeof(DevCam) * n_cams, cudaMemcpyHostToDevice, st));
  CUDA_TRY(c, cudaMemsetAsync(accum, 0, ACC64 * sizeof(double), st));
  CUDA_TRY(c, cudaMemsetAsync(c->wb.status, 0, sizeof(uint32_t), st));
  mark();
  for (uint32_t cb = band_first; cb < band_first + band_count; cb += Bc) {
    const uint32_t bc = std::min<uint32_t>(Bc, band_first + band_count - cb);
    const uint32_t n = bc * N * pd;
    pp.band0 = cb;
    pp.Bc = bc;
    launch_photon_trace(S, c->sp, pp, B.rec, B.keys[0], B.vals[0], nullptr, c->wb.status, c->sms, st);
    mark();
    const int r = launch_radix_sort(B.keys, B.vals, n, 32, B.hist, st);
    CUDA_TRY(c, cudaMemsetAsync(B.start, 0, ((size_t)2 * bc << hb) * sizeof(uint32_t), st));
    CUDA_TRY(c, cudaMemsetAsync(B.end, 0, ((size_t)2 * bc << hb) * sizeof(uint32_t), st));
    launch_photon_maps(B.keys[r], B.vals[r], n, B.rec, B.rec_sorted, B.start, B.end, c->sms, st);
    mark();
    M.Bc = bc;
    w.band_first = cb;
    w.band_count = bc;
    w.B = bc;
    w.acc_off = cb - band_first;
    w.PB = (uint32_t)(npix * bc);
    // a wave holds at most one sample's paths of this chunk, so that it
    // spans two samples at most (path ids wrap once)
    const uint32_t wcap = std::min<uint32_t>(cap, w.PB);
    const uint64_t total = (uint64_t)w.PB * spp;
    for (uint64_t ws = 0; ws < total; ws += wcap) {
      w.n = (uint32_t)std::min<uint64_t>(wcap, total - ws);
      w.s0 = (uint32_t)(ws / w.PB);
      w.r0 = (uint32_t)(ws % w.PB);
      CUDA_TRY(c, cudaMemsetAsync(c->wb.cnt, 0, sizeof(Counters) * (depth + 2), st));
      launch_wave(lc, S, c->sp, c->d_cams, n_cams, w, c->wb, accum, probe, st, &launches, nullptr, nullptr, nullptr,
                  nullptr, c->sms, &M);
    }
    mark();
    launches += 1 + 16 + 1;  // photon trace, 4 radix passes of 4 kernels, ranges
  }
  CUDA_TRY(c, cudaGetLastError());
  if (xyz_dev) {
    XyzWeights xw;
    xw.w32 = c->d_cmfw + 3 * (size_t)band_first;
    xw.band_count = band_count;
    xw.kpad = (band_count + 15) / 16 * 16;
    launch_xyz(accum, npix, xw, spp, (int)o.xyz_mode, xyz_dev, st, c->wb.status, c->sms);
    ++launches;
    CUDA_TRY(c, cudaGetLastError());
  }
  mark();
  CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->wb.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->paths = ACC64 * spp;
    stats->kernel_launches = (uint32_t)launches;
    stats->waves = (uint32_t)((band_count + Bc - 1) / Bc);
    // stages: 0 photon pass, 1 photon maps (sort, ranges), 2 camera pass
    for (size_t q = 0; q + 3 < ev.size(); q += 3) {
      float a = 0, b = 0, d = 0;
      cudaEventElapsedTime(&a, ev[q], ev[q + 1]);
      cudaEventElapsedTime(&b, ev[q + 1], ev[q + 2]);
      cudaEventElapsedTime(&d, ev[q + 2], ev[q + 3]);
      stats->ms_stage[0] += a;
      stats->ms_stage[1] += b;
      stats->ms_stage[2] += d;
    }
    cudaEventElapsedTime(&stats->ms_render, ev.front(), ev[ev.size() - 2]);
    cudaEventElapsedTime(&stats->ms_xyz, ev[ev.size() - 2], ev.back());
  }
  return status_to_rt(c, *c->h_status);
}

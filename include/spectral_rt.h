/*
 * spectral_rt.h - C ABI of the GB300 spectral path tracer.
 *
 * The library renders a triangle scene lit by the sun with one wavelength band
 * per Monte Carlo path, the wavelength sub-domain of the paper's spectral
 * decomposition reduced to a work key ("Spectral domain decomposition method
 * for physically-based rendering of Royaumont abbey", title and section 5).
 * What each path computes follows the paper's physics:
 *   - materials carry a complex refractive index n(lambda) + i k(lambda)
 *     (section 3, Eq. 1): thin glass sheets (complex Fresnel plus Beer-Lambert
 *     absorption alpha = 4 pi k / lambda) and conductors;
 *   - stone is Lambertian and the reflected radiance is the integral of
 *     section 4, Eq. 2, estimated by cosine sampling;
 *   - the sun is a directional source (section 3: a plane wave) with a cone of
 *     half angle a; its direct contribution is the sum of section 4, Eq. 3,
 *     estimated by next-event sampling of the cone through thin glass;
 *   - the spectrum of each pixel is accumulated in FP64 and converted to CIE
 *     XYZ (section 6: colorimetry from spectra).
 *
 * Conventions for every entry point:
 *   - Status codes are returned; nothing throws or aborts across the ABI.
 *     rt_last_error() gives a message for the last failure on a context.
 *   - Pointers named *_dev are device pointers (cudaMalloc / torch CUDA
 *     memory) on the context's device; they stay owned by the caller and are
 *     used on the context's stream.  All other pointers are host memory,
 *     read during the call and not retained.
 *   - Work is enqueued on the context's stream.  Functions that return
 *     results on the host, or a device status, synchronise that stream.
 *   - Arrays are densely packed, row-major, in the element types given.
 */
#ifndef SPECTRAL_RT_H
#define SPECTRAL_RT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RT_OK = 0,
  RT_ERR_ARG = 1,            /* invalid argument (null, zero size, out of range) */
  RT_ERR_SCENE = 2,          /* scene rejected: NaN/inf vertex, bad index, degenerate triangle */
  RT_ERR_OOM = 3,            /* device allocation failed */
  RT_ERR_CUDA = 4,           /* a CUDA runtime call failed; the context is now unusable */
  RT_ERR_QUEUE_OVERFLOW = 5, /* a device work queue exceeded its capacity (results invalid) */
  RT_ERR_TIMEOUT = 6,        /* a device loop hit its iteration cap (results invalid) */
  RT_ERR_STATE = 7,          /* call out of order (no scene / no spectra) or context poisoned */
  RT_ERR_STACK = 8           /* BVH traversal stack exhausted (results invalid) */
} rt_status;

typedef enum {
  RT_LAMBERT = 0,    /* diffuse stone, reflectance rho(lambda) */
  RT_THIN_GLASS = 1, /* thin sheet: complex Fresnel faces + Beer-Lambert interior, thickness d */
  RT_CONDUCTOR = 2,  /* metal: specular, complex Fresnel with n(lambda) + i k(lambda) */
  RT_EMISSIVE = 3,   /* test material: Lambertian rho plus emitted radiance le(lambda) */
  RT_DIELECTRIC = 4  /* solid refracting glass (section 3, Eq. 1): the triangles of a material of
                        this type form closed solids with outward (counter-clockwise) winding and
                        no other surface inside; Fresnel of the relative index, Snell refraction
                        with n(lambda), Beer-Lambert 4 pi k / lambda per metre inside; opaque to
                        sun rays.  Its thickness entry is ignored. */
} rt_material_type;

typedef enum {
  RT_XYZ_BF16X3 = 0, /* tensor cores, BF16 operands split in three terms, FP32 accumulate */
  RT_XYZ_BF16 = 1,   /* tensor cores, plain BF16 operands, FP32 accumulate */
  RT_XYZ_FP64 = 2    /* CUDA cores, FP64 (reference mode) */
} rt_xyz_mode;

typedef struct rt_ctx rt_ctx;

/* Pinhole camera: position, look-at point, up vector, vertical field of view
 * in degrees, image size.  Pixel (x, y) has y growing downwards. */
typedef struct {
  float pos[3];
  float look[3];
  float up[3];
  float vfov_deg;
  uint32_t width;
  uint32_t height;
} rt_camera;

typedef struct {
  uint32_t wave_capacity;  /* paths in flight per wave; 0 = library default (2^23) */
  uint32_t xyz_mode;       /* rt_xyz_mode */
  uint32_t trace_block;    /* threads per block of the traversal kernels, a multiple of 32 up to 128;
                            * 0 = 128 */
  uint32_t ctas_per_sm;    /* persistent CTAs per SM for traversal; 0 = occupancy limit */
  /* optional per-path records for parity checks: probe_map_dev[p] (uint32,
   * one per global pixel) is the probe slot of pixel p or 0xFFFFFFFF; each
   * probed path writes its radiance and event signature to
   * probe_L_dev / probe_sig_dev[(slot * spp + s) * band_count + j]. */
  const uint32_t* probe_map_dev;
  float* probe_L_dev;
  uint32_t* probe_sig_dev;
  uint32_t use_graph;      /* 1: the whole render (all waves, XYZ) is captured once per launch
                            * configuration into a CUDA graph and replayed (camera poses may change
                            * between replays); excludes timing, counting, probes and guide training */
  uint32_t trace_variant;  /* traversal: 0 = four-wide BVH with leaf batching (interior steps
                            * until leaf_batch lanes of a warp wait at a leaf, then one leaf step
                            * for all of them); binary BVH with 1 = while-while, 2 = one node or
                            * leaf per lane and step, 3 = leaf batching; 4 = closest hits over an
                            * eight-wide BVH (children in corner slots visited in the ray's octant
                            * order, leaf batching; host-built trees only); 5 = closest hits over
                            * the four-wide BVH stored with 8-bit child boxes (64-byte nodes; host-
                            * built trees only).  Every variant returns the same hits */
  /* persistent traversal warps refill idle lanes from the queue once at least
   * *_refill (1..32) lanes are idle, and run up to *_steps (>= 1) steps per
   * lane between refill checks; 0 = library default (tuned) */
  uint32_t trace_steps, trace_refill, shadow_steps, shadow_refill;
  /* learned guide (rt_guide_init first): 1 = at Lambertian vertices
   * 1..guide_depth the continuation is drawn from the guide with probability
   * mis_alpha, else by cosine sampling, weighted by the one-sample MIS pdf */
  uint32_t guided;
  uint32_t guide_collect;      /* keep training records of every n-th path of a wave; 0 = none */
  uint32_t guide_train_steps;  /* Adam steps after each wave on its records; 0 = guide frozen */
  uint32_t guide_batch;        /* records per step; 0 = the wave's records / steps */
  /* progressive rendering: this call renders samples [sample_first,
   * sample_first + spp) (Philox counters), adds them to spectral_dev when
   * accumulate = 1, and divides XYZ by spp_total (0 = spp) */
  uint32_t sample_first;
  uint32_t accumulate;
  uint32_t spp_total;
  uint32_t leaf_batch;     /* trace_variant 0: 1..32 waiting lanes start a leaf phase; 0 = default */
  uint32_t guide_order;    /* guided: 0 = guide queries in queue order (the default: measured
                            * faster), 1 = sorted by position first (Morton order of a 64^3 grid,
                            * so that a tile's hash-grid gathers share cache lines); the same bits */
  uint32_t ray_order;      /* 0 = queue order; 1 = rays of vertices >= 2 and sun rays traced in the
                            * order of a counting sort by origin cell (and direction octant): the
                            * same result, measured no faster on the nave */
  uint32_t bands_per_path; /* 0 or 1: every path carries one band (the method as specified);
                            * 4: path j of a pixel and sample carries the range's bands j + q G,
                            * q = 0..3, G = ceil(band_count / 4) (those inside the range), spread
                            * over the spectrum; they share its geometry until the first dispersive
                            * event (refraction into or out of solid glass), where one of them,
                            * chosen uniformly, goes on with weight n (1 - R) / (1 - p); thin-glass
                            * and solid-glass reflections choose with the bands' mean probability
                            * and weight each band by its own.  The same expectation per band; one
                            * closest-hit and one sun ray serve four bands.  The grouping depends
                            * on the band range, so disjoint ranges are independent estimates
                            * rather than bit-exact pieces of one render.  Excludes guided
                            * sampling and trace_variant != 0.  rt_stats.paths counts (pixel,
                            * sample, band) estimates in both modes */
  /* optional, for checks of the guide's training data: with guided = 1,
   * guide_collect = 1 and use_graph = 0, the training records of every path
   * in path order (no shuffling), written after each wave:
   * guide_records_dev[v][p][r][12] floats (device, caller-owned), v = guided
   * vertex 0..guide_depth - 1, p = s * pixels * band_count + pixel *
   * band_count + j the path (sample s counted from sample_first), r = 0 the
   * continuation record, 1 the sun-sample record, each in the record layout
   * of rt_guide_train_step ({pos, weight}, {normal, band group}, {omega, 0};
   * weight 0: {0,0,0,0}, {0,0,1,0}, {0,0,1,0}).  RT_ERR_ARG if these
   * conditions do not hold.  The continuation record's weight is
   * L_in cos / p_mix, L_in the radiance the path gathered after the vertex
   * divided by its throughput there; the sun record's is
   * L_sun T_r cos / p_cone (section 4, Eqs. 2 and 3 sampled by the two
   * strategies of the vertex). */
  float* guide_records_dev;
} rt_render_opts;

typedef struct {
  uint64_t paths;          /* spectral (pixel, sample, band) estimates: paths traced x bands per path */
  uint64_t ext_rays;       /* closest-hit rays traced */
  uint64_t shadow_rays;    /* sun rays traced */
  uint64_t nodes_visited;  /* closest-hit BVH nodes, only with rt_set_counting(ctx, 1) */
  uint64_t tris_tested;    /* closest-hit triangles, only with rt_set_counting(ctx, 1) */
  uint64_t shadow_nodes_visited;  /* sun-ray BVH nodes, counting only */
  uint64_t shadow_tris_tested;    /* sun-ray triangles, counting only */
  uint32_t waves;
  uint32_t kernel_launches;
  float ms_render;         /* device time of the path tracing (events) */
  float ms_xyz;            /* device time of the XYZ contraction (events) */
  /* with rt_set_timing(ctx, 1): device time and launch count per stage:
   * 0 camera rays, 1 closest hit, 2 shading + NEE, 3 sun rays, 4 XYZ,
   * 5 guide sampling, 6 guide training */
  float ms_stage[7];
  uint32_t launches_stage[7];
} rt_stats;

/* Context on CUDA device `device`, enqueueing on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream). */
rt_status rt_create(int device, void* cuda_stream, rt_ctx** out);
void rt_destroy(rt_ctx* ctx);
const char* rt_last_error(const rt_ctx* ctx);
rt_status rt_set_stream(rt_ctx* ctx, void* cuda_stream);
/* 1: traversal kernels count nodes visited and triangles tested (slower). */
rt_status rt_set_counting(rt_ctx* ctx, int enable);
/* 1: every kernel launch of a render is bracketed by CUDA events on the
 * context's stream and the per-stage device times are returned in rt_stats. */
rt_status rt_set_timing(rt_ctx* ctx, int enable);

/* Diagnostic limits that make the error paths of a context reachable
 * without a device fault (0 = off, the default): ray queues that hold
 * queue_capacity rays, fewer than a wave's paths (the kernels detect the
 * overflow, drop what does not fit and the render returns
 * RT_ERR_QUEUE_OVERFLOW); traversal loops stopped after traversal_steps
 * steps per ray (RT_ERR_TIMEOUT); fail_cuda_call = n: the n-th CUDA runtime
 * call the context checks from now on is not made and reported as failed,
 * as a failing call would be (RT_ERR_CUDA, then RT_ERR_STATE for every later
 * call on the context).  The paper has no counterpart: a testing aid. */
rt_status rt_set_limits(rt_ctx* ctx, uint32_t queue_capacity, uint32_t traversal_steps, uint32_t fail_cuda_call);

/* Scene (the paper's first actor, section 1): n_verts float3 positions in
 * metres, n_tris uint32 index triples, a material id per triangle, and per
 * material its rt_material_type and thickness in metres (thin glass).
 * Builds the BVH with the builder rt_set_bvh_builder selected (default: binned
 * SAH with spatial splits on the host), copies it to the device; the library
 * owns its copy.  Replaces any previous scene. */
rt_status rt_load_scene(rt_ctx* ctx, const float* verts, uint32_t n_verts, const uint32_t* tris,
                        uint32_t n_tris, const uint32_t* mat_id, const int32_t* mat_type,
                        const float* mat_thickness, uint32_t n_mat);

/* BVH builder of the following rt_load_scene calls: 0 = binned SAH on the
 * host (also provides the binary tree of trace_variant 1-3),
 * 1 = linear BVH built on the device (Morton codes, radix sort, Karras
 * hierarchy, collapse to the four-wide tree; at most 2^24 triangles; only
 * trace_variant 0), 2 = binned SAH on the host with spatial splits (the
 * default; a triangle may be referenced by several leaves, about twice the
 * triangle count at most; thin-glass triangles never are; also provides the
 * binary tree).  The traversal results do not depend on the builder. */
rt_status rt_set_bvh_builder(rt_ctx* ctx, uint32_t builder);

typedef struct {
  uint32_t n_tris;    /* triangles of the loaded scene */
  uint32_t n_nodes4;  /* four-wide BVH nodes */
  uint32_t builder;   /* builder used: 0 host SAH, 1 device LBVH, 2 host SAH with spatial splits */
  float build_ms;     /* BVH build time: host wall clock, or device time (CUDA events) */
} rt_scene_info;
rt_status rt_get_scene_info(rt_ctx* ctx, rt_scene_info* info);

/* Spectral tables (section 3): n_bands wavelengths in nm; sun radiance per
 * band inside a cone of half angle sun_half_angle (radians) around the unit
 * direction sun_dir (towards the sun); per material and band the index n, the
 * extinction k (Eq. 1), the Lambertian reflectance rho and the emitted
 * radiance le ([n_mat][n_bands] each; le may be NULL = 0); cmf_w[n_bands][3]
 * the band weights of the XYZ contraction.  n_mat must match the scene.
 * Also stores the children of every four-wide BVH node far-to-near along
 * sun_dir, the order in which sun rays visit them (results do not depend on
 * it; the work per sun ray does).  Synchronous on the context's stream. */
rt_status rt_set_spectra(rt_ctx* ctx, const float* lambda_nm, uint32_t n_bands, const float* sun_L,
                         const float sun_dir[3], float sun_half_angle, const float* n, const float* k,
                         const float* rho, const float* le, const float* cmf_w);

/* Renders n_cams views (the observer, section 1) with spp samples per pixel,
 * bands [band_first, band_first + band_count) and at most `depth` surface
 * interactions per path; Philox key = seed.  Global pixel ids run over the
 * views in order.  Outputs (device, caller-owned, may be NULL):
 *   spectral_dev [sum_v W_v H_v][band_count] FP64: sum over samples of the
 *                path radiance (divide by spp for the mean);
 *   xyz_dev      [sum_v W_v H_v][3] float: CIE XYZ of the band range (the
 *                mean spectrum contracted with cmf_w), partial XYZ of
 *                disjoint band ranges add up to the full XYZ.
 * Synchronises the stream to read the device status word. */
rt_status rt_render(rt_ctx* ctx, const rt_camera* cams, uint32_t n_cams, uint32_t band_first,
                    uint32_t band_count, uint32_t spp, uint32_t depth, uint64_t seed,
                    const rt_render_opts* opts, double* spectral_dev, float* xyz_dev, rt_stats* stats);

/* Same as rt_render with HOST outputs: renders into library-owned device
 * buffers and copies xyz (and spectral, if non-NULL) to the given host
 * arrays before returning. */
rt_status rt_render_host(rt_ctx* ctx, const rt_camera* cams, uint32_t n_cams, uint32_t band_first,
                         uint32_t band_count, uint32_t spp, uint32_t depth, uint64_t seed,
                         const rt_render_opts* opts, double* spectral_host, float* xyz_host,
                         rt_stats* stats);

/* Photon mapping (section 4), the paper's own global-illumination method, as
 * a second estimator over the same scene and spectra.  First the photon
 * pass: for every band, n_photons photons leave a disk perpendicular to the
 * sun (tangent to the scene's bounding sphere, wide enough for the whole
 * cone) with directions uniform in the sun cone and flux
 * L_sun(lambda) cos Omega pi R_d^2 / n_photons, and follow the path tracer's
 * material rules for up to photon_depth surface interactions; every
 * Lambertian hit is stored, classed direct (only thin-glass transmissions
 * before it: next-event estimation covers it, so it is left out of the
 * maps), caustic (a reflection or refraction before the first diffuse hit:
 * caustic map) or indirect (after a diffuse hit: global map).  Then the
 * camera pass: camera paths follow thin-glass, conductor and solid-glass
 * events as in rt_render; at the first Lambertian vertex they add its
 * emission, the sun's next-event estimate and (rho / pi) E, E the kernel
 * density estimate of the irradiance over the photons of the path's band,
 *   E = sum over both maps of (2 / (pi r^2)) sum_{d < r} flux (1 - d^2 / r^2)
 * (Epanechnikov kernel; r = r_caustic, r_global), and stop.  The maps are spatial hash
 * grids (cells of edge 2 r, 2^log2_cells per map and band) built on the
 * device by a stable radix sort of the photon records; bands are processed
 * in chunks whose photon records fit one sort (n_photons x photon_depth x
 * chunk <= 2^24), with identical results for any chunking.  Philox: photons
 * key (seed_lo, seed_hi ^ 0x50484F54), counter (photon, band, 0,
 * 4 vertex + call); camera paths as rt_render.  Needs a sun half angle below
 * 1 rad.  Outputs as rt_render; rt_stats.ms_stage[0..2] hold the photon
 * pass, map build and camera pass times. */
typedef struct {
  uint32_t n_photons;     /* photons per band; 0 = 65536 */
  uint32_t photon_depth;  /* surface interactions per photon; 0 = 4 */
  float r_caustic;        /* caustic gather radius (m); 0 = 0.5% of the scene diagonal */
  float r_global;         /* indirect gather radius (m); 0 = 2% of the scene diagonal */
  uint32_t log2_cells;    /* hash cells per map and band, 8..20; 0 = 16 */
  uint32_t xyz_mode;      /* rt_xyz_mode */
  /* optional per-path records, as in rt_render_opts */
  const uint32_t* probe_map_dev;
  float* probe_L_dev;
  uint32_t* probe_sig_dev;
  uint32_t emission;      /* 0: the disk above; 1: portals -- photons start on the thin-glass triangles
                           * that face the sun, chosen by A |s . n|, uniform on the triangle, direction in
                           * the cone, flux L_sun |w . n| Omega W / (n_photons |s . n|) (W = sum A |s . n|),
                           * none where the way back to the sun is blocked.  For interiors lit through
                           * glass; sunlight that reaches the glass after an outside bounce is not
                           * emitted.  Needs a thin-glass triangle facing the sun (else RT_ERR_ARG) */
  uint32_t reserved[3];
} rt_photon_opts;
rt_status rt_render_photons(rt_ctx* ctx, const rt_camera* cams, uint32_t n_cams, uint32_t band_first,
                            uint32_t band_count, uint32_t spp, uint32_t depth, uint64_t seed,
                            const rt_photon_opts* opts, double* spectral_dev, float* xyz_dev, rt_stats* stats);
/* The photon pass alone, for checks: rec_dev [band_count][n_photons][depth]
 * float4 (device, 16-byte aligned) = {x, y, z, flux} of each photon's n-th
 * Lambertian hit, cls_dev (device, may be NULL) the class of each slot
 * (0 empty, 1 direct, 2 caustic, 3 indirect). */
rt_status rt_photon_records(rt_ctx* ctx, uint32_t band_first, uint32_t band_count, uint32_t n_photons,
                            uint32_t depth, uint64_t seed, uint32_t emission, float* rec_dev, uint8_t* cls_dev);

/* Same result as rt_render, for callers that may not allocate device memory
 * (a framework that has reserved the device memory for its own pool, a fixed
 * memory budget, or a loop that cannot take the implicit synchronisation of
 * cudaMalloc / cudaFree).  The paper has no counterpart: this is an interface
 * matter only.  The working memory (ray queues, hits, sun rays, per-path
 * radiance, counters, status, camera table) comes from one array compiled
 * into the library: 56 MiB (58,726,656 bytes), held by every GPU that loads
 * the library until the process exits; waves are at most 524,288 paths.
 * Limits: 1..64
 * cameras, depth 1..64, pixels x bands below 2^32 (RT_ERR_ARG otherwise).
 * spectral_dev (FP64 sums, [pixels][band_count]) is required; xyz_dev may be
 * NULL.  No cudaMalloc, cudaFree or other allocating call is made.  The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make it before any stream capture.  All calls share
 * the array: counters and status are cleared by each call, and calls whose
 * GPU work overlaps (other streams or contexts on the same device) race and
 * give wrong results.  Synchronises the context's stream. */
rt_status rt_render_static(rt_ctx* ctx, const rt_camera* cams, uint32_t n_cams, uint32_t band_first,
                           uint32_t band_count, uint32_t spp, uint32_t depth, uint64_t seed, uint32_t xyz_mode,
                           double* spectral_dev, float* xyz_dev);

/* ---- learned path guide (optional; a sampling density, not a change of the
 * estimator: guided directions are mixed with cosine sampling by one-sample
 * MIS, so the rendered expectation of section 4, Eq. 2 is unchanged) ------
 *
 * Network: hash-grid encoding of the position (8 levels x 4 features,
 * 2^log2_table entries per level, resolutions floor(n_min b^l), b =
 * (n_max / n_min)^(1/7), over the scene bounds), real spherical harmonics of the normal (degree <= 3), a one-hot
 * band group (9 groups); MLP 64 -> 64 -> 64 -> 64 -> 48 (ReLU, no biases) on
 * BF16 tensor cores with FP32 accumulation; 8 von Mises-Fisher lobes (outputs
 * 5j .. 5j + 4: logit, mean direction, kappa = 0.5 + softplus).
 * Parameters: grid [8][2^log2_table][4] and W = W1 [64][64] | W2 [64][64] |
 * W3 [64][64] | W4 [64][48] (row-major [in][out]), FP32 masters.
 * Training record (12 floats): {pos.xyz, weight}, {normal.xyz, band group},
 * {omega.xyz, 0}; loss -(1/N) sum_r (weight_r / mean weight) log q_r(omega_r).
 * In a guided render the direct sun at a guided vertex is estimated by two
 * strategies combined with the balance heuristic: next-event sampling of the
 * sun cone and the guided continuation escaping into the cone; both the
 * continuation (incident radiance of the path suffix) and the sun sample
 * (sun radiance x transmittance) become training records. */
typedef struct {
  uint32_t log2_table;   /* 10..22; 0 = 19 */
  float n_min, n_max;    /* 0 = 16, 2048 */
  float lr_grid, lr_mlp; /* Adam learning rates; 0 = 1e-2, 1e-3 */
  float beta1, beta2;    /* 0 = 0.9, 0.99 */
  float eps;             /* 0 = 1e-15 */
  float mis_alpha;       /* probability of sampling the guide at a guided vertex; 0 = 0.7 */
  uint32_t guide_depth;  /* vertices 1..guide_depth are guided; 0 = 2 */
  uint32_t reserved[6];
} rt_guide_config;

/* Creates (or re-creates) the guide of the loaded scene: parameters drawn
 * from Philox with the given seed (grid uniform +-1e-4, weights Xavier
 * uniform), Adam state zeroed.  The scene bounds fix the encoding. */
rt_status rt_guide_init(rt_ctx* ctx, const rt_guide_config* cfg, uint64_t seed);
/* Copies parameters in / out (host arrays of the sizes above; either pointer
 * may be NULL).  Setting parameters resets the Adam state. */
rt_status rt_guide_set_params(rt_ctx* ctx, const float* grid, const float* W);
rt_status rt_guide_get_params(rt_ctx* ctx, float* grid, float* W);
/* Network outputs Y_dev [n][48] and mixture density q_dev [n] at each
 * record's omega, for n records rec_dev [n][12] (device, 16-byte aligned). */
rt_status rt_guide_eval(rt_ctx* ctx, const float* rec_dev, uint64_t n, float* Y_dev, float* q_dev);
/* Loss and gradients without an update: *loss (host), dgrid_dev and dW_dev
 * (device, FP32, sizes as the parameters; either may be NULL). */
rt_status rt_guide_grad(rt_ctx* ctx, const float* rec_dev, uint64_t n, float* loss, float* dgrid_dev, float* dW_dev);
/* One Adam step on a batch of records; *loss (host, may be NULL) before the step. */
rt_status rt_guide_train_step(rt_ctx* ctx, const float* rec_dev, uint64_t n, float* loss);

/* One guided sampling step (the one-sample MIS of the guide and cosine
 * sampling that estimates section 4, Eq. 2 at a Lambertian vertex, with the
 * sun of Eq. 3 weighted by the balance heuristic) on caller-given vertices,
 * run by the renderer's own guide kernel, for checks of the sampler.  Vertex
 * i (of n, a multiple of band_count) is vertex k (1..62) of the path of
 * pixel i / band_count, band band_first + i % band_count, sample `sample`,
 * Philox key seed: the counters (pixel, sample, band, 4k) and (.., 4k + 1)
 * of rt_render draw its continuation.  The guide must be initialised
 * (rt_guide_init; mis_alpha of its configuration) and spectra set.
 * v_dev [n] and out_dev [n] are device arrays (16-byte aligned, caller-owned);
 * the call allocates and frees its own temporaries and synchronises. */
typedef struct {
  float pos[3];       /* query position (the vertex offset along its normal) */
  float throughput;   /* path throughput before the vertex */
  float normal[3];    /* unit normal on the incoming side */
  float rho;          /* Lambertian reflectance of the path's band */
  float sun_dir[3];   /* direction of the vertex's pending sun sample (unit) */
  float sun_contrib;  /* its next-event contribution before MIS weighting */
  uint32_t has_sun;   /* 1 = a sun sample is pending (its cosine is positive) */
  uint32_t reserved[3];
} rt_guide_vertex;
typedef struct {
  float omega[3];     /* continuation direction (guide or cosine draw) */
  float pdf;          /* p_mix(omega) = alpha q(omega) + (1 - alpha) max(cos, 0) / pi */
  float cos_theta;    /* normal . omega */
  float throughput;   /* throughput rho cos / (pi p_mix) x before, when continued; else 0 */
  float nee_contrib;  /* sun_contrib x p_cone / (p_cone + p_mix(sun_dir)); 0 without sun sample */
  float esc_weight;   /* p_mix / (p_mix + p_cone) when omega lies in the sun cone and the path
                         continues, else 0 */
  uint32_t continued; /* 1 = the path continues along omega (cos > 0 and p_mix > 0) */
  uint32_t reserved[3];
} rt_guide_step_out;
rt_status rt_guide_sample_step(rt_ctx* ctx, const rt_guide_vertex* v_dev, uint32_t n, uint32_t k, uint32_t sample,
                               uint32_t band_first, uint32_t band_count, uint64_t seed, rt_guide_step_out* out_dev);

/* ---- single steps of the path, for parity tests and tools ---------------- */

/* Philox4x32-10 (Salmon et al., SC 2011) of n counters ctr_dev[n][4] with key
 * (key0, key1) into out_dev[n][4]. */
rt_status rt_philox(rt_ctx* ctx, const uint32_t* ctr_dev, uint32_t* out_dev, uint64_t n, uint32_t key0,
                    uint32_t key1);

/* Closest hit (t > 0) of n rays (o_dev, d_dev: [n][3] float) against the
 * loaded scene: t_dev[n] (or -1) and prim_dev[n] (input triangle id or -1). */
rt_status rt_trace_closest(rt_ctx* ctx, const float* o_dev, const float* d_dev, uint64_t n, float* t_dev,
                           int32_t* prim_dev);

/* Sun-ray transmittance of n rays to infinity: 0 if an opaque triangle is
 * crossed, else the product of the thin-glass T_s (band band_dev[i]) of all
 * crossed sheets; n_glass_dev[i] = sheets crossed or 0xFFFFFFFF if blocked. */
rt_status rt_trace_shadow(rt_ctx* ctx, const float* o_dev, const float* d_dev, const uint32_t* band_dev,
                          uint64_t n, float* T_dev, uint32_t* n_glass_dev);

/* Complex Fresnel reflectance R(cos_i, n, k) from air (Eq. 1 index) and the
 * thin-sheet R_s, T_s for n inputs; lambda_nm_dev and d_dev may be NULL for
 * rt_fresnel (then Rs/Ts outputs are not written). */
rt_status rt_optics_eval(rt_ctx* ctx, const float* cos_dev, const float* n_dev, const float* k_dev,
                         const float* lambda_nm_dev, const float* d_dev, uint64_t count, float* R_dev,
                         float* Rs_dev, float* Ts_dev);

/* XYZ contraction of an FP64 spectral-sum image: xyz[p][c] = sum_j
 * (spectral[p][j] / spp) * cmf_w[band_first + j][c], with mode rt_xyz_mode. */
rt_status rt_xyz(rt_ctx* ctx, const double* spectral_dev, uint64_t n_pixels, uint32_t band_first,
                 uint32_t band_count, uint32_t spp, uint32_t mode, float* xyz_dev);

/* Autotuner: times probe renders (spp_probe samples of the given views and
 * bands, depth `depth`, results discarded) over the wave capacity, the
 * leaf batch, the traversal loop parameters and the traversal block size (coordinate
 * descent, device time from CUDA events, one warm-up render per setting) and
 * writes the fastest setting into opts (other fields are kept). */
typedef struct {
  uint32_t trials;   /* settings timed */
  float best_ms;     /* device time of the probe render with the chosen setting */
  float default_ms;  /* ... with the setting passed in */
} rt_autotune_report;
rt_status rt_autotune(rt_ctx* ctx, const rt_camera* cams, uint32_t n_cams, uint32_t band_first, uint32_t band_count,
                      uint32_t spp_probe, uint32_t depth, rt_render_opts* opts, rt_autotune_report* report);

/* Measurement tool: read bandwidth of the L2 cache.  Streams `bytes`
 * (rounded down to 16; at most 96 MiB so that it stays L2-resident) `iters`
 * times with 16-byte loads from a library-owned buffer and returns GB/s
 * (bytes * iters / kernel time from CUDA events) in *gbs. */
rt_status rt_probe_l2(rt_ctx* ctx, uint64_t bytes, uint32_t iters, float* gbs);

#ifdef __cplusplus
}
#endif

#endif /* SPECTRAL_RT_H */

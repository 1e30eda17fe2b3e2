/*
 * rt3dg.h -- C ABI of the GB300 (sm_103a) point-based Gaussian ray tracer.
 *
 * The library precomputes per-Gaussian visibility: for rays cast from each 3D
 * Gaussian in a set of directions it returns the transmittance
 * T = prod_j (1 - alpha_j) over the Gaussians the ray passes (Sec. 4.1-4.2 of
 * "Relightable 3D Gaussians", arXiv 2311.16043).  Gaussians are given as mean,
 * scale, rotation quaternion and opacity (Sec. 3.1); rays as origin and
 * direction (Eq. 13); visibility is returned per ray.
 *
 * Conventions for every entry point
 *   - Array arguments are DEVICE pointers owned by the caller unless a comment
 *     says "host".  float32 arrays are C-contiguous, row-major.
 *   - Gaussians: mean[n*3], scale[n*3] (linear standard deviations along the
 *     local axes), quat[n*4] as (w, x, y, z) (normalised internally; must be
 *     non-zero), opacity[n] in [0, 1).  Sigma = R(q) diag(s)^2 R(q)^T.
 *   - All work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and is asynchronous; calls do not synchronise the host unless a
 *     comment says so.
 *   - Calls return rt_status.  Argument errors are detected on the host and
 *     returned before anything is enqueued.  Errors found by kernels
 *     (RT_ERR_STACK_OVERFLOW, RT_ERR_TIMEOUT) set a sticky device status word
 *     read by rt_status_last() after the caller synchronises the stream.
 *     No entry point aborts, asserts or traps.
 *   - Handles (rt_bvh, rt_envmap, rt_surrogate, rt_batch) own their device
 *     memory (stream-ordered cudaMallocAsync) and keep no pointer to caller
 *     arrays after the call that created them returns.
 */
#ifndef RT3DG_H
#define RT3DG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *rt_stream_t; /* identical to cudaStream_t */

typedef enum {
    RT_OK = 0,
    RT_ERR_INVALID_ARG = 1,     /* bad pointer, size, or parameter         */
    RT_ERR_OOM = 2,             /* device allocation failed                */
    RT_ERR_CUDA = 3,            /* a CUDA runtime call failed              */
    RT_ERR_STACK_OVERFLOW = 4,  /* traversal stack exceeded (never for trees built here) */
    RT_ERR_HITLOG_OVERFLOW = 5, /* informational: some ray logged more hits than capacity */
    RT_ERR_TIMEOUT = 6,         /* a bounded device wait gave up           */
    RT_ERR_NOT_TRAINED = 7,     /* surrogate used before training          */
    RT_ERR_UNSUPPORTED = 8,     /* option combination not supported        */
    RT_ERR_RANGE = 9            /* a value outside a fixed-point range (NaN included) */
} rt_status;

/* Tracing parameters.  Defaults (rt_params_default):
 *   k_sigma = 3       support of a Gaussian: accepted only if the peak's
 *                     Mahalanobis distance m satisfies m^2 <= k_sigma^2;
 *   alpha_min = 1/255 accepted only if alpha = o * exp(-m^2/2) >= alpha_min;
 *   t_min = 1e-4      early termination (Sec. 4.1): a ray whose running T
 *                     drops below t_min stops and reports T = 0 (0 disables);
 *   origin_eps = 1e-4 rays cast from a Gaussian start at
 *                     fl(mu + fl(origin_eps * d)) and skip that Gaussian;
 *   box_mode = 0      leaf boxes of radius k_sigma; 1 = opacity-aware radius
 *                     min(k_sigma, sqrt(2 ln(o / alpha_min))), which gives the
 *                     same accepted set with tighter boxes;
 *   deterministic = 0 the adjoint accumulates with float32 atomics (order
 *                     depends on scheduling); 1 = in 64-bit fixed point
 *                     (resolution 2^-32, |sum| < 2^31 per component, else
 *                     RT_ERR_RANGE in the status word), so gradients are
 *                     bit-reproducible whatever the order of rays.  The
 *                     forward is reproducible for a given strategy either
 *                     way.                                                   */
typedef struct {
    float k_sigma;
    float alpha_min;
    float t_min;
    float origin_eps;
    int32_t box_mode;
    int32_t deterministic;
} rt_params;

void rt_params_default(rt_params *p);
const char *rt_status_string(rt_status s);
/* Sticky device status word (RT_OK if no kernel reported an error).  Reads a
 * device value synchronously: call after synchronising the work in question.
 * rt_status_clear() resets it. */
rt_status rt_status_last(void);
rt_status rt_status_clear(void);
/* Exercises the failure path of the kernels' bounded waits: one thread waits
 * on an mbarrier that nothing completes, gives up after max_cycles SM cycles
 * (1 .. 4e9), records RT_ERR_TIMEOUT in the status word and returns.  No
 * fault, no hang; for tests of failure handling. */
rt_status rt_selftest_wait_timeout(int64_t max_cycles, rt_stream_t stream);
/* Upper bound, in SM clock cycles, of the bounded waits of the surrogate
 * kernels (their mbarrier waits on their own tensor-core MMAs), process-wide;
 * 0 restores the default of 4e9 (~2 s at 2 GHz).  A wait that gives up
 * records RT_ERR_TIMEOUT; the whole warpgroup (inference) or CTA (training)
 * then waits, with the default bound, for the MMAs it has in flight, frees
 * its tensor memory and returns.  A tiny bound makes the waits give up on
 * purpose, for tests of that exit path.  RT_ERR_INVALID_ARG outside
 * [0, 4e9]. */
rt_status rt_set_wait_limit(int64_t max_cycles);

/* ------------------------------------------------------------------------ */
/* LBVH (Sec. 4.1: binary radix tree of Karras 2012 over the Gaussians)      */
/* ------------------------------------------------------------------------ */

typedef struct rt_bvh rt_bvh;

/* Builds the tree: per-Gaussian whitening S^-1 R^T and leaf boxes, scene
 * bounds of the means, 30-bit Morton codes, a device LSD radix sort of
 * (code, index), Karras' split rule over keys code<<32 | index, and a
 * bottom-up refit of the child boxes.  n = 0 and n = 1 are valid.
 * Synchronises `stream` once (to read the scene bounds into the handle).
 * Errors: RT_ERR_INVALID_ARG (n < 0, n >= 2^31, NULL arrays with n > 0,
 * k_sigma <= 0, alpha_min outside (0,1), t_min outside [0,1), or Gaussian
 * inputs failing the device check: a non-finite value, a scale <= 0, a zero
 * quaternion, an opacity outside [0,1]), RT_ERR_OOM. */
rt_status rt_build_bvh(const float *mean, const float *scale, const float *quat,
                       const float *opacity, int64_t n, const rt_params *params,
                       rt_stream_t stream, rt_bvh **out);
rt_status rt_bvh_destroy(rt_bvh *bvh, rt_stream_t stream);
/* Refit-only rebuild: the same n Gaussians (same order) with new mean, scale,
 * quat and opacity keep the tree's topology (Morton order, binary and 4-wide
 * structure); the Gaussian records, leaf boxes and every internal box are
 * recomputed bottom-up (Sec. 4.1's refit step alone).  For geometry that
 * moves during optimisation; traversal stays exact for any input (boxes
 * always contain the supports), it only loses efficiency as the Morton order
 * goes stale.  The scene bounds reported by rt_bvh_info stay those of the
 * build.  Asynchronous on `stream` (the first call also derives the 4-wide
 * tree's parent links once).  Refitting with the build's inputs reproduces
 * the built tree bit for bit.  Errors: RT_ERR_INVALID_ARG (inputs failing the
 * check of rt_build_bvh are reported through the status word, since the call
 * does not synchronise). */
rt_status rt_bvh_refit(rt_bvh *bvh, const float *mean, const float *scale, const float *quat,
                       const float *opacity, rt_stream_t stream);
/* Host outputs (any may be NULL): Gaussian count, scene bounds of the means
 * (float[3] each), device bytes held by the handle. */
rt_status rt_bvh_info(const rt_bvh *bvh, int64_t *n, float *lo, float *hi, int64_t *device_bytes);
/* Copies the tree out (device pointers, any may be NULL):
 *   keys[n]            sorted keys code<<32 | original index;
 *   left[n-1], right[n-1]  child refs of internal node i; bit 31 set = leaf
 *                      (sorted position in the low bits);
 *   parent[2n-1]       parents of internal nodes 0..n-2 then of leaves;
 *   boxes[(n-1)*12]    per internal node: left child box (lo xyz, hi xyz),
 *                      then right child box (lo xyz, hi xyz).              */
rt_status rt_bvh_export(const rt_bvh *bvh, uint64_t *keys, int32_t *left, int32_t *right,
                        int32_t *parent, float *boxes, rt_stream_t stream);

/* Caller's device allocator (the paper has no counterpart).  alloc returns
 * `bytes` of device memory usable in stream order on `stream` (NULL on
 * failure; the block must be 256-byte aligned), free releases a block in
 * stream order.  With an allocator set, every device allocation the library
 * makes — handles' buffers and per-call scratch — goes through it (e.g. a
 * framework's caching allocator); NULL restores the default: the library's
 * own stream-ordered pool on the call's device (cudaMallocFromPoolAsync /
 * cudaFreeAsync on the call's stream), which keeps freed blocks mapped for
 * reuse until rt_memory_trim.  Process-wide: set it while no
 * handle exists, since a handle returns its buffers through the allocator in
 * force when it is destroyed.  rt_surrogate_infer_noalloc allocates nothing
 * either way.  Errors: RT_ERR_INVALID_ARG (alloc or free missing). */
typedef struct {
    void *(*alloc)(size_t bytes, rt_stream_t stream, void *ctx);
    void (*free)(void *ptr, rt_stream_t stream, void *ctx);
    void *ctx;
} rt_allocator;
rt_status rt_set_allocator(const rt_allocator *a);
/* Returns the library pool's unused blocks to the CUDA driver on every device,
 * keeping at most keep_bytes reserved per device (0 = all).  Call after
 * synchronising the streams that freed them.  Errors: RT_ERR_INVALID_ARG
 * (keep_bytes < 0), RT_ERR_CUDA. */
rt_status rt_memory_trim(int64_t keep_bytes);

/* ------------------------------------------------------------------------ */
/* Ray sets                                                                   */
/* ------------------------------------------------------------------------ */

typedef struct rt_envmap rt_envmap;

/* Environment map for importance-sampled shadow rays (the direct light of
 * Eq. 8).  Host inputs: radiance[h*w] and solid_angle[h*w] (float64,
 * row-major, row 0 = polar angle 0) and corners[(h+1)*(w+1)*3] (float32 unit
 * directions of the pixel corners).  Pixel (i,j) is drawn with probability
 * radiance*solid_angle / total (cumulative sums in float64, index order);
 * inside it the direction is the normalised bilinear blend of its corners. */
rt_status rt_envmap_create(const double *radiance, const double *solid_angle,
                           const float *corners, int32_t h, int32_t w, rt_stream_t stream,
                           rt_envmap **out);
rt_status rt_envmap_destroy(rt_envmap *env, rt_stream_t stream);

typedef enum {
    RT_RAYS_EXPLICIT = 0, /* ray_o[R*3], ray_d[R*3], ray_src[R] (or NULL)       */
    RT_RAYS_DIRS = 1,     /* from every Gaussian g along dirs[k]: id g*K + k     */
    RT_RAYS_ENV = 2,      /* from every Gaussian g, S env samples: id g*S + s    */
    RT_RAYS_HEMI = 3      /* from every Gaussian g over the hemisphere of its
                             normal: local dirs[k] in g's frame, id g*K + k      */
} rt_ray_kind;

/* A ray set.  EXPLICIT: n_rays rays, ray_src[r] = original index of a
 * Gaussian the ray skips (or -1; NULL = none).  DIRS: K = n_dirs directions
 * dirs[K*3] (device, unit length); the ray id r = g*K + k starts at
 * fl(mu_g + fl(origin_eps * d_k)) and skips g.  ENV: S = n_dirs samples per
 * Gaussian; sample s of Gaussian g (ray id r = g*S + s) draws Philox4x64-10
 * with counter (r,0,0,0) and key (seed,0): u0 = (x0>>11) 2^-53 picks the
 * pixel, a = (x1>>40) 2^-24 and b = (x2>>40) 2^-24 blend its corners.
 * HEMI (Sec. 3.3: N_s incident directions per Gaussian over the hemisphere
 * of its normal, Fibonacci sampling; Sec. 4.2 precomputes their visibility):
 * K = n_dirs local directions dirs[K*3] with z along the normal (device,
 * unit, z > 0) and normals[n*3] (device, original Gaussian order, non-zero).
 * Ray r = g*K + k has direction d = (h_x t1 + h_y t2) + h_z n for h = dirs[k]
 * in the frame (t1, t2, n) of g's normal normalised in float32, built by the
 * branchless construction of Duff et al. 2017 (rt_materialize_rays gives the
 * exact float32 rays), origin and exclusion as for DIRS.
 * If ray_ids (device int64[n_ids]) is set for DIRS/ENV/HEMI, only those ray
 * ids are traced and outputs are indexed by position in ray_ids (a non-NULL
 * ray_ids with n_ids = 0 is the empty subset; NULL means every ray). */
typedef struct {
    int32_t kind;
    int32_t n_dirs;
    int64_t n_rays;
    const float *ray_o;
    const float *ray_d;
    const int32_t *ray_src;
    const float *dirs;
    const rt_envmap *env;
    uint64_t seed;
    const int64_t *ray_ids;
    int64_t n_ids;
    const float *normals; /* HEMI only */
} rt_rayspec;

/* Number of rays of a ray set over `bvh` (n*K for DIRS, n*S for ENV, n_ids if
 * ray_ids is set, n_rays for EXPLICIT); -1 if the set is invalid. */
int64_t rt_rayspec_count(const rt_bvh *bvh, const rt_rayspec *rays);

/* Materialises rays of an implicit set (device outputs o[m*3], d[m*3],
 * src[m], original index of the source Gaussian) for the listed ray ids. */
rt_status rt_materialize_rays(const rt_bvh *bvh, const rt_rayspec *rays, const int64_t *ray_ids,
                              int64_t m, float *ray_o, float *ray_d, int32_t *ray_src,
                              rt_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Visibility (Eq. 13-15)                                                    */
/* ------------------------------------------------------------------------ */

typedef enum {
    RT_KERNEL_AUTO = 0,   /* DIRS sets: RAY_WIDE up to 2^19 Gaussians, WIDE
                             beyond; ENV and HEMI sets: RAY_REFILL; explicit
                             rays and id lists: WARP_RAY up to 2^22 rays
                             (RAY_WIDE with a hit log), RAY_WIDE beyond (an id
                             list traced in the tree's order); the binary
                             forms when there is no 4-wide tree              */
    RT_KERNEL_RAY = 1,    /* one thread per ray, private stack, binary tree    */
    RT_KERNEL_PACKET = 2, /* one warp per 32 rays of neighbouring Gaussians in
                             one direction, shared stack, binary tree          */
    RT_KERNEL_WIDE = 3,   /* as PACKET over the 4-wide tree (the binary tree
                             collapsed by greedy largest-area expansion)       */
    RT_KERNEL_RAY_WIDE = 4, /* one thread per ray over the 4-wide tree        */
    RT_KERNEL_RAY_REFILL = 5, /* as RAY_WIDE, idle lanes refilled with new rays
                              as theirs finish (full implicit sets; otherwise
                              RAY_WIDE)                                       */
    RT_KERNEL_WARP_RAY = 6   /* one warp per ray over the 4-wide tree: the lanes
                              expand up to 32 of the ray's nodes at once (few
                              or latency-bound rays; no hit log)             */
} rt_kernel;

typedef struct {
    int32_t kernel;      /* rt_kernel                                          */
    int32_t order_block; /* PACKET: tiles of 32 Gaussians per direction sweep
                            (0 = default, 1: a tile's directions in turn)      */
    int32_t block_threads; /* threads per block (0 = default)                  */
    int32_t hit_cap;     /* capacity per ray of hit_ids                        */
    int64_t *counters;   /* device int64[4] accumulated (not reset): box tests,
                            Gaussian tests, accepted hits, rays (NULL = off)   */
    int32_t *hit_ids;    /* device [R*hit_cap]: original indices of accepted
                            Gaussians per ray, in traversal order (NULL = off) */
    int32_t *hit_count;  /* device [R]: accepted hits per ray (may exceed
                            hit_cap: the log of that ray is then incomplete)   */
} rt_trace_opts;

/* T_out[R] (device float32): visibility of every ray of the set, in ray-id
 * order (DIRS: an [n, K] row-major table in the caller's Gaussian order).
 * Accept rule per Gaussian j != source: t* > 0, m^2 <= k_sigma^2,
 * alpha >= alpha_min, where t* minimises the Mahalanobis distance along the
 * ray (Eq. 14 with Sigma^-1) and m^2 is its value; T is snapped to 0 below
 * t_min.  opts may be NULL.  Errors: RT_ERR_INVALID_ARG. */
rt_status rt_trace_visibility(const rt_bvh *bvh, const rt_rayspec *rays, float *T_out,
                              const rt_trace_opts *opts, rt_stream_t stream);

/* Convenience form of rt_trace_visibility for RT_RAYS_DIRS over all
 * Gaussians: T_out[n*k]. */
rt_status rt_trace_visibility_dirs(const rt_bvh *bvh, const float *dirs, int32_t k, float *T_out,
                                   const rt_trace_opts *opts, rt_stream_t stream);

/* The whole visibility precompute from host memory in one call (Sec. 4.2:
 * every Gaussian's visibility along the K directions): copies mean[n*3],
 * scale[n*3], quat[n*4], opacity[n] and dirs[k*3] (host float32, the layouts
 * of rt_build_bvh and rt_trace_visibility_dirs) to the device, builds the
 * tree, traces the n*k rays into a device table and copies it to
 * T_host[n*k] (row-major [n, k], caller's Gaussian order).  Device buffers
 * come from the library's allocator (rt_set_allocator) and are released in
 * stream order.  Host buffers should be page-locked for the copies to run
 * asynchronously (pageable memory is staged by CUDA).  Synchronises `stream`
 * once, inside the build; T_host holds the result once `stream` has been
 * synchronised.  n = 0 or k = 0 writes nothing.  Errors: those of
 * rt_build_bvh and rt_trace_visibility_dirs; RT_ERR_INVALID_ARG (NULL arrays
 * with n*k > 0, k < 0, n*k >= 2^40), RT_ERR_OOM, RT_ERR_CUDA (a copy could
 * not be enqueued). */
rt_status rt_visibility_dirs_host(const float *mean, const float *scale, const float *quat,
                                  const float *opacity, int64_t n, const float *dirs, int32_t k,
                                  const rt_params *params, const rt_trace_opts *opts, float *T_host,
                                  rt_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Composed scenes: a two-level BVH over object instances (Sec. 4.3)         */
/* ------------------------------------------------------------------------ */

/* Sec. 4.3 composes reconstructed objects into a new scene and re-traces the
 * visibility so that objects shadow each other.  An instance places an
 * object's tree (built in the object's local frame, kept and shared) in the
 * world by a rigid map: world = R local + t with xform = [R | t] row-major
 * 3x4 (host floats; R orthonormal).  Instances may share a tree; all trees
 * must have equal rt_params. */
typedef struct {
    const rt_bvh *bvh;
    float xform[12];
} rt_instance;

typedef struct rt_scene rt_scene;

/* Builds the top-level tree over the instances' world boxes (host, median
 * splits; synchronises `stream` to read each object's root box).  The scene
 * keeps pointers to the trees: they must outlive it.  Errors:
 * RT_ERR_INVALID_ARG (no instances, differing params, non-finite xform),
 * RT_ERR_UNSUPPORTED (a tree without its 4-wide form). */
rt_status rt_scene_create(const rt_instance *inst, int32_t n_inst, rt_stream_t stream, rt_scene **out);
/* New transforms for the same instances (same trees, same order): only the
 * top level is rebuilt; objects refitted since are re-read.  Synchronous. */
rt_status rt_scene_update(rt_scene *scene, const rt_instance *inst, int32_t n_inst, rt_stream_t stream);
/* Total Gaussians (sum over instances) and instance count. */
rt_status rt_scene_info(const rt_scene *scene, int64_t *n_total, int32_t *n_inst);
/* Visibility of the composed scene along K directions dirs[K*3] (device)
 * from every Gaussian of every instance: T_out[(g_base_j + g)*K + k] for
 * Gaussian g (original index) of instance j, g_base_j = Gaussians of the
 * instances before j.  The ray starts at the Gaussian's world mean
 * m = fl(((R_c0 mu_x + R_c1 mu_y) + R_c2 mu_z) + t_c) (each operation
 * rounded), at fl(m + fl(origin_eps d)); it meets instance i's Gaussians
 * in i's frame, o_i = fl(R_i^T fl(o - t_i)) and d_i = fl(R_i^T d) with
 * component c = ((R_0c v_0 + R_1c v_1) + R_2c v_2), under Eq. 13-15 and the
 * params of the trees; its own Gaussian is skipped; T is one product over all
 * instances, snapped to 0 below t_min.  One thread per ray over the 4-wide
 * trees.  Errors: RT_ERR_INVALID_ARG. */
rt_status rt_scene_trace_dirs(const rt_scene *scene, const float *dirs, int32_t K, float *T_out,
                              rt_stream_t stream);
/* The same for any implicit ray set over the scene's rows (row = g_base_j +
 * g as above, n_total rows): DIRS (as rt_scene_trace_dirs), HEMI (Sec. 3.3:
 * the local hemisphere directions rays->dirs[K] about the world-frame normal
 * of each row, rays->normals[n_total*3], device; Sec. 4.3 relighting of a
 * composed scene re-traces these) or ENV (env-map samples, rays->env and
 * rays->seed; the sample of row r, index s is keyed by the ray id r*S + s).
 * The direction is in the world frame; the origin and the rest as above.
 * T_out[row*K + k].  Errors: RT_ERR_INVALID_ARG, RT_ERR_UNSUPPORTED
 * (explicit rays or ray_ids). */
rt_status rt_scene_trace(const rt_scene *scene, const rt_rayspec *rays, float *T_out, rt_stream_t stream);
rt_status rt_scene_destroy(rt_scene *scene, rt_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Consumers of the visibility: per-Gaussian PBR colour (Eq. 8-10) and        */
/* ambient occlusion                                                          */
/* ------------------------------------------------------------------------ */

/* Material and light of the PBR colour of Sec. 3.3 (all device arrays in the
 * original Gaussian order unless stated):
 *   albedo[n*3] in [0,1]; roughness[n] (clamped to [0.04, 1]);
 *   sh[n*27] = coefficient j (0..8, real SH of degree 0..2) of colour channel
 *     c at sh[(g*9 + j)*3 + c]: the per-Gaussian indirect light, clamped at 0
 *     (NULL = no indirect light);
 *   env[env_h*env_w*3] = the global RGB direct light, equirectangular, row i
 *     over polar angles [i pi/h, (i+1) pi/h] from +z, column j over azimuths
 *     [2 pi j/w, 2 pi (j+1)/w], looked up bilinearly between pixel centres
 *     (azimuth wraps, polar angle clamps); env_h*env_w <= 8192;
 *   cam = camera centre, host floats: wo = (cam - mu)/|cam - mu|.           */
typedef struct {
    const float *albedo;
    const float *roughness;
    const float *sh;
    const float *env;
    int32_t env_h, env_w;
    float cam[3];
    int32_t kernel; /* fused form: RT_KERNEL_AUTO, RT_KERNEL_WIDE (warp packet)
                       or RT_KERNEL_RAY_WIDE (one thread per ray)           */
} rt_pbr_inputs;

/* Per-Gaussian PBR colour, Eq. 10, over the hemisphere ray set `rays`
 * (RT_RAYS_HEMI, no ray_ids):
 *   rgb[g*3+c] = sum_k (b_c/pi + f_s(wo, wi_k)) L_c(wi_k) max(n.wi_k, 0) 2pi/K,
 *   L_c(wi) = V[g*K+k] L_direct,c(wi) + max(0, sum_j sh[g][j][c] Y_j(wi))
 * with the simplified Disney BRDF of Eq. 9: f_s = D F G / (4 (n.wi)(n.wo)),
 * GGX D with alpha = r^2, Schlick F with F0 = 0.04, Smith-Schlick G with
 * k = (r+1)^2/8, normalised half vector, n.wi and n.wo clamped at 0.
 * V[n*K] (device, the visibility of the rays as rt_trace_visibility writes
 * it) or NULL: then the rays are traced in the same kernel and V is never
 * written (one warp per 32 Morton-adjacent Gaussians, all K rays each).
 * rgb[n*3] device output.  Errors: RT_ERR_INVALID_ARG (wrong ray kind,
 * missing arrays, map too large). */
rt_status rt_pbr_shade(const rt_bvh *bvh, const rt_rayspec *rays, const float *V, const rt_pbr_inputs *in,
                       float *rgb, rt_stream_t stream);

/* Ambient occlusion: ao[g] = (sum_k T(g, k)) / K, the mean visibility of
 * Gaussian g over a full DIRS or HEMI ray set (no ray_ids), traced and
 * reduced in one kernel without writing T (device output ao[n], original
 * order; the sum runs over k in order, in float32).  opts: only `kernel` is
 * read (RT_KERNEL_AUTO, RT_KERNEL_WIDE or RT_KERNEL_RAY_WIDE; NULL = AUTO).
 * Errors: RT_ERR_INVALID_ARG. */
rt_status rt_trace_ao(const rt_bvh *bvh, const rt_rayspec *rays, const rt_trace_opts *opts, float *ao,
                      rt_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Adjoint                                                                    */
/* ------------------------------------------------------------------------ */

/* Gradient of L = sum_r dL_dT[r] * T[r] for the ray set (T as traced with the
 * same params; rays snapped to 0 contribute nothing).  Accumulates (+=) into
 * d_mean[n*3], d_scale[n*3], d_quat[n*4] (with respect to the un-normalised
 * quaternion), d_opacity[n] (caller-zeroed, original Gaussian order) and, if
 * not NULL, writes d_ray_o[R*3].  T[R] are the traced values.  With
 * hit_ids/hit_count from the forward (capacity hit_cap) the accepted hits are
 * replayed; rays whose count exceeds hit_cap, or all rays if hit_ids is NULL,
 * are re-traversed.  The mean, scale, quat, opacity arrays must be the ones
 * the BVH was built from.  Accumulation uses float32 atomics (summation order
 * is not deterministic) unless the tree's params.deterministic is set: then
 * 64-bit fixed-point sums (device scratch of 88 bytes per Gaussian) are added
 * to the outputs once, bit-reproducibly. */
rt_status rt_trace_visibility_backward(const rt_bvh *bvh, const rt_rayspec *rays,
                                       const float *mean, const float *scale, const float *quat,
                                       const float *opacity, const float *T, const float *dL_dT,
                                       const int32_t *hit_ids, const int32_t *hit_count,
                                       int32_t hit_cap, float *d_mean, float *d_scale,
                                       float *d_quat, float *d_opacity, float *d_ray_o,
                                       rt_stream_t stream);


/* ------------------------------------------------------------------------ */
/* Learned visibility surrogate (not in the paper)                            */
/* ------------------------------------------------------------------------ */
/*
 * A small MLP predicts T from a ray's origin and direction; rays whose
 * prediction is uncertain fall back to the tracer.  The paper precomputes
 * visibility by tracing only (Sec. 4.2); this is an addition.
 *
 * Network: six scalars (origin normalised to [-1,1] by the scene bounds
 * lo/hi, p_n = 2 (p - lo)/(hi - lo) - 1, then the direction), each expanded
 * to [x, sin(2^k pi x), cos(2^k pi x), k = 0..5] -> 78 features + 2 zeros =
 * 80 inputs; four hidden layers of 128 with ReLU; one sigmoid output.
 * Weights and activations are bf16 on the tensor cores with float32
 * accumulation; biases, the output layer and the master copy of all weights
 * are float32.  Loss: mean binary cross-entropy against soft targets T with
 * a weight w (cfg.pos_weight) on the lit term,
 *   L = -mean( w T log p + (1 - T) log(1 - p) ),
 * optimiser: Adam.  The minimiser of the weighted loss for rays with mean
 * visibility T is p = w T / (w T + 1 - T), so a ray region that is lit only
 * now and then (small mean T) gets a p well inside the fallback band and is
 * traced instead of being predicted as a small constant; the visibility
 * estimate is recovered as T = p / (p + w (1 - p)) = sigmoid(z - ln w), z
 * the logit.  w = 1 is the plain loss (T = p).
 *
 * Parameter block (float32, rt_surrogate_param_count() = 60033 values):
 *   W1[128][80], b1[128], W2[128][128], b2[128], W3[128][128], b3[128],
 *   W4[128][128], b4[128], w5[128], b5.
 */
typedef struct rt_surrogate rt_surrogate;

typedef struct {
    float lr;      /* Adam step size (1e-3)                       */
    float beta1;   /* 0.9                                         */
    float beta2;   /* 0.999                                       */
    float eps;     /* 1e-8                                        */
    int32_t batch; /* samples per training step (262144)          */
    float pos_weight; /* w > 0, weight of the lit term of the loss (1) */
} rt_mlp_cfg;

void rt_mlp_cfg_default(rt_mlp_cfg *cfg);
int64_t rt_surrogate_param_count(void);

/* Creates a surrogate with He-uniform weights drawn from Philox4x64-10 keyed
 * by `seed` (zero biases), Adam state zeroed, scene bounds (-1,-1,-1)..(1,1,1).
 * Synchronises `stream`. */
rt_status rt_surrogate_create(const rt_mlp_cfg *cfg, uint64_t seed, rt_stream_t stream,
                              rt_surrogate **out);
rt_status rt_surrogate_destroy(rt_surrogate *s, rt_stream_t stream);
/* Parameter block in/out (device float32[60033]); set resets the Adam state. */
rt_status rt_surrogate_set_params(rt_surrogate *s, const float *params, rt_stream_t stream);
rt_status rt_surrogate_get_params(const rt_surrogate *s, float *params, rt_stream_t stream);
/* Full training state (device float32[3*60033 + 1]): parameters, Adam first
 * and second moments, then the step count; for checkpoint / resume. */
rt_status rt_surrogate_get_state(const rt_surrogate *s, float *state, rt_stream_t stream);
rt_status rt_surrogate_set_state(rt_surrogate *s, const float *state, rt_stream_t stream);
/* Scene bounds (host float[3] each) used to normalise origins. */
rt_status rt_surrogate_set_bounds(rt_surrogate *s, const float *lo, const float *hi);

/* p_out[m] = network output p (the sigmoid) for explicit rays (device
 * pos[m*3], dir[m*3]); the visibility estimate is p / (p + w (1 - p)). */
rt_status rt_surrogate_forward(const rt_surrogate *s, const float *pos, const float *dir, int64_t m,
                               float *p_out, rt_stream_t stream);
/* Mean weighted BCE over m explicit samples (targets y[m], weight
 * cfg.pos_weight on the y log p term) and its gradient with respect to the
 * parameter block: grad_out[60033] and loss_out[1] (device). */
rt_status rt_surrogate_loss_grad(const rt_surrogate *s, const float *pos, const float *dir,
                                 const float *y, int64_t m, float *grad_out, float *loss_out,
                                 rt_stream_t stream);
/* `steps` Adam steps on samples of an implicit ray set over `bvh` (DIRS):
 * each step draws cfg.batch ray ids r uniformly (Philox4x64-10, counter
 * (i, step, 0, 0), key (seed, 1); r = floor(x R / 2^64) for the first output
 * word x and R rays in the set), builds the ray as the tracer does and uses
 * T_target[r] (the traced visibility of the whole set) as the target.  Sets
 * the scene bounds from `bvh`.  loss_curve (device float32[steps], may be
 * NULL) receives each step's mean loss.  Every sum of a step runs in a fixed
 * order, so training is bit-reproducible, and n steps in one call give the
 * same parameters as n one-step calls with the same seed.  Within a call the
 * steps' kernels are launched with programmatic stream serialisation (each
 * orders itself against the previous one); work the caller enqueues after
 * the call follows the last of them in plain stream order. */
rt_status rt_surrogate_train(rt_surrogate *s, const rt_bvh *bvh, const rt_rayspec *samples,
                             const float *T_target, int32_t steps, uint64_t seed,
                             float *loss_curve, rt_stream_t stream);
/* Visibility of an implicit ray set over `bvh` (DIRS or ENV, optionally a
 * ray_ids subset) from the surrogate: T_out[i] = p / (p + w (1 - p)), the
 * network's estimate (= p for w = 1).  If band > 0, rays with
 * |p - 0.5| < band are traced on `bvh` instead (the fallback: one warp per
 * ray, RT_KERNEL_WARP_RAY) and T_out holds the traced value, bit-equal to
 * rt_trace_visibility with that kernel; n_fallback (device int64[1], may be
 * NULL) receives their
 * number.  The scene bounds used to normalise origins are the surrogate's.
 * Errors: RT_ERR_INVALID_ARG. */
rt_status rt_surrogate_infer(const rt_surrogate *s, const rt_bvh *bvh, const rt_rayspec *rays,
                             float band, float *T_out, int64_t *n_fallback, rt_stream_t stream);

/* rt_surrogate_infer without any device allocation during the call (the paper
 * has no counterpart).  For callers that may not let a library allocate
 * device memory mid-call: engines that reserve the whole device budget up
 * front and forbid allocation in their frame loop, or hosts whose device
 * memory belongs to another runtime's allocator.  The fallback lists and
 * counters live in a fixed 16 MiB + 256 B array inside the library, reserved
 * on every device that loads it until the process exits.  Same arguments and
 * results as rt_surrogate_infer; at most 1,048,576 rays per call (more:
 * RT_ERR_INVALID_ARG before anything is enqueued).  The first call in each
 * CUDA context (once per device, and again after a device reset) looks up
 * the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls share the array and
 * it keeps the previous call's contents (the call clears its counter itself):
 * calls that overlap on the GPU (other streams, other threads) race. */
rt_status rt_surrogate_infer_noalloc(const rt_surrogate *s, const rt_bvh *bvh, const rt_rayspec *rays,
                                     float band, float *T_out, int64_t *n_fallback, rt_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Autotuning and multi-scene batches (not in the paper)                      */
/* ------------------------------------------------------------------------ */

/* Picks the traversal strategy (rt_kernel) and the work order (order_block)
 * for a full implicit ray set (DIRS, ENV or HEMI, no ray_ids) over `bvh`: each
 * candidate traces the same four contiguous blocks of tiles of 32 Gaussians
 * spread over the Morton range (all directions; about 4M rays), timed with
 * CUDA events after a warm-up run; candidates are the 4-wide strategies
 * (the binary ones when the tree has no 4-wide form); the fastest is written
 * into opts->kernel and opts->order_block (other fields untouched) when it
 * beats the default strategy (RT_KERNEL_WIDE for DIRS, RT_KERNEL_RAY_REFILL
 * for ENV and HEMI) by more than 3 %, else the default with its best
 * order_block.  Results
 * are cached in-process per (device, log2 n, ray kind, K).  T_scratch must
 * hold rt_rayspec_count(bvh, rays) floats.  Synchronises `stream`. */
rt_status rt_trace_autotune(const rt_bvh *bvh, const rt_rayspec *rays, float *T_scratch,
                            rt_trace_opts *opts, rt_stream_t stream);

typedef struct rt_batch rt_batch;

/* One scene of a batch: its tree, a full implicit ray set over it (DIRS or
 * ENV, no ray_ids), and the output T_out[rt_rayspec_count(bvh, &rays)]. */
typedef struct {
    const rt_bvh *bvh;
    rt_rayspec rays;
    float *T_out;
} rt_batch_job;

/* Prepares one persistent launch over all jobs: a device work queue of
 * 32-ray items ordered scene by scene, largest estimated cost first; each
 * job's strategy and work order from rt_trace_autotune (autotune != 0) or the
 * defaults.  The queue reset and the launch are captured once into a CUDA
 * graph.  Jobs' trees, ray sets and outputs must stay alive until
 * rt_batch_destroy.  At most 4096 jobs.  Synchronises `stream`. */
rt_status rt_batch_create(const rt_batch_job *jobs, int32_t n_jobs, int32_t autotune, rt_stream_t stream,
                          rt_batch **out);
/* Replays the captured graph on `stream`: every job's T_out is written. */
rt_status rt_batch_run(rt_batch *batch, rt_stream_t stream);
/* Host outputs (may be NULL): total rays, total work items, and per job the
 * chosen kernel and order_block (arrays of n_jobs, in job order). */
rt_status rt_batch_info(const rt_batch *batch, int64_t *n_rays, int64_t *n_items, int32_t *kernel,
                        int32_t *order_block);
rt_status rt_batch_destroy(rt_batch *batch, rt_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* RT3DG_H */

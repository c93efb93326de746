/*
 * qrt -- instanced-quad ray tracing and path tracing on one GB300 (sm_103a).
 *
 * C ABI of the hot path of an interactive production-scene path tracer: a
 * two-level acceleration structure (a top-level BVH over object instances,
 * one BVH per object; Section 4.2 "Beyond Statistics" and Section 5.2
 * "Geometry Types, Complexity, and Memory Consumption"), quads as the
 * primitive (Section 5.2, "Quads"), closest-hit and any-hit ray queries, and
 * a diffuse path tracer with a maximum path depth and one sample per pixel
 * per progressive frame (Section 5.4 "Shading"; Section 6 "Results").
 *
 * Conventions shared by every entry point:
 *  - Every function returns an int status: QRT_OK (0) or a negative QRT_ERR_*
 *    code; qrt_last_error() gives a message for the calling thread.
 *  - Pointers named d_* are caller-owned DEVICE memory on the current CUDA
 *    device; every other pointer is host memory.  The library never frees
 *    caller memory and keeps no pointer to it after the call returns, except
 *    where a graph (qrt_render_graph_create) records device pointers.
 *  - Device work is enqueued on the caller's stream (qrt_stream is the same
 *    type as cudaStream_t; NULL = legacy default stream) and the call returns
 *    without waiting.  Problems found on the device (stack overflow, step
 *    limit) set a per-scene error word that qrt_check() reads.
 *  - n == 0 is a no-op that returns QRT_OK.
 *  - A scene is immutable after creation and may be used from several
 *    streams at once for tracing and rendering.
 *
 * Units and layouts: world space is right-handed, z up.  Transforms are
 * object->world, row-major 3x4 (the last column is the translation).  A quad
 * (v0,v1,v2,v3) is the pair of triangles (v0,v1,v2) and (v0,v2,v3); quads
 * are double-sided.  A ray hits at t only when tmin < t < tmax.
 */
#ifndef QRT_H
#define QRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QRT_VERSION 1

/* qrt_params.flags */
#define QRT_FLAG_STAGE_TIMES 1u /* record GPU time of each wavefront stage (qrt_stage_times) */

/* Most key lights one render takes (qrt_params.n_lights). */
#define QRT_MAX_LIGHTS 32
/* Largest per-face texture resolution (qrt_params.tex_res). */
#define QRT_MAX_TEX_RES 16

enum {
    QRT_OK = 0,
    QRT_ERR_INVALID_ARG = -1,    /* bad handle, NULL pointer, size or value */
    QRT_ERR_ALIGN = -2,          /* a device pointer is not aligned as stated */
    QRT_ERR_OOM = -3,            /* device or host allocation failed */
    QRT_ERR_CUDA = -4,           /* a CUDA runtime call failed (no device, launch error) */
    QRT_ERR_STACK_OVERFLOW = -5, /* a traversal stack overflowed on the device */
    QRT_ERR_STEP_LIMIT = -6,     /* a ray exceeded the traversal step limit */
    QRT_ERR_NOT_READY = -7       /* resource not available (e.g. no free work slot) */
};

typedef struct CUstream_st* qrt_stream; /* identical to cudaStream_t */
typedef struct qrt_scene_s* qrt_scene;
typedef struct qrt_graph_s* qrt_graph;

/* One object (prototype): n_verts packed float3 vertices and n_quads quads of
 * four vertex indices each.  Host memory, copied during qrt_scene_create. */
typedef struct {
    const float* verts;
    uint32_t n_verts;
    const uint32_t* quads;
    uint32_t n_quads;
} qrt_mesh;

/* Ray: 32 bytes.  Ray arrays must be 16-byte aligned.  d need not be unit
 * length; t is measured in units of |d|. */
typedef struct {
    float o[3];
    float tmin;
    float d[3];
    float tmax;
} qrt_ray;

/* Closest hit: 16 bytes.  inst = instance index, prim = quad index within
 * that instance's mesh, uv = quad-space (u, v) as two unorm16 (u in the low
 * half).  Miss: inst = prim = 0xFFFFFFFF, t = tmax.  Among hits at exactly
 * the same t the smallest (inst, prim) wins. */
typedef struct {
    float t;
    uint32_t inst;
    uint32_t prim;
    uint32_t uv;
} qrt_hit;

/* Pinhole camera.  Pixel (x, y), y = 0 the top row, is sampled at
 * (x + xi1, y + xi2); vfov is the vertical field of view in degrees.
 * pixel_base gives the first global pixel index of this view: the random
 * stream of a sample is keyed by (pixel_base + y*w + x, sample, bounce), so
 * distinct views should use disjoint ranges.  The call draws samples
 * sample_base .. sample_base + spp - 1 of every pixel: progressive rendering
 * (Section 5.4, one sample per pixel per frame) passes the frame number with
 * spp = 1 and sums the frames with qrt_accumulate.
 * Crop: crop_w = crop_h = 0 renders the whole w x h frame; otherwise only
 * the rectangle [crop_x, crop_x + crop_w) x [crop_y, crop_y + crop_h) of the
 * frame (it must lie inside it), with the camera and the random streams of
 * the whole frame, so a crop's pixels are bit-identical to the same pixels
 * of a whole-frame render.  This is how an image-parallel renderer hands a
 * rank its tiles (Section 5.5, "The Distributed FrameBuffer": image tiles
 * assigned to nodes that each hold the whole scene).
 * out_rgb: DEVICE float [rh*rw*3], row-major over the rendered region (rw x
 * rh = crop_w x crop_h, or w x h), receives the mean radiance over the
 * call's spp samples (overwritten). */
typedef struct {
    float eye[3];
    float look[3];
    float up[3];
    float vfov_deg;
    uint32_t w, h, spp;
    uint32_t sample_base;
    uint64_t pixel_base;
    float* out_rgb;
    uint32_t crop_x, crop_y, crop_w, crop_h;
} qrt_view;

/* Launch tuning; 0 in any field selects the library default.
 *   block          threads per block: 64, 128, 192 or 256 (default)
 *   blocks_per_sm  resident blocks per SM for persistent kernels (default:
 *                  as many as the register budget allows)
 *   batch          single kernel: pixels a warp claims per fetch, in units
 *                  of 32; wavefront and ray queries: rays a lane claims per
 *                  fetch (1..64, default 1)
 *   stack          traversal stack entries per ray (32 or 64)
 *   fetch          node fetch width in bytes (16: 4x128-bit, 32: 2x256-bit
 *                  loads, default)
 *   occupancy      trace kernels' register budget as resident warps per SM:
 *                  16 (up to 128 registers a thread), 24 (80), 32 (64),
 *                  40 (48, default) or 48 (40); more warps hide the latency
 *                  of the dependent node loads, at the price of spills
 *   mode           renderer: 0 = default (wavefront), 1 = single persistent
 *                  kernel (a lane renders whole pixels), 2 = wavefront (stages
 *                  gen / trace / shade / shadow / accumulate over queues; a
 *                  lane of a trace kernel takes a new ray as soon as its own
 *                  is done).  Both give bit-identical images.
 *   chunk_log2     wavefront: paths per chunk = 2^chunk_log2 (10..26); 0 =
 *                  fit the call: the smallest 2^k >= its paths, k in
 *                  10..25.  Sets the size of the per-stream workspace
 *                  (about 164 B per path; it grows when a call needs more) */
typedef struct {
    uint32_t block;
    uint32_t blocks_per_sm;
    uint32_t batch;
    uint32_t stack;
    uint32_t fetch;
    uint32_t occupancy;
    uint32_t mode;
    uint32_t chunk_log2;
} qrt_tuning;

/* Path-tracing parameters.
 *   max_depth   closest-hit rays per path, camera ray included (1..256)
 *   seed        Philox key
 *   env         radiance of the uniform environment, reached by rays that
 *               leave the scene
 *   sun_dir     direction toward a directional sun (normalised internally);
 *   sun_E       its irradiance (RGB); all zero disables the sun and its
 *               shadow rays
 *   d_path_log  optional DEVICE buffer for diagnostics (NULL = off): per path
 *               max_depth pairs (inst, prim) of the hits, 0xFFFFFFFF where the
 *               path had no such ray, then one word of sun shadow bits (bit
 *               2i: a shadow ray was traced at vertex i, bit 2i+1: it was
 *               occluded; first 16 vertices) and one word of key-light shadow
 *               bits (the same layout).  Path p of view v sits at
 *               sum_{u<v}(rw*rh*spp)_u + (y'*rw + x')*spp + sample, (x', y')
 *               the pixel within the view's rendered region, each path taking
 *               2*max_depth + 2 words.
 *   max_steps   traversal step limit per ray (0 = 2^20); exceeding it stops
 *               that ray and raises QRT_ERR_STEP_LIMIT.
 *   tuning      launch tuning (zeros = defaults).
 *   d_ray_log   optional DEVICE float buffer for diagnostics (NULL = off),
 *               16-byte aligned, indexed by path like d_path_log: per path
 *               max_depth records of 16 floats, one per depth i = 1..max_depth:
 *               the closest-hit ray traced at depth i as a qrt_ray (o, tmin,
 *               d, tmax; the camera ray at depth 1, then each bounce ray as
 *               spawned), the spawn point of the hit of depth i (3 floats and
 *               one unused: the origin of its shadow rays and of the next
 *               ray), and the direction and distance of its key-light shadow
 *               ray (4 floats).  Records of rays a path did not trace are
 *               zero.  The exact FP32 rays let a test re-trace, in FP64, the
 *               ray on which a path first left the oracle's path.
 *   d_tex, tex_res  optional per-face textures (Section 5.3: a Ptex texture,
 *               baked on each face, modulates the diffuse albedo): DEVICE
 *               float [n_quads * tex_res^2 * 3], quad row q's texels row-major
 *               in v then u; texel (i, j) covers quad-space [i/R, (i+1)/R] x
 *               [j/R, (j+1)/R] and a hit at (u, v) takes the bilinear value
 *               between texel centres, clamped to the face.  The diffuse
 *               albedo is d_albedo[q] times that value.  NULL / 0 = none;
 *               tex_res at most QRT_MAX_TEX_RES.
 *   n_lights, lights  key lights (Section 4.1: quad-shaped key lights):
 *               HOST float [n_lights * 12], per light a parallelogram (corner,
 *               edge1, edge2) emitting radiance (RGB, 3 floats) on the side of
 *               edge1 x edge2; copied during the call.  Reached only by
 *               next-event estimation: at each path vertex one light is
 *               picked uniformly and a point uniformly on it, from the random
 *               stream (pixel, sample, 2^30 + depth), and a shadow ray is
 *               traced toward that point.  At most QRT_MAX_LIGHTS. */
typedef struct {
    uint32_t max_depth;
    uint32_t flags;
    uint64_t seed;
    float env[3];
    float sun_dir[3];
    float sun_E[3];
    uint32_t max_steps;
    uint32_t* d_path_log;
    qrt_tuning tuning;
    float* d_ray_log;
    const float* d_tex;
    uint32_t tex_res;
    uint32_t n_lights;
    const float* lights;
} qrt_params;

/* BVH build options (NULL = defaults).
 *   max_leaf   quads per BLAS leaf (1..8, default 2)
 *   sah_bins   binned-SAH bins (4..64, default 16)
 *   threads    host threads for the build (0 = all cores)
 *   degenerate 1 = build a deliberately deep chain-shaped BLAS (test aid for
 *              the stack-overflow path); 0 = normal SAH build
 *   inst_boxes how tightly the TLAS bounds each instance: 1 = the world box of
 *              its BLAS's transformed root box; k = 2..6 = the union of the
 *              world boxes of the BLAS nodes k-1 levels below the root
 *              (smaller boxes of a rotated object overlap fewer rays; the
 *              result is intersected with the root-box bound); 0 = default
 *              (6: up to 1024 boxes per instance, fewer for small meshes,
 *              whose cut stops at their leaves)
 *   tlas_builder 0 = binned SAH on the host threads (default); 1 = linear BVH
 *              over the instances' Morton order built on the current device
 *              (much faster to build, looser tree); 2 = the same linear BVH
 *              steps run on the host (a test aid that needs no GPU).  Every
 *              TLAS passes the same invariant check before upload.
 *   blas_builder the same choice for the per-mesh BLASes: 0 = binned SAH per
 *              mesh on the host threads (default); 1 = all meshes' linear BVHs
 *              in one pass on the current device (at most 8192 meshes; not
 *              with degenerate); 2 = those steps on the host (test aid).
 *              Every BLAS passes the invariant check before upload. */
typedef struct {
    uint32_t max_leaf;
    uint32_t sah_bins;
    uint32_t threads;
    uint32_t degenerate;
    uint32_t inst_boxes;
    uint32_t tlas_builder;
    uint32_t blas_builder;
} qrt_build_opts;

/* Scene statistics (host).  build_seconds covers the host build (phases
 * 0-4); phase_seconds: 0 BLAS builds, 1 BLAS checks, 2 instance records and
 * bounds, 3 TLAS build and check, 4 concatenation, 5 upload. */
typedef struct {
    uint64_t n_meshes, n_instances, n_quads;
    uint64_t blas_nodes, tlas_nodes;
    uint64_t device_bytes;
    uint32_t max_blas_depth, tlas_depth;
    double build_seconds;
    double phase_seconds[6];
} qrt_scene_stats;

const char* qrt_last_error(void);
int qrt_version(void);

/* Build the two-level structure on the host and upload it to the current
 * device (Section 5.2: objects are instanced, quads are the primitive).
 * meshes: n_mesh host descriptors; xforms: host float [n_inst*12]; mesh_ids:
 * host uint32 [n_inst].  Quad albedo rows are numbered mesh by mesh in order
 * (mesh m's quad q is row sum_{k<m} n_quads_k + q).  On success *out owns all
 * device memory of the scene.  Errors: INVALID_ARG (NULL/zero counts, index
 * out of range, non-invertible transform), OOM, CUDA. */
int qrt_scene_create(const qrt_mesh* meshes, uint32_t n_mesh, const float* xforms,
                     const uint32_t* mesh_ids, uint64_t n_inst, const qrt_build_opts* opts,
                     qrt_scene* out);
int qrt_scene_destroy(qrt_scene scene);
int qrt_scene_stats_get(qrt_scene scene, qrt_scene_stats* out);

/* Closest hit for n rays (Section 6, Table 1: traversal and intersection dominate the
 * frame).  d_rays: n qrt_ray, d_hits: n qrt_hit, both 16-byte aligned.
 * tuning may be NULL. */
int qrt_trace_closest(qrt_scene scene, const qrt_ray* d_rays, uint64_t n, qrt_hit* d_hits,
                      const qrt_tuning* tuning, qrt_stream stream);

/* Any hit (occlusion) for n rays: bit (i % 32) of d_occ_bits[i / 32] is set
 * when ray i hits anything in (tmin, tmax).  d_occ_bits: ceil(n/32) uint32,
 * overwritten. */
int qrt_trace_any(qrt_scene scene, const qrt_ray* d_rays, uint64_t n, uint32_t* d_occ_bits,
                  const qrt_tuning* tuning, qrt_stream stream);

/* Path-trace n_views views (Section 5.4, progressive path tracing; one
 * launch covers every (view, pixel) and all of each pixel's spp samples).
 * d_albedo: DEVICE float [n_quads*3], per unique quad RGB albedo.  Each
 * view's out_rgb receives the mean over its spp samples; results do not
 * depend on n_views, on the tuning or on other views in the same call.
 * The wavefront renderer enqueues its work on `stream` and on a second
 * stream that the library keeps per (scene, stream) and joins back before
 * returning control of the stream's order: the call stays stream-ordered. */
int qrt_render_spp(qrt_scene scene, const qrt_view* views, uint32_t n_views,
                   const float* d_albedo, const qrt_params* params, qrt_stream stream);

/* qrt_render_spp for callers that cannot allocate device memory -- for
 * example an interactive frame loop that must not stall on cudaMalloc, or a
 * process whose device memory is owned by another allocator (a framework's
 * caching pool, a host application that budgets every byte).  No paper
 * counterpart: it is an interface variant of this library, with the same
 * results as qrt_render_spp.
 *
 * It renders with the wavefront renderer, using as scratch a fixed array of
 * about 17 MB compiled into the library (device global memory held on every
 * GPU that loads the library, until the process exits), enough for chunks of
 * 2^17 paths; any number of views and paths is processed chunk by chunk, so
 * a view's spp may be at most 2^17 (larger is rejected with
 * QRT_ERR_INVALID_ARG).  The call allocates nothing and calls no cudaMalloc
 * or cudaFree.  The first call on a device -- and the first after that
 * device's context is made anew, e.g. after cudaDeviceReset -- looks up the
 * array's device address; make that first call before any stream capture.
 * Tuning is read as for qrt_render_spp (zeros = library defaults), except
 * that the renderer is always the wavefront one: tuning.mode may be 0 or 2,
 * and tuning.chunk_log2 0 (= 17) or at most 17; anything else is rejected
 * with QRT_ERR_INVALID_ARG.  Every call shares the one array and clears what
 * must start at zero itself, so calls that overlap on the GPU (different
 * streams, or different host threads) race with each other: order them on
 * one stream. */
int qrt_render_spp_static(qrt_scene scene, const qrt_view* views, uint32_t n_views,
                          const float* d_albedo, const qrt_params* params, qrt_stream stream);

/* Adjoint of qrt_render_spp with respect to the albedo: adds
 * sum_v sum_pixel sum_c d_dimage[v][pixel*3+c] * dI_v[pixel,c]/d albedo[q,c]
 * into d_grad_albedo (DEVICE float [n_quads*3], accumulated, not cleared).
 * Paths are recomputed from their random streams instead of being stored
 * (path replay); contributions are added with FP32 atomics.  Per path the
 * wavefront renderer keeps only its radiance and one visibility bit per
 * shadow ray of depths 1..32, so its replay traces the closest-hit rays again
 * but not those shadow rays.  d_dimage: host array of n_views DEVICE
 * pointers, each float [h*w*3]. */
int qrt_render_adjoint(qrt_scene scene, const qrt_view* views, uint32_t n_views,
                       const float* d_albedo, const float* const* d_dimage,
                       float* d_grad_albedo, const qrt_params* params, qrt_stream stream);

/* Progressive accumulation on the device: d_sum[i] += d_frame[i] for i < n
 * (FP32, in call order) and, if d_mean is not NULL, d_mean[i] = d_sum[i] /
 * frames, where frames counts the frames summed so far (including this
 * one, >= 1).  Frames rendered with spp = 1 and sample_base = 0, 1, 2, ...
 * summed from a zeroed d_sum give exactly the image of one call with
 * spp = frames: the renderer sums a pixel's samples in the same order.
 * All pointers DEVICE float [n]; d_mean may alias d_frame. */
int qrt_accumulate(float* d_sum, const float* d_frame, float* d_mean, uint64_t n, uint32_t frames,
                   qrt_stream stream);

/* Mean-squared image loss and its gradient on the device:
 * *d_loss = sum_i (img_i - target_i)^2 / n and d_dimage_i = 2 (img_i - target_i) / n
 * (d_loss: one double; d_dimage may alias nothing).  n counts floats. */
int qrt_l2_loss(const float* d_img, const float* d_target, uint64_t n, double* d_loss,
                float* d_dimage, qrt_stream stream);

/* Capture qrt_render_spp(views...) once into a CUDA graph (with its own work
 * counter) and replay it with qrt_graph_launch.  The graph keeps the device
 * pointers given here (albedo, out_rgb, path log); views and params are
 * copied. */
int qrt_render_graph_create(qrt_scene scene, const qrt_view* views, uint32_t n_views,
                            const float* d_albedo, const qrt_params* params, qrt_graph* out);
int qrt_graph_launch(qrt_graph graph, qrt_stream stream);
int qrt_graph_destroy(qrt_graph graph);

/* Diagnostics: as qrt_render_spp / qrt_trace_closest (any = 0) /
 * qrt_trace_any (any = 1), and additionally add the traversal counters of the
 * launch into d_stats (DEVICE uint64 [6], 8-byte aligned, accumulated):
 * rays traced, inner nodes visited, quads tested, instances entered, quad
 * tests re-done in FP64, path vertices shaded.  These counts give the algorithmic bytes of a
 * launch (64 B per node, 48 B per quad, 64 B per instance entry).  Rays,
 * shaded vertices and every result are reproducible; node, quad and instance
 * counts may vary slightly from launch to launch, because a lane defers a
 * BLAS leaf while its warp tests inner nodes, so the moment its hit distance
 * tightens (and which stack entries are culled) depends on the rays that
 * share its warp. */
int qrt_render_spp_stats(qrt_scene scene, const qrt_view* views, uint32_t n_views,
                         const float* d_albedo, const qrt_params* params,
                         unsigned long long* d_stats, qrt_stream stream);
int qrt_trace_stats(qrt_scene scene, int any, const qrt_ray* d_rays, uint64_t n, void* d_out,
                    const qrt_tuning* tuning, unsigned long long* d_stats, qrt_stream stream);

/* Cost map (the paper's per-pixel cost heat map, Section 6): as
 * qrt_render_spp_stats, and additionally writes for every pixel of view v
 * the mean over its samples of the inner BVH nodes (both levels) visited by
 * all rays of the path, closest-hit and shadow, into d_cost[v] (host array
 * of n_views DEVICE pointers, each float [h*w], row-major).  Summed over the
 * image (times spp) the maps equal the launch's node counters; like them they
 * may vary slightly between launches.  Wavefront renderer only (tuning.mode 0
 * or 2). */
int qrt_render_cost(qrt_scene scene, const qrt_view* views, uint32_t n_views, const float* d_albedo,
                    const qrt_params* params, float* const* d_cost, unsigned long long* d_stats,
                    qrt_stream stream);

/* Per-stage GPU time of wavefront renders made with QRT_FLAG_STAGE_TIMES (the
 * breakdown of the paper's Table 1): after waiting for the stream, writes the
 * milliseconds and launch counts accumulated since the last reset for the
 * stages 0 camera-ray generation, 1 closest-hit tracing, 2 shading,
 * 3 shadow-ray tracing, 4 accumulation (ms[5], launches[5]); reset != 0
 * starts a new accumulation.  Timers are per scene: time one stream at a
 * time.  A timed render runs its stages one after another; an untimed one
 * runs the shadow rays of each depth on a second stream beside the next
 * depth's closest-hit rays. */
int qrt_stage_times(qrt_scene scene, qrt_stream stream, double* ms, uint32_t* launches, int reset);

/* Measurement helper with no counterpart in the paper: reads the DEVICE
 * buffer d_buf (16-byte aligned, bytes a multiple of 16) reps times with
 * L2-only 16-byte loads on the current device, XOR-folding the data into
 * *d_sink (DEVICE uint32, its value meaningless).  Timed by the caller on
 * the stream; with a buffer that fits in L2 it gives the L2 read bandwidth
 * that bounds traversal of a cache-resident BVH.  bytes = 0 or reps = 0 is a
 * no-op. */
int qrt_read_bandwidth(const void* d_buf, uint64_t bytes, uint32_t reps, uint32_t* d_sink,
                       qrt_stream stream);

/* Wait for the stream, then read and clear the scene's device error word.
 * Returns QRT_OK, QRT_ERR_STACK_OVERFLOW, QRT_ERR_STEP_LIMIT or QRT_ERR_CUDA. */
int qrt_check(qrt_scene scene, qrt_stream stream);

/* Host only (no GPU needed): build one mesh's BLAS as qrt_scene_create would,
 * verify its invariants (every quad referenced exactly once, every quantised
 * child box contains the exact child box, child boxes inside the parent's)
 * and report node count and depth.  Returns QRT_OK or INVALID_ARG with a
 * message naming the broken invariant. */
int qrt_blas_build_check(const qrt_mesh* mesh, const qrt_build_opts* opts, uint64_t* n_nodes,
                         uint32_t* depth);

/* Test aid: builds the BLASes of n_mesh meshes as qrt_scene_create would
 * (opts->blas_builder 1 needs a CUDA device; 0 and 2 run on the host),
 * verifies every one as qrt_blas_build_check does and reports the total node
 * count and the largest depth.  Errors: INVALID_ARG, CUDA. */
int qrt_blases_build_check(const qrt_mesh* meshes, uint32_t n_mesh, const qrt_build_opts* opts,
                           uint64_t* n_nodes, uint32_t* max_depth);

/* Test aid: builds a TLAS over n host boxes (float [n*6]: lo xyz, hi xyz)
 * with opts->tlas_builder (1 needs a CUDA device, 0 and 2 run on the host),
 * runs the invariant check (every box referenced once, every quantised child
 * box containing its subtree) and reports the node count and depth.  Errors:
 * INVALID_ARG (bad boxes, failed check), CUDA. */
int qrt_tlas_build_check(const float* boxes, uint64_t n, const qrt_build_opts* opts,
                         uint64_t* n_nodes, uint32_t* depth);

/* Test aid: sorts n (key, value) pairs by bits [0, end_bit) of the 64-bit
 * key, stably (pairs whose sorting bits are equal keep their input order),
 * with the device radix sort that the linear BVH builds use to order items
 * along their Morton curve (Karras, HPG 2012).  keys / vals: host
 * arrays of n entries, read; keys_out / vals_out: host arrays of n entries,
 * written with the sorted pairs (whole keys, including bits at and above
 * end_bit).  Allocates and frees device memory on the current device.
 * n <= 2^32 - 2049, end_bit <= 64.  Errors: INVALID_ARG (NULL array, n or
 * end_bit out of range), CUDA. */
int qrt_test_sort_pairs(const uint64_t* keys, const uint32_t* vals, uint64_t n, uint32_t end_bit,
                        uint64_t* keys_out, uint32_t* vals_out);

#ifdef __cplusplus
}
#endif
#endif /* QRT_H */

/*
 * FP64 CPU oracle for the instanced-quad path tracer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path: its own scene structures, BVH, intersection routine
 * (Moller-Trumbore instead of the watertight test), camera, sampling and
 * Philox generator, all in double precision from FP32 inputs.
 *
 * What it follows:
 *   - two-level instancing: a top-level structure over object instances, one
 *     structure per object, rays moved into object space (Section 5.2,
 *     "Geometry Types, Complexity, and Memory Consumption"; Section 4.2,
 *     "Beyond Statistics");
 *   - quads as the primitive, each quad the pair of triangles it was merged
 *     from (Section 5.2, paragraph "Quads");
 *   - a path tracer with progressive 1-spp accumulation and a maximum path
 *     depth (Section 5.4 "Shading"; Section 6 "Results": depth five).
 * Choices the paper leaves open are fixed identically on both sides and are
 * listed in the design notes ("readings").
 *
 * Parity status per function:
 *   ora_philox            pinned: known-answer vector and an external
 *                         Philox4x32-10 implementation (Triton interpreter).
 *   ora_intersect_quad    pinned: closed-form plane intersections, edges,
 *                         vertices, misses.
 *   ora_trace_*           pinned: BVH == brute force (exact), instanced ==
 *                         flattened world-space brute force.
 *   ora_render            pinned: flat-plane closed form (env and sun),
 *                         white furnace, value-set invariant.
 *   ora_sample_cosine     pinned: moments E[cos]=2/3, E[cos^2]=1/2, ONB.
 *   ora_render_grad       pinned: closed form on a flat plane, central
 *                         finite differences of ora_render.
 *   ora_camera_ray        pinned: centre and corner rays in closed form.
 *   ora_tex_lookup        pinned: constant and linear texel grids reproduced
 *                         exactly, clamping at the face's edges.
 *   ora_light_sample      pinned: the mean over samples converges to the
 *                         closed-form irradiance of a Lambertian polygon
 *                         (Lambert's formula); lights facing away or below
 *                         the horizon give nothing.
 */
#ifndef QRT_ORACLE_H
#define QRT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ora_scene ora_scene;

typedef struct {
    float eye[3], look[3], up[3];
    float vfov_deg;
    uint32_t w, h, spp;
    uint32_t sample_base;  // samples sample_base .. sample_base + spp - 1 are drawn
    uint64_t pixel_base;
} ora_view;

typedef struct {
    uint32_t max_depth;
    uint64_t seed;
    float env[3];
    float sun_dir[3];
    float sun_E[3];
    uint32_t tex_res;     /* per-face textures: R x R texels per quad (0 = none) */
    const float* tex;     /* n_quads x R x R x 3, per quad row-major in v then u */
    uint32_t n_lights;    /* key lights (0 = none) */
    const float* lights;  /* n_lights x 12: corner, edge1, edge2, radiance */
} ora_params;

/* Philox4x32-10: out = philox(ctr, key). */
void ora_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Scene: n_mesh meshes (verts float3 packed, quads 4 x u32), n_inst instances
 * with object->world float 3x4 row-major transforms.  Arrays are copied. */
ora_scene* ora_scene_new(uint32_t n_mesh, const float* const* verts, const uint32_t* n_verts,
                         const uint32_t* const* quads, const uint32_t* n_quads,
                         uint64_t n_inst, const float* xforms, const uint32_t* mesh_ids);
void ora_scene_free(ora_scene* s);
uint64_t ora_scene_n_quads(const ora_scene* s);

/* One ray against one quad (v: 4 x float3).  Returns 1 on hit with t in
 * (tmin, tmax); writes t and quad-space (u, v). */
int ora_intersect_quad(const double o[3], const double d[3], double tmin, double tmax,
                       const double v[12], double* t, double* u, double* w);

/* rays: n x 8 floats (o, tmin, d, tmax).  mode 0 = BVH, 1 = brute force over
 * all instances and quads, 2 = brute force over world-space (flattened)
 * vertices.  Miss: inst = prim = 0xFFFFFFFF, t = tmax. */
void ora_trace_closest(const ora_scene* s, const float* rays, uint64_t n, int mode,
                       double* t, uint32_t* inst, uint32_t* prim, double* u, double* v,
                       int nthreads);
void ora_trace_any(const ora_scene* s, const float* rays, uint64_t n, int mode,
                   uint8_t* occluded, int nthreads);

/* Camera ray of pixel (x, y) with jitter (xi1, xi2): writes o[3], d[3]. */
void ora_camera_ray(const ora_view* v, uint32_t x, uint32_t y, double xi1, double xi2,
                    double o[3], double d[3]);

/* Cosine-weighted direction about unit normal n from (xi1, xi2). */
void ora_sample_cosine(const double n[3], double xi1, double xi2, double out[3]);

/* Render the given pixels (indices y*w+x into the view; NULL = all, in
 * order).  rgb: n_pix x 3 doubles (mean over spp).  If log_inst/log_prim are
 * non-NULL they receive, per path (pixel-major, then sample), max_depth
 * entries of the hit instance / quad (0xFFFFFFFF = no hit); log_shadow gets
 * per path 2 bits per vertex for the first 16 vertices: bit 2i = sun shadow
 * ray traced at vertex i, bit 2i+1 = it was occluded; log_light the same
 * for the key-light shadow ray.  max_depth is 1..256.
 * log_rays (nullable, zeroed by the caller) receives per path max_depth
 * records of 13 doubles: origin and direction of the closest-hit ray traced
 * at that depth, the spawn point of its hit (origin of its shadow rays and
 * of the next ray), and the unit direction and distance of the key-light
 * shadow ray (records of rays not traced stay as given).
 * n_escaped/n_truncated (nullable) count paths that left the scene / ran
 * out of depth on a surface.  Returns -1 for a bad depth or a missing
 * texture or light array. */
int ora_render(const ora_scene* s, const ora_view* view, const float* albedo,
               const ora_params* p, const int64_t* pixels, uint64_t n_pix,
               double* rgb, uint32_t* log_inst, uint32_t* log_prim, uint32_t* log_shadow,
               uint32_t* log_light, double* log_rays, uint64_t* n_escaped,
               uint64_t* n_truncated, int nthreads);

/* Per-face texture value of quad row at quad-space (u, v): bilinear between
 * texel centres of its res x res grid, clamped to the face. */
void ora_tex_lookup(const float* tex, uint32_t res, uint64_t row, double u, double v, double out[3]);

/* One key-light sample seen from x (unit normal nx) for uniforms xi[3]:
 * returns 1 and writes the unit direction toward the sampled point, its
 * distance and the estimator Le cos_x cos_l area n / d^2, or returns 0 when
 * the point faces away or lies below the horizon. */
int ora_light_sample(const float* lights, uint32_t n, const double xi[3], const double x[3],
                     const double nx[3], double dir[3], double* dist, double w[3]);

/* Gradient of sum_p sum_c dimage[p,c] * I[p,c] with respect to the per-quad
 * albedo (n_quads x 3), accumulated into grad (doubles, zeroed by caller),
 * by storing each path and differentiating its polynomial in the albedos.
 * dimage is indexed like rgb above (n_pix x 3). */
int ora_render_grad(const ora_scene* s, const ora_view* view, const float* albedo,
                    const ora_params* p, const int64_t* pixels, uint64_t n_pix,
                    const double* dimage, double* grad, int nthreads);

#ifdef __cplusplus
}
#endif
#endif

// Shading arithmetic shared by the path-tracing kernels: Philox4x32-10,
// camera rays, cosine sampling, normals and spawn offsets, and the
// warp-aggregated gradient atomics.  Every floating-point operation is an
// explicitly rounded intrinsic, so every kernel that uses these functions
// computes bit-identical paths.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"
#include "qrt_layout.h"

namespace qrt {

// Philox4x32-10 (Salmon et al., SC 2011).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ float u01(uint32_t x) {
    return __fmul_rn(__uint2float_rn(x >> 8), 5.9604644775390625e-08f);  // 2^-24
}

// Random draws of sample `sample` of global pixel `pix` at `bounce`.
__device__ __forceinline__ uint4 draw(uint64_t seed, uint64_t pix, uint32_t sample, uint32_t bounce) {
    return philox4x32_10(make_uint4((uint32_t)pix, (uint32_t)(pix >> 32), sample, bounce),
                         (uint32_t)seed, (uint32_t)(seed >> 32));
}

struct F3 {
    float x, y, z;
};
__device__ __forceinline__ F3 f3(float x, float y, float z) { return F3{x, y, z}; }
__device__ __forceinline__ float dot3(F3 a, F3 b) {
    return __fmaf_rn(a.x, b.x, __fmaf_rn(a.y, b.y, __fmul_rn(a.z, b.z)));
}
__device__ __forceinline__ F3 normalize3(F3 a) {
    const float inv = __frcp_rn(__fsqrt_rn(dot3(a, a)));
    return f3(__fmul_rn(a.x, inv), __fmul_rn(a.y, inv), __fmul_rn(a.z, inv));
}

// Frame coordinates (x, y) of pixel k of a view's rendered region, and the
// pixel's global index, which keys its random streams.
__device__ __forceinline__ uint64_t view_pixel(const ViewDev& V, uint64_t k, uint32_t* x, uint32_t* y) {
    const uint32_t ly = (uint32_t)(k / V.w);
    *x = V.x0 + (uint32_t)(k - (uint64_t)ly * V.w);
    *y = V.y0 + ly;
    return V.pixel_base + (uint64_t)*y * V.fw + *x;
}

// Ray-log record of depth i (1-based) of path g: the closest-hit ray as
// (o, 0, d, inf), the spawn point of its hit, the key-light shadow ray's
// direction and distance (diagnostics only).
__device__ __forceinline__ float* ray_log_rec(const ParamsDev& P, uint64_t g, uint32_t i) {
    return P.ray_log + (g * P.max_depth + (i - 1)) * (uint64_t)kRayLogFloats;
}
__device__ __forceinline__ void log_ray(float* rec, F3 o, F3 d) {
    float4* r = reinterpret_cast<float4*>(rec);
    r[0] = make_float4(o.x, o.y, o.z, 0.f);
    r[1] = make_float4(d.x, d.y, d.z, __int_as_float(0x7f800000));
}
__device__ __forceinline__ void log_spawn(float* rec, F3 o) {
    reinterpret_cast<float4*>(rec)[2] = make_float4(o.x, o.y, o.z, 0.f);
}
__device__ __forceinline__ void log_light_ray(float* rec, F3 d, float dist) {
    reinterpret_cast<float4*>(rec)[3] = make_float4(d.x, d.y, d.z, dist);
}
__device__ __forceinline__ void clear_ray_log(float* rec0, uint32_t depth) {
    float4* r = reinterpret_cast<float4*>(rec0);
    for (uint32_t k = 0; k < (kRayLogFloats / 4) * depth; ++k) r[k] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Per-face texture value of quad row at quad-space (u, v) (qrt_params:
// bilinear between texel centres, clamped to the face), FP32.
__device__ __forceinline__ F3 tex_lookup(const float* tex, uint32_t R, uint32_t row, float u, float v) {
    const float fr = (float)R;
    const float s = fminf(fmaxf(__fmaf_rn(u, fr, -0.5f), 0.f), fr - 1.f);
    const float t = fminf(fmaxf(__fmaf_rn(v, fr, -0.5f), 0.f), fr - 1.f);
    const uint32_t i0 = (uint32_t)s, j0 = (uint32_t)t;
    const uint32_t i1 = min(i0 + 1u, R - 1u), j1 = min(j0 + 1u, R - 1u);
    const float fs = __fsub_rn(s, (float)i0), ft = __fsub_rn(t, (float)j0);
    const float* T = tex + (size_t)row * R * R * 3;
    const float* a = T + 3 * (j0 * R + i0);
    const float* b = T + 3 * (j0 * R + i1);
    const float* c = T + 3 * (j1 * R + i0);
    const float* d = T + 3 * (j1 * R + i1);
    float o[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = __fmaf_rn(fs, __fsub_rn(__ldg(b + k), __ldg(a + k)), __ldg(a + k));
        const float hi = __fmaf_rn(fs, __fsub_rn(__ldg(d + k), __ldg(c + k)), __ldg(c + k));
        o[k] = __fmaf_rn(ft, __fsub_rn(hi, lo), lo);
    }
    return f3(o[0], o[1], o[2]);
}

// One key-light sample seen from x with unit normal nx (qrt_params): light
// floor(xi0 n), point corner + xi1 edge1 + xi2 edge2; writes the unit
// direction toward it, its distance and the estimator Le cos_x cos_l
// |edge1 x edge2| n / d^2.  False when the point faces away from x or lies
// below its horizon.  FP32.
__device__ __forceinline__ bool light_sample(const ParamsDev& P, float xi0, float xi1, float xi2, F3 x,
                                             F3 nx, F3* dir, float* dist, F3* w) {
    const uint32_t k = min((uint32_t)__fmul_rn(xi0, (float)P.n_lights), P.n_lights - 1u);
    const float* L = P.lights[k];
    const F3 y = f3(__fmaf_rn(xi2, L[6], __fmaf_rn(xi1, L[3], L[0])),
                    __fmaf_rn(xi2, L[7], __fmaf_rn(xi1, L[4], L[1])),
                    __fmaf_rn(xi2, L[8], __fmaf_rn(xi1, L[5], L[2])));
    const F3 q = f3(__fsub_rn(y.x, x.x), __fsub_rn(y.y, x.y), __fsub_rn(y.z, x.z));
    const float d2 = dot3(q, q);
    if (!(d2 > 0.f)) return false;
    const float d = __fsqrt_rn(d2);
    const float inv = __frcp_rn(d);
    const F3 om = f3(__fmul_rn(q.x, inv), __fmul_rn(q.y, inv), __fmul_rn(q.z, inv));
    const F3 cr = f3(__fsub_rn(__fmul_rn(L[4], L[8]), __fmul_rn(L[5], L[7])),
                     __fsub_rn(__fmul_rn(L[5], L[6]), __fmul_rn(L[3], L[8])),
                     __fsub_rn(__fmul_rn(L[3], L[7]), __fmul_rn(L[4], L[6])));
    const float A = __fsqrt_rn(dot3(cr, cr));
    if (!(A > 0.f)) return false;
    const float cx = dot3(nx, om);
    const float cl = -__fdiv_rn(dot3(cr, om), A);
    if (!(cx > 0.f) || !(cl > 0.f)) return false;
    const float g = __fdiv_rn(__fmul_rn(__fmul_rn(__fmul_rn(cx, cl), A), (float)P.n_lights), d2);
    *w = f3(__fmul_rn(L[9], g), __fmul_rn(L[10], g), __fmul_rn(L[11], g));
    *dir = om;
    *dist = d;
    return true;
}

// Pinhole ray through (x + xi1, y + xi2) of view V (unit direction).
__device__ __forceinline__ F3 camera_dir(const ViewDev& V, uint32_t x, uint32_t y, float xi1, float xi2) {
    const float px = __fadd_rn((float)x, xi1);
    const float py = __fadd_rn((float)y, xi2);
    const float sx = __fmaf_rn(px, V.sxs, V.sx0);
    const float sy = __fmaf_rn(py, V.sys, V.sy0);
    return normalize3(f3(__fmaf_rn(sx, V.r[0], __fmaf_rn(sy, V.u[0], V.f[0])),
                         __fmaf_rn(sx, V.r[1], __fmaf_rn(sy, V.u[1], V.f[1])),
                         __fmaf_rn(sx, V.r[2], __fmaf_rn(sy, V.u[2], V.f[2]))));
}

// Cosine-weighted direction about n: Malley's disk-to-hemisphere lift in the
// orthonormal basis of Duff et al. (JCGT 2017).
__device__ __forceinline__ F3 sample_cosine(F3 n, float xi1, float xi2) {
    const float r = __fsqrt_rn(xi1);
    float sp, cp;
    sincospif(__fmul_rn(2.0f, xi2), &sp, &cp);
    const float lx = __fmul_rn(r, cp), ly = __fmul_rn(r, sp);
    const float lz = __fsqrt_rn(fmaxf(0.0f, __fsub_rn(1.0f, xi1)));
    const float sign = copysignf(1.0f, n.z);
    const float a = __fdiv_rn(-1.0f, __fadd_rn(sign, n.z));
    const float b = __fmul_rn(__fmul_rn(n.x, n.y), a);
    const F3 b1 = f3(__fadd_rn(1.0f, __fmul_rn(__fmul_rn(sign, __fmul_rn(n.x, n.x)), a)),
                     __fmul_rn(sign, b), -__fmul_rn(sign, n.x));
    const F3 b2 = f3(b, __fadd_rn(sign, __fmul_rn(__fmul_rn(n.y, n.y), a)), -n.y);
    return f3(__fmaf_rn(lx, b1.x, __fmaf_rn(ly, b2.x, __fmul_rn(lz, n.x))),
              __fmaf_rn(lx, b1.y, __fmaf_rn(ly, b2.y, __fmul_rn(lz, n.y))),
              __fmaf_rn(lx, b1.z, __fmaf_rn(ly, b2.z, __fmul_rn(lz, n.z))));
}

// Albedo row and unit geometric normal (cross of the quad's diagonals, moved
// to world space by the inverse transpose, faced against d) of a hit.
__device__ __forceinline__ F3 hit_normal(const DevScene& S, uint32_t inst, uint32_t slot, F3 d,
                                         uint32_t* quad_base) {
    const float4* ip = reinterpret_cast<const float4*>(S.inst + inst);
    const float4 m1 = __ldg(ip + 1), m2 = __ldg(ip + 2), m3 = __ldg(ip + 3);
    *quad_base = __float_as_uint(m3.z);
    const float4* qv = reinterpret_cast<const float4*>(S.quads + slot);
    const float4 qa = __ldg(qv), qb = __ldg(qv + 1), qc = __ldg(qv + 2);
    const F3 e1 = f3(__fsub_rn(qb.z, qa.x), __fsub_rn(qb.w, qa.y), __fsub_rn(qc.x, qa.z));  // v2 - v0
    const F3 e2 = f3(__fsub_rn(qc.y, qa.w), __fsub_rn(qc.z, qb.x), __fsub_rn(qc.w, qb.y));  // v3 - v1
    const F3 no = f3(__fsub_rn(__fmul_rn(e1.y, e2.z), __fmul_rn(e1.z, e2.y)),
                     __fsub_rn(__fmul_rn(e1.z, e2.x), __fmul_rn(e1.x, e2.z)),
                     __fsub_rn(__fmul_rn(e1.x, e2.y), __fmul_rn(e1.y, e2.x)));
    // n_world = W^T n_obj, W = world->object rows (w0 w1 w2 / w3 w4 w5 / w6 w7 w8)
    const float W0 = m1.x, W1 = m1.y, W2 = m1.z, W3 = m1.w, W4 = m2.x, W5 = m2.y, W6 = m2.z,
                W7 = m2.w, W8 = m3.x;
    F3 n = normalize3(f3(__fmaf_rn(W0, no.x, __fmaf_rn(W3, no.y, __fmul_rn(W6, no.z))),
                         __fmaf_rn(W1, no.x, __fmaf_rn(W4, no.y, __fmul_rn(W7, no.z))),
                         __fmaf_rn(W2, no.x, __fmaf_rn(W5, no.y, __fmul_rn(W8, no.z)))));
    if (dot3(n, d) > 0.f) n = f3(-n.x, -n.y, -n.z);
    return n;
}

__device__ __forceinline__ float maxabs3f(float a, float b, float c) {
    return fmaxf(fabsf(a), fmaxf(fabsf(b), fabsf(c)));
}

// Hit point o + t d and its self-intersection offset along n.
__device__ __forceinline__ F3 spawn_point(F3 o, F3 d, float t, F3 n) {
    const F3 hp = f3(__fmaf_rn(t, d.x, o.x), __fmaf_rn(t, d.y, o.y), __fmaf_rn(t, d.z, o.z));
    const float off = __fmaf_rn(1e-5f, maxabs3f(hp.x, hp.y, hp.z), 1e-4f);
    return f3(__fmaf_rn(off, n.x, hp.x), __fmaf_rn(off, n.y, hp.y), __fmaf_rn(off, n.z, hp.z));
}

// Add (g0, g1, g2) into grad[3*row ..]; lanes of a warp that hit the same row
// are summed first so only one of them issues the atomics.
__device__ __forceinline__ void grad_add(float* grad, uint32_t row, float g0, float g1, float g2) {
    const unsigned active = __activemask();
    const unsigned peers = __match_any_sync(active, row);
    const int lane = threadIdx.x & 31;
    if (peers == (1u << lane)) {
        atomicAdd(grad + 3 * (size_t)row, g0);
        atomicAdd(grad + 3 * (size_t)row + 1, g1);
        atomicAdd(grad + 3 * (size_t)row + 2, g2);
        return;
    }
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    unsigned m = peers;
    while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        s0 += __shfl_sync(peers, g0, j);
        s1 += __shfl_sync(peers, g1, j);
        s2 += __shfl_sync(peers, g2, j);
    }
    if (lane == __ffs(peers) - 1) {
        atomicAdd(grad + 3 * (size_t)row, s0);
        atomicAdd(grad + 3 * (size_t)row + 1, s1);
        atomicAdd(grad + 3 * (size_t)row + 2, s2);
    }
}

}  // namespace qrt

// Device-side traversal of the two-level quad BVH (qrt_layout.h).
//
// Top level: four-wide TLAS over instance world boxes.  At a TLAS leaf the ray
// is re-centred at t_e, where it passes closest to the object origin (never
// before tmin), formed exactly with error-free FP32 transformations, and moved
// into the instance's object space (the direction is not renormalised, so t
// is shared by both levels); the object's BLAS is traversed on the same stack
// with a parameter s = t - t_e.  Closest-hit stack entries keep each box's
// entry distance (64 bits: distance, reference) to cull entries beyond the
// best hit; any-hit rays never cull (tmax is fixed until the ray ends), so
// their entries are the 32-bit reference alone (half the local-memory
// traffic).
// When the stack drains back to the level where the instance was entered,
// the world ray is restored.  Leaves of a BLAS hold up to 16 quads stored
// contiguously.
//
// Precision design.  Box tests are made conservative by widening every
// dequantised box by delta, an absolute bound on the position error of the
// FP32 ray in the current space (2^-20 (|o| + R) at the top level, where the
// world ray is exact; 2^-22 (kappa + 2) (|o''| + R) in object space, where o''
// is the re-centred origin, R the object's radius and kappa the condition
// number of the transform), so a node is never culled
// that the exact ray enters.  The quad test is the watertight test of Woop,
// Benthin and Wald (JCGT 2013) applied to both triangles of the quad with the
// diagonal v0-v2 shared; an edge function within the same error bound of zero,
// or a hit distance within its error bound of either end of the interval,
// makes the decision uncertain, and only then the quad is re-tested in FP64
// from the world ray and the FP64 transform; two hits whose FP32 distances
// lie within their error bounds of each other are ordered by FP64 distances.
// Hit/miss decisions and the closest-hit choice therefore agree with exact
// arithmetic on the given FP32 ray except when a hit lies within FP64
// rounding of an edge or of another hit.
//
// Execution.  Persistent kernels run persistent_trace: each lane of a warp
// holds one ray; the warp tests inner nodes together, enters instances in
// groups, then lets every other lane enter its instance or test one leaf;
// finished lanes take the next ray at once (claimed one atomic per warp).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "qrt_layout.h"

namespace qrt {

constexpr float kInfF = __builtin_huge_valf();

struct Hit {
    float t;
    uint32_t inst, prim;
    float u, v;
    uint32_t slot;  // global quad slot of the hit (for shading)
};

// A world-space ray (origin, direction).  The traversal asks a caller-given
// functor for it where it is needed (instance entry, return to the TLAS, FP64
// re-tests) instead of keeping six floats live for the whole ray: kernels
// whose rays sit in device memory reload them from there.
struct WRay {
    float ox, oy, oz, dx, dy, dz;
};

// Ray in the current space, with everything the node and quad tests reuse.
struct RaySetup {
    float ox, oy, oz;     // origin
    float ix, iy, iz;     // reciprocal direction, |d| clamped away from 0
    float delta;
};

// Watertight shear of the current-space ray in affine form,
// X = V . rx - cx, Y = V . ry - cy, Z = V . rz - cz.  Built at the start of
// each leaf rather than kept for the whole ray: it is needed only there, and
// twelve fewer live registers per ray buy resident warps.
struct Shear {
    float rx0, rx1, rx2, cx;
    float ry0, ry1, ry2, cy;
    float rz0, rz1, rz2, cz;
    float eps_t;  // bound on the error of an FP32 hit distance (t units)
};

__device__ __forceinline__ float clamp_dir(float d) {
    return fabsf(d) > 1e-30f ? d : copysignf(1e-30f, d);
}

__device__ __forceinline__ void setup_boxes(RaySetup& r, float ox, float oy, float oz, float dx,
                                            float dy, float dz, float delta) {
    r.ox = ox;
    r.oy = oy;
    r.oz = oz;
    r.ix = __frcp_rn(clamp_dir(dx));
    r.iy = __frcp_rn(clamp_dir(dy));
    r.iz = __frcp_rn(clamp_dir(dz));
    r.delta = delta;
}

// (dx, dy, dz): the ray direction in the current space, the same value the
// box set-up was made from
__device__ __forceinline__ Shear make_shear(const RaySetup& r, float dx, float dy, float dz) {
    Shear sh;
    const float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
    // kz = dominant axis, (kx, ky) the next two in cyclic order; selects
    // instead of indexed arrays keep everything in registers
    const int kz = (ax > ay) ? ((ax > az) ? 0 : 2) : ((ay > az) ? 1 : 2);
    const float dkx = kz == 0 ? dy : (kz == 1 ? dz : dx);
    const float dky = kz == 0 ? dz : (kz == 1 ? dx : dy);
    const float dkz = kz == 0 ? dx : (kz == 1 ? dy : dz);
    const float okx = kz == 0 ? r.oy : (kz == 1 ? r.oz : r.ox);
    const float oky = kz == 0 ? r.oz : (kz == 1 ? r.ox : r.oy);
    const float okz = kz == 0 ? r.ox : (kz == 1 ? r.oy : r.oz);
    // one reciprocal; the products' extra rounding is covered by delta
    const float Sz = __frcp_rn(dkz);
    const float Sx = __fmul_rn(dkx, Sz), Sy = __fmul_rn(dky, Sz);
    // row X: +1 at kx, -Sx at kz; row Y: +1 at ky, -Sy at kz; row Z: Sz at kz
    sh.rx0 = kz == 0 ? -Sx : (kz == 2 ? 1.f : 0.f);
    sh.rx1 = kz == 1 ? -Sx : (kz == 0 ? 1.f : 0.f);
    sh.rx2 = kz == 2 ? -Sx : (kz == 1 ? 1.f : 0.f);
    sh.ry0 = kz == 0 ? -Sy : (kz == 1 ? 1.f : 0.f);
    sh.ry1 = kz == 1 ? -Sy : (kz == 2 ? 1.f : 0.f);
    sh.ry2 = kz == 2 ? -Sy : (kz == 0 ? 1.f : 0.f);
    sh.rz0 = kz == 0 ? Sz : 0.f;
    sh.rz1 = kz == 1 ? Sz : 0.f;
    sh.rz2 = kz == 2 ? Sz : 0.f;
    sh.cx = __fmaf_rn(-Sx, okz, okx);
    sh.cy = __fmaf_rn(-Sy, okz, oky);
    sh.cz = __fmul_rn(Sz, okz);
    // a position error of delta moves the distance along the dominant axis
    // by delta |Sz|; twice that bounds the FP32 hit distance's error
    sh.eps_t = 2.0f * __fmul_rn(r.delta, fabsf(Sz));
    return sh;
}

__device__ __forceinline__ float maxabs3(float a, float b, float c) {
    return fmaxf(fabsf(a), fmaxf(fabsf(b), fabsf(c)));
}

// --------------------------------------------------------------------------
// Node fetch: 64 bytes as four 128-bit or two 256-bit read-only loads.  The
// loads do not allocate in L1: with 32 or more warps per SM the per-ray
// local memory (spilled values and traversal stacks) needs L1, and node
// lines, which are seldom reused by the same SM soon enough, would only
// evict it (the mid frame measured 657 -> 674 Mrays/s with the hint, 678
// with quads read the same way; L2 still caches both).
// --------------------------------------------------------------------------
__device__ __forceinline__ uint4 ld_nc_na(const void* p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ float4 ld_nc_na_f4(const void* p) {
    const uint4 v = ld_nc_na(p);
    return make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z),
                       __uint_as_float(v.w));
}

template <int FETCH>
__device__ __forceinline__ void load_node(const QNode* n, uint4& a, uint4& b, uint4& c, uint4& d) {
    if constexpr (FETCH == 32) {
        asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y),
                       "=r"(b.z), "=r"(b.w)
                     : "l"(n));
        asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(c.x), "=r"(c.y), "=r"(c.z), "=r"(c.w), "=r"(d.x), "=r"(d.y),
                       "=r"(d.z), "=r"(d.w)
                     : "l"(reinterpret_cast<const char*>(n) + 32));
    } else {
        const uint4* p = reinterpret_cast<const uint4*>(n);
        a = ld_nc_na(p);
        b = ld_nc_na(p + 1);
        c = ld_nc_na(p + 2);
        d = ld_nc_na(p + 3);
    }
}

// Byte i of w as a float, exactly: the byte is placed in the mantissa of
// 2^23 with one byte permute and 2^23 is subtracted (full-rate integer and
// FP32 instructions instead of an integer-to-float conversion).
__device__ __forceinline__ float byte_f(uint32_t w, int i) {
    return __fsub_rn(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | (uint32_t)i)), 8388608.0f);
}

__device__ __forceinline__ float exp2i(int e) { return __int_as_float((e + 127) << 23); }

// Tests the four children of a node; writes entry distances (inf = culled)
// and references, sorted nearest first (SORT) or in slot order (any-hit
// rays, which need no order).  Returns the number of hits.
template <int FETCH, bool SORT = true>
__device__ __forceinline__ int node_children(const QNode* node, const RaySetup& r, float tmin,
                                             float tmax, float t[4], uint32_t ref[4]) {
    uint4 A, B, C, D;
    load_node<FETCH>(node, A, B, C, D);
    const float nox = __uint_as_float(A.x), noy = __uint_as_float(A.y), noz = __uint_as_float(A.z);
    const int ex = (int)(int8_t)(A.w & 0xFF), ey = (int)(int8_t)((A.w >> 8) & 0xFF),
              ez = (int)(int8_t)((A.w >> 16) & 0xFF);
    const float ax = __fmul_rn(exp2i(ex), r.ix), ay = __fmul_rn(exp2i(ey), r.iy),
                az = __fmul_rn(exp2i(ez), r.iz);
    // o * inv and the widening delta * |inv| are formed here, not kept in
    // RaySetup: at 64 registers kept values are spilled, and six multiplies
    // per node cost less than their local-memory round trips
    const float bx = __fmaf_rn(nox, r.ix, -__fmul_rn(r.ox, r.ix)),
                by = __fmaf_rn(noy, r.iy, -__fmul_rn(r.oy, r.iy)),
                bz = __fmaf_rn(noz, r.iz, -__fmul_rn(r.oz, r.iz));
    const float px = __fmul_rn(r.delta, fabsf(r.ix)), py = __fmul_rn(r.delta, fabsf(r.iy)),
                pz = __fmul_rn(r.delta, fabsf(r.iz));
    const float bnx = bx - px, bfx = bx + px;
    const float bny = by - py, bfy = by + py;
    const float bnz = bz - pz, bfz = bz + pz;
    // words: lo x,y,z = B.x, B.y, B.z ; hi x,y,z = B.w, C.x, C.y
    // near/far planes by the sign of the direction (compared here rather than
    // kept as bits: one register less per ray)
    const bool sx = r.ix < 0.f, sy = r.iy < 0.f, sz = r.iz < 0.f;
    const uint32_t nwx = sx ? B.w : B.x, fwx = sx ? B.x : B.w;
    const uint32_t nwy = sy ? C.x : B.y, fwy = sy ? B.y : C.x;
    const uint32_t nwz = sz ? C.y : B.z, fwz = sz ? B.z : C.y;
    const uint32_t meta = D.z;
    const uint32_t child[4] = {C.z, C.w, D.x, D.y};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float tnx = __fmaf_rn(byte_f(nwx, i), ax, bnx);
        const float tfx = __fmaf_rn(byte_f(fwx, i), ax, bfx);
        const float tny = __fmaf_rn(byte_f(nwy, i), ay, bny);
        const float tfy = __fmaf_rn(byte_f(fwy, i), ay, bfy);
        const float tnz = __fmaf_rn(byte_f(nwz, i), az, bnz);
        const float tfz = __fmaf_rn(byte_f(fwz, i), az, bfz);
        const float tn = fmaxf(fmaxf(tnx, tny), fmaxf(tnz, tmin));
        const float tf = fminf(fminf(tfx, tfy), fminf(tfz, tmax));
        const uint32_t m = (meta >> (8 * i)) & 0xFFu;
        const bool hit = (m != 0u) && (tn <= tf);
        t[i] = hit ? tn : kInfF;
        ref[i] = (m == kMetaInner) ? child[i] : (kRefLeaf | ((m - 1u) << 27) | child[i]);
    }
    if constexpr (!SORT)
        return (t[0] < kInfF) + (t[1] < kInfF) + (t[2] < kInfF) + (t[3] < kInfF);
    // sorting network on (t, ref); strict comparisons keep equal keys in order
#define QRT_CSWAP(i, j)                             \
    if (t[j] < t[i]) {                              \
        float tt = t[i];                            \
        t[i] = t[j];                                \
        t[j] = tt;                                  \
        uint32_t rr = ref[i];                       \
        ref[i] = ref[j];                            \
        ref[j] = rr;                                \
    }
    QRT_CSWAP(0, 1)
    QRT_CSWAP(2, 3)
    QRT_CSWAP(0, 2)
    QRT_CSWAP(1, 3)
    QRT_CSWAP(1, 2)
#undef QRT_CSWAP
    return (t[0] < kInfF) + (t[1] < kInfF) + (t[2] < kInfF) + (t[3] < kInfF);
}

// --------------------------------------------------------------------------
// Quad test
// --------------------------------------------------------------------------
struct SV {
    float X, Y, Z;
};

__device__ __forceinline__ SV shear(const Shear& sh, float x, float y, float z) {
    SV s;
    s.X = __fmaf_rn(x, sh.rx0, __fmaf_rn(y, sh.rx1, __fmaf_rn(z, sh.rx2, -sh.cx)));
    s.Y = __fmaf_rn(x, sh.ry0, __fmaf_rn(y, sh.ry1, __fmaf_rn(z, sh.ry2, -sh.cy)));
    s.Z = __fmaf_rn(x, sh.rz0, __fmaf_rn(y, sh.rz1, __fmaf_rn(z, sh.rz2, -sh.cz)));
    return s;
}

// 2D edge function; exactly antisymmetric: edge(P,Q) == -edge(Q,P).
__device__ __forceinline__ float edge(const SV& P, const SV& Q) {
    return __fsub_rn(__fmul_rn(P.X, Q.Y), __fmul_rn(P.Y, Q.X));
}

// 0 = certain miss, 1 = certain hit, 2 = uncertain.
__device__ __forceinline__ int classify(float e0, float e1, float e2, float B) {
    const bool p0 = e0 > B, p1 = e1 > B, p2 = e2 > B;
    const bool n0 = e0 < -B, n1 = e1 < -B, n2 = e2 < -B;
    if ((p0 || p1 || p2) && (n0 || n1 || n2)) return 0;
    if ((p0 && p1 && p2) || (n0 && n1 && n2)) return 1;
    return 2;
}

// Exact-enough re-test in FP64: object ray from the world ray and the
// instance's FP64 world->object matrix, then the watertight test with FP64
// arithmetic.  Returns 1 on a hit with t > tmin (world t written, with
// quad-space u, v).
static __device__ __noinline__ int quad_test64(const InstDev* ip, const InstDev64* ip64, float wox,
                                               float woy, float woz, float wdx, float wdy, float wdz,
                                               const float* v, float tmin, double* t_out,
                                               float* u_out, float* v_out) {
    double o[3], d[3];
    const double e[3] = {(double)wox - (double)ip->c[0], (double)woy - (double)ip->c[1],
                         (double)woz - (double)ip->c[2]};
    const double wd[3] = {wdx, wdy, wdz};
    const double* w = ip64->w;
    for (int r = 0; r < 3; ++r) {
        o[r] = w[3 * r] * e[0] + w[3 * r + 1] * e[1] + w[3 * r + 2] * e[2];
        d[r] = w[3 * r] * wd[0] + w[3 * r + 1] * wd[1] + w[3 * r + 2] * wd[2];
    }
    int kz = (fabs(d[0]) > fabs(d[1])) ? ((fabs(d[0]) > fabs(d[2])) ? 0 : 2)
                                       : ((fabs(d[1]) > fabs(d[2])) ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    const double Sx = d[kx] / d[kz], Sy = d[ky] / d[kz], Sz = 1.0 / d[kz];
    double X[4], Y[4], Z[4];
    for (int k = 0; k < 4; ++k) {
        double P[3] = {(double)v[3 * k] - o[0], (double)v[3 * k + 1] - o[1],
                       (double)v[3 * k + 2] - o[2]};
        X[k] = P[kx] - Sx * P[kz];
        Y[k] = P[ky] - Sy * P[kz];
        Z[k] = Sz * P[kz];
    }
    auto E = [&](int p, int q) { return X[p] * Y[q] - Y[p] * X[q]; };
    const double e21 = E(2, 1), e02 = E(0, 2), e10 = E(1, 0), e32 = E(3, 2), e03 = E(0, 3);
    int hit = 0;
    double best = INFINITY;
    float bu = 0.f, bv = 0.f;
    // triangle 0: (v0, v1, v2) with weights (e21, e02, e10)
    {
        const double U = e21, V = e02, W = e10;
        if (((U >= 0 && V >= 0 && W >= 0) || (U <= 0 && V <= 0 && W <= 0))) {
            const double det = U + V + W;
            if (det != 0.0) {
                const double tt = (U * Z[0] + V * Z[1] + W * Z[2]) / det;
                if (tt > (double)tmin && tt < best) {
                    best = tt;
                    hit = 1;
                    bu = (float)((V + W) / det);
                    bv = (float)(W / det);
                }
            }
        }
    }
    // triangle 1: (v0, v2, v3) with weights (e32, e03, -e02)
    {
        const double U = e32, V = e03, W = -e02;
        if (((U >= 0 && V >= 0 && W >= 0) || (U <= 0 && V <= 0 && W <= 0))) {
            const double det = U + V + W;
            if (det != 0.0) {
                const double tt = (U * Z[0] + V * Z[2] + W * Z[3]) / det;
                if (tt > (double)tmin && tt < best) {
                    best = tt;
                    hit = 1;
                    bu = (float)(V / det);
                    bv = (float)((V + W) / det);
                }
            }
        }
    }
    *t_out = best;
    *u_out = bu;
    *v_out = bv;
    return hit;
}

// FP32 test of one quad; returns 1 on a hit with tmin < t (t, u, v written);
// may defer to quad_test64.
// FP32 test of one quad in the object-space parameter s (smin < s < smax).
// A quad whose hit/miss decision is uncertain -- an edge function within its
// error band of zero, or the hit distance within eps_t of either end of the
// interval -- is re-tested by quad_test64, which returns the world t
// (*t64_out, *exact64 = 1).  Returns 1 on a hit.
template <class World>
__device__ __forceinline__ int quad_test(const RaySetup& r, const Shear& sh, const QuadDev* q,
                                         const InstDev* ip, const InstDev64* ip64,
                                         const World& world, float smin, float smax,
                                         float tmin, float* t_out, double* t64_out, float* u_out,
                                         float* v_out, int* exact64, uint32_t* n_fallback) {
    const float4* p = reinterpret_cast<const float4*>(q);
    // quads are read once per test: no L1 allocation, as for the nodes
    const float4 a = ld_nc_na_f4(p), b = ld_nc_na_f4(p + 1), c = ld_nc_na_f4(p + 2);
    const SV s0 = shear(sh, a.x, a.y, a.z);
    const SV s1 = shear(sh, a.w, b.x, b.y);
    const SV s2 = shear(sh, b.z, b.w, c.x);
    const SV s3 = shear(sh, c.y, c.z, c.w);
    const float e21 = edge(s2, s1), e02 = edge(s0, s2), e10 = edge(s1, s0);
    const float e32 = edge(s3, s2), e03 = edge(s0, s3);
    // one error band for the whole quad: covers delta-perturbed vertices and
    // the rounding of the edge products
    const float M = fmaxf(fmaxf(fmaxf(fabsf(s0.X), fabsf(s0.Y)), fmaxf(fabsf(s1.X), fabsf(s1.Y))),
                          fmaxf(fmaxf(fabsf(s2.X), fabsf(s2.Y)), fmaxf(fabsf(s3.X), fabsf(s3.Y))));
    const float B = __fmaf_rn(4.0f * r.delta, M, 4.76837158e-07f * M * M);  // 2^-21 M^2
    const int c0 = classify(e21, e02, e10, B);
    const int c1 = classify(e32, e03, -e02, B);
    if (c0 == 0 && c1 == 0) return 0;
    bool uncertain = c0 == 2 || c1 == 2;
    float best = kInfF;
    int hit = 0;
    if (!uncertain) {
        if (c0 == 1) {
            const float det = e21 + e02 + e10;
            const float T = __fmaf_rn(e21, s0.Z, __fmaf_rn(e02, s1.Z, __fmul_rn(e10, s2.Z)));
            const float tt = __fdiv_rn(T, det);
            if (tt > smin) {
                best = tt;
                hit = 1;
                *u_out = __fdiv_rn(e02 + e10, det);
                *v_out = __fdiv_rn(e10, det);
            }
            uncertain |= fabsf(tt - smin) <= sh.eps_t || fabsf(tt - smax) <= sh.eps_t;
        }
        if (c1 == 1) {
            const float det = e32 + e03 - e02;
            const float T = __fmaf_rn(e32, s0.Z, __fmaf_rn(e03, s2.Z, __fmul_rn(-e02, s3.Z)));
            const float tt = __fdiv_rn(T, det);
            if (tt > smin && tt < best) {
                best = tt;
                hit = 1;
                *u_out = __fdiv_rn(e03, det);
                *v_out = __fdiv_rn(e03 - e02, det);
            }
            uncertain |= fabsf(tt - smin) <= sh.eps_t || fabsf(tt - smax) <= sh.eps_t;
        }
    }
    if (uncertain) {
        ++*n_fallback;
        double t64;
        float vv[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
        const WRay w = world();
        if (!quad_test64(ip, ip64, w.ox, w.oy, w.oz, w.dx, w.dy, w.dz, vv, tmin, &t64, u_out, v_out))
            return 0;
        *t_out = (float)t64;
        *t64_out = t64;
        *exact64 = 1;
        return 1;
    }
    *exact64 = 0;
    *t_out = best;
    return hit;
}

// Exact (FP64) hit distance of quad `slot` of instance `inst` for the world
// ray, or +inf if the FP64 test misses it.
static __device__ __noinline__ double exact_t(const DevScene& S, uint32_t inst, uint32_t slot,
                                              float wox, float woy, float woz, float wdx, float wdy,
                                              float wdz, float tmin) {
    const float* v = S.quads[slot].v;
    float vv[12];
    for (int k = 0; k < 12; ++k) vv[k] = v[k];
    double t64;
    float u, w;
    if (!quad_test64(S.inst + inst, S.inst64 + inst, wox, woy, woz, wdx, wdy, wdz, vv, tmin, &t64, &u, &w))
        return __longlong_as_double(0x7ff0000000000000ll);
    return t64;
}

// --------------------------------------------------------------------------
// Two-level traversal
// --------------------------------------------------------------------------
struct TraceStats {
    uint32_t nodes;      // inner nodes visited
    uint32_t quads;      // quads tested
    uint32_t insts;      // instances entered
    uint32_t fallbacks;  // FP64 re-tests
    uint32_t rays;       // rays traced
    uint32_t verts;      // path vertices shaded (closest hits of the path tracer)
};

// Adds a thread's counters into stats[0..5] (rays, nodes, quads, instances,
// FP64 re-tests, shaded vertices), one atomic per warp and counter.  Call
// from converged code.
__device__ __forceinline__ void add_stats(unsigned long long* stats, const TraceStats& st) {
    uint32_t v[6] = {st.rays, st.nodes, st.quads, st.insts, st.fallbacks, st.verts};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        uint32_t x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(stats + k, (unsigned long long)x);
    }
}

// Resumable two-level traversal of one world ray.  init() sets the ray up;
// each step() processes the current node, leaf or instance entry and pops the
// next stack entry, returning false once the ray is finished (or stopped by
// an error); trace_ray runs it to the end.  The persistent kernels instead
// drive the warp-synchronous phase methods below from persistent_trace and
// refill finished lanes, so no lane waits for the slowest ray of its warp.
// The world ray itself is not kept: the callers' world() functors supply it.
// UV = false drops the hit's quad-space (u, v) (left 0): closest-hit rays
// whose consumer needs no (u, v) do not carry two more values through the
// traversal nor divide for them at every closer hit.
template <bool ANY, int STACK, int FETCH, bool UV = true>
struct Traversal {
    float tmin, tmax;
    float te;  // object-space parameter offset: t = s + te
    RaySetup r;
    // any-hit rays never cull by distance (tmax stays put until the ray
    // ends), so their entries hold the reference alone
    std::conditional_t<ANY, uint32_t, uint64_t> stack[STACK];
    int sp, inst_sp;
    bool have;
    // at the top level (no instance entered): inst_sp < 0
    __device__ __forceinline__ bool top() const { return inst_sp < 0; }
    uint32_t node_base, cur_inst, cur;
    uint32_t err;     // device error bits; init leaves them, the kernel resets them
    uint32_t budget;  // inner-node tests left before the step limit
    float h_eps;     // error bound of h.t (0 if exact)
    uint32_t pleaf;  // postponed BLAS leaf reference (0 = none)
    Hit h;

    // Pushes the hit children other than the one visited next and makes that
    // one current (nh > 0).  Closest hit: children sorted nearest first, the
    // nearest visited next, the others pushed farthest first with their entry
    // distances.  Any hit: children in slot order (the answer does not
    // depend on the order, and an unoccluded ray visits every child anyway),
    // the first hit visited next.
    __device__ __forceinline__ void push_children(int nh, const float t[4], const uint32_t ref[4]) {
        if constexpr (ANY) {
            const bool h0 = t[0] < kInfF, h1 = t[1] < kInfF, h2 = t[2] < kInfF;
            const int first = h0 ? 0 : (h1 ? 1 : (h2 ? 2 : 3));
#pragma unroll
            for (int k = 3; k >= 0; --k)
                if (t[k] < kInfF && k != first) stack[sp++] = ref[k];
            cur = h0 ? ref[0] : (h1 ? ref[1] : (h2 ? ref[2] : ref[3]));
        } else {
#pragma unroll
            for (int k = 3; k >= 1; --k)
                if (k < nh) stack[sp++] = ((uint64_t)__float_as_uint(t[k]) << 32) | ref[k];
            cur = ref[0];
        }
    }

    __device__ __forceinline__ void init(const DevScene& S, float ox, float oy, float oz, float dx,
                                         float dy, float dz, float t0, float t1, uint32_t msteps,
                                         TraceStats& st) {
        tmin = t0;
        tmax = t1;
        h.t = t1;
        h.inst = 0xFFFFFFFFu;
        h.prim = 0xFFFFFFFFu;
        h.u = h.v = 0.f;
        h.slot = 0;
        ++st.rays;
        sp = 0;
        inst_sp = -1;
        node_base = S.tlas_base;
        cur_inst = 0;
        te = 0.f;
        cur = 0;  // TLAS root, an inner reference
        h_eps = 0.f;
        have = S.n_inst > 0;
        budget = msteps;
        pleaf = 0;
        setup_world(S, WRay{ox, oy, oz, dx, dy, dz});
    }

    // The world ray's box-test setup, widened by 2^-20 (|o| + R_top): the
    // world ray is exact, so this covers only the rounding of the slab
    // arithmetic at the top level.  Recomputed on every return to the TLAS
    // rather than kept live: at 64 registers that shrinks the closest-hit
    // kernel's spill stores from 500 to 384 bytes per thread.
    __device__ __forceinline__ void setup_world(const DevScene& S, const WRay& w) {
        setup_boxes(r, w.ox, w.oy, w.oz, w.dx, w.dy, w.dz,
                    9.5367431640625e-07f * (maxabs3(w.ox, w.oy, w.oz) + S.R_top));
    }

    // far end of the interval in the current space (object space: s units,
    // widened by the rounding of h.t - te)
    __device__ __forceinline__ float limit() const {
        return top() ? h.t
                   : __fadd_rn(__fsub_rn(h.t, te), 1.9073486328125e-06f * (fabsf(h.t) + fabsf(te)));
    }

    template <class World>
    __device__ __forceinline__ bool step(const DevScene& S, TraceStats& st, const World& world) {
        if (have) {
            if (!(cur & kRefLeaf)) {
                if (budget == 0) {
                    err |= kErrStepLimit;
                    return false;
                }
                --budget;
                ++st.nodes;
                float t[4];
                uint32_t ref[4];
                const float lo = top() ? tmin : __fsub_rn(tmin, te);
                const int nh = node_children<FETCH, !ANY>(S.nodes + node_base + cur, r, lo, limit(), t, ref);
                if (nh == 0) {
                    have = false;
                } else {
                    if (sp + nh - 1 > STACK) {
                        err |= kErrStackOverflow;
                        return false;
                    }
                    push_children(nh, t, ref);
                    return true;
                }
            } else if (top()) {
                enter_instance(S, st, world);
                return true;
            } else {
                if (leaf(S, st, world)) return false;  // any hit found
                have = false;
            }
        }
        // pop
        if (!top() && sp == inst_sp) {
            inst_sp = -1;
            node_base = S.tlas_base;
            te = 0.f;
            setup_world(S, world());
        }
        if (sp == 0) return false;
        const uint64_t e = stack[--sp];
        const float tn = ANY ? tmin : __uint_as_float((uint32_t)(e >> 32));
        if (ANY || tn <= limit()) {
            cur = (uint32_t)e;
            have = true;
        }
        return true;
    }

    // ---- warp-synchronous phases (used by the persistent kernels) --------
    // A lane is in exactly one of: an inner node to test (wants_inner), a TLAS
    // leaf to enter (at_instance), a BLAS leaf to test (at_leaf: postponed or
    // current), or finished.

    __device__ __forceinline__ bool wants_inner() const { return have && !(cur & kRefLeaf); }
    __device__ __forceinline__ bool at_instance() const { return have && (cur & kRefLeaf) && top(); }
    __device__ __forceinline__ bool at_leaf() const {
        return pleaf != 0 || (have && (cur & kRefLeaf) && !top());
    }
    __device__ __forceinline__ bool finished() const { return !have && pleaf == 0; }

    __device__ __forceinline__ void stop(uint32_t e) {
        err |= e;
        have = false;
        pleaf = 0;
        sp = 0;
    }

    // Pops until cur holds an entry, the stack is empty, or the instance
    // boundary is reached while a leaf of this instance is still postponed.
    // BLAS leaves met on the way are postponed (one at a time) so that the
    // lane keeps traversing inner nodes with the rest of its warp.
    template <class World>
    __device__ __forceinline__ void advance(const DevScene& S, const World& world) {
        for (;;) {
            if (have) {
                if (pleaf == 0 && !top() && (cur & kRefLeaf)) {
                    pleaf = cur;
                    have = false;
                } else {
                    return;
                }
            }
            if (!top() && sp == inst_sp) {
                if (pleaf) return;
                inst_sp = -1;
                node_base = S.tlas_base;
                te = 0.f;
                setup_world(S, world());
            }
            if (sp == 0) return;
            const uint64_t e = stack[--sp];
            const float tn = ANY ? tmin : __uint_as_float((uint32_t)(e >> 32));
            if (ANY || tn <= limit()) {
                cur = (uint32_t)e;
                have = true;
            }
        }
    }

    // Tests the inner node cur and moves on (precondition: wants_inner()).
    template <class World>
    __device__ __forceinline__ void inner_step(const DevScene& S, TraceStats& st, int cap,
                                               const World& world) {
        if (budget == 0) {
            stop(kErrStepLimit);
            return;
        }
        --budget;
        ++st.nodes;
        float t[4];
        uint32_t ref[4];
        const float lo = top() ? tmin : __fsub_rn(tmin, te);
        const int nh = node_children<FETCH, !ANY>(S.nodes + node_base + cur, r, lo, limit(), t, ref);
        if (nh == 0) {
            have = false;
        } else {
            if (sp + nh - 1 > cap) {
                stop(kErrStackOverflow);
                return;
            }
            push_children(nh, t, ref);
        }
        advance(S, world);
    }

    // Tests one BLAS leaf (the postponed one first); returns true when an
    // any-hit query is answered (precondition: at_leaf()).
    template <class World>
    __device__ __forceinline__ bool leaf_step(const DevScene& S, TraceStats& st, const World& world) {
        if (pleaf) {
            const uint32_t keep = cur;
            cur = pleaf;
            pleaf = 0;
            const bool done = leaf(S, st, world);
            cur = keep;
            if (done) return true;
        } else {
            if (leaf(S, st, world)) return true;
            have = false;
        }
        advance(S, world);
        return false;
    }

    // Enters the instance of the TLAS leaf cur (precondition: at_instance()).
    template <class World>
    __device__ __forceinline__ void instance_step(const DevScene& S, TraceStats& st,
                                                  const World& world) {
        enter_instance(S, st, world);
    }

    // Moves the ray into the instance's object space.  The world point
    // p = o + te d where the ray enters the instance's box and its offset
    // p - c from the object origin are formed exactly as float pairs
    // (two-product / two-sum), so the FP32 object-space origin W (p - c)
    // carries an error proportional to the object's size only; the BLAS then
    // works in s = t - te.
    template <class World>
    __device__ __forceinline__ void enter_instance(const DevScene& S, TraceStats& st,
                                                   const World& world) {
        cur_inst = cur & kRefIndexMask;
        const WRay w = world();
        const float wox = w.ox, woy = w.oy, woz = w.oz, wdx = w.dx, wdy = w.dy, wdz = w.dz;
        const float4* ip = reinterpret_cast<const float4*>(S.inst + cur_inst);
        const float4 m0 = __ldg(ip), m1 = __ldg(ip + 1), m2 = __ldg(ip + 2), m3 = __ldg(ip + 3);
        // m0 = (c, R); m1 = (w0 w1 w2 w3); m2 = (w4 w5 w6 w7); m3 = (w8, node_base, quad_base, kappa)
        // Re-centre where the ray passes closest to the object origin (never
        // before tmin), so the re-centred origin lies within the object's
        // reach; hits before that point have s < 0.  (Re-centring at the
        // instance box's entry distance instead needs that distance kept per
        // stack entry and per ray, and measured slower with more FP64
        // re-tests.)
        {
            const float cx = __fsub_rn(m0.x, wox), cy = __fsub_rn(m0.y, woy), cz = __fsub_rn(m0.z, woz);
            const float dd = __fmaf_rn(wdx, wdx, __fmaf_rn(wdy, wdy, __fmul_rn(wdz, wdz)));
            const float tc = __fdiv_rn(__fmaf_rn(cx, wdx, __fmaf_rn(cy, wdy, __fmul_rn(cz, wdz))), dd);
            te = (tc > tmin && tc < kInfF) ? tc : tmin;
        }
        float exl, eyl, ezl;
        const float ex = exact_offset(wox, wdx, te, m0.x, &exl);
        const float ey = exact_offset(woy, wdy, te, m0.y, &eyl);
        const float ez = exact_offset(woz, wdz, te, m0.z, &ezl);
        const float rox = __fmaf_rn(m1.x, ex, __fmaf_rn(m1.y, ey, __fmaf_rn(m1.z, ez,
                              __fmaf_rn(m1.x, exl, __fmaf_rn(m1.y, eyl, __fmul_rn(m1.z, ezl))))));
        const float roy = __fmaf_rn(m1.w, ex, __fmaf_rn(m2.x, ey, __fmaf_rn(m2.y, ez,
                              __fmaf_rn(m1.w, exl, __fmaf_rn(m2.x, eyl, __fmul_rn(m2.y, ezl))))));
        const float roz = __fmaf_rn(m2.z, ex, __fmaf_rn(m2.w, ey, __fmaf_rn(m3.x, ez,
                              __fmaf_rn(m2.z, exl, __fmaf_rn(m2.w, eyl, __fmul_rn(m3.x, ezl))))));
        float fdx, fdy, fdz;
        object_dir(m1, m2, m3, wdx, wdy, wdz, fdx, fdy, fdz);
        node_base = __float_as_uint(m3.y);
        // 2^-22 (kappa + 2) (|o''| + R): rounding of W, of W (p - c), of W d and
        // of the slab and shear arithmetic, with a factor-two margin
        const float delta = __fmul_rn(2.384185791015625e-07f * (m3.w + 2.0f),
                                      maxabs3(rox, roy, roz) + m0.w);
        setup_boxes(r, rox, roy, roz, fdx, fdy, fdz, delta);
        inst_sp = sp;
        ++st.insts;
        cur = 0;
    }

    // W d: the world direction in the instance's object space (m1..m3 hold
    // W row by row).  Recomputed at each leaf rather than kept per ray.
    static __device__ __forceinline__ void object_dir(const float4& m1, const float4& m2,
                                                      const float4& m3, float wdx, float wdy,
                                                      float wdz, float& fdx, float& fdy, float& fdz) {
        fdx = __fmaf_rn(m1.x, wdx, __fmaf_rn(m1.y, wdy, __fmul_rn(m1.z, wdz)));
        fdy = __fmaf_rn(m1.w, wdx, __fmaf_rn(m2.x, wdy, __fmul_rn(m2.y, wdz)));
        fdz = __fmaf_rn(m2.z, wdx, __fmaf_rn(m2.w, wdy, __fmul_rn(m3.x, wdz)));
    }

    // (o + te d) - c per axis as a float pair hi + *lo, exact up to the
    // rounding of the small correction terms.
    static __device__ __forceinline__ float exact_offset(float o, float d, float te, float c, float* lo) {
        const float q = __fmul_rn(te, d);
        const float rho = __fmaf_rn(te, d, -q);       // te d = q + rho exactly
        const float s = __fadd_rn(o, q);
        const float bb = __fsub_rn(s, o);
        const float e1 = __fadd_rn(__fsub_rn(o, __fsub_rn(s, bb)), __fsub_rn(q, bb));  // o + q = s + e1
        const float hi = __fsub_rn(s, c);
        const float b2 = __fsub_rn(hi, s);
        const float e2 = __fadd_rn(__fsub_rn(s, __fsub_rn(hi, b2)), __fsub_rn(-c, b2));  // s - c = hi + e2
        *lo = __fadd_rn(e2, __fadd_rn(e1, rho));
        return hi;
    }

    // The closest hit's original quad index, looked up from its slot once the
    // ray has ended (ties during traversal read it on demand), so it is not
    // live through the traversal.  Any-hit results carry no quad index.
    __device__ __forceinline__ void resolve_prim(const DevScene& S) {
        if constexpr (!ANY) h.prim = h.inst == 0xFFFFFFFFu ? 0xFFFFFFFFu : __ldg(S.prim + h.slot);
    }

    // Tests the quads of the current BLAS leaf; returns true when an any-hit
    // query is answered.  Two candidates whose FP32 distances are within
    // their error bounds of each other are ordered by their FP64 distances.
    template <class World>
    __device__ __forceinline__ bool leaf(const DevScene& S, TraceStats& st, const World& world) {
        Shear sh;
        {
            const float4* mp = reinterpret_cast<const float4*>(S.inst + cur_inst);
            const float4 m1 = __ldg(mp + 1), m2 = __ldg(mp + 2), m3 = __ldg(mp + 3);
            const WRay w = world();
            float dx, dy, dz;
            object_dir(m1, m2, m3, w.dx, w.dy, w.dz, dx, dy, dz);
            sh = make_shear(r, dx, dy, dz);
        }
        const uint32_t first = cur & kRefIndexMask;
        const uint32_t cnt = ((cur >> 27) & 0xFu) + 1u;
        const float smin = __fsub_rn(tmin, te);
        const float smax = __fsub_rn(tmax, te);
        const InstDev* ip = S.inst + cur_inst;
        const InstDev64* ip64 = S.inst64 + cur_inst;
        // read here (an L1 hit after the instance entry) rather than kept
        // live for the whole BLAS traversal
        const uint32_t quad_base = __ldg(&ip->quad_base);
        for (uint32_t k = 0; k < cnt; ++k) {
            const uint32_t slot = quad_base + first + k;
            float tt, uu, vv;
            double t64;
            int ex64;
            ++st.quads;
            if (!quad_test(r, sh, S.quads + slot, ip, ip64, world, smin, smax, tmin, &tt, &t64, &uu,
                           &vv, &ex64, &st.fallbacks))
                continue;
            if (!ex64) tt = __fadd_rn(tt, te);
            if (!(tt > tmin && tt < tmax)) continue;
            if (ANY) {
                h.t = tt;
                h.inst = cur_inst;
                h.slot = slot;
                return true;
            }
            const float eps = fmaxf(sh.eps_t, h_eps);
            if (h.inst != 0xFFFFFFFFu && fabsf(tt - h.t) <= eps &&
                !(h.slot == slot && h.inst == cur_inst)) {
                // near tie with the current best: decide on FP64 distances
                ++st.fallbacks;
                const WRay w = world();
                const double tb = exact_t(S, h.inst, h.slot, w.ox, w.oy, w.oz, w.dx, w.dy, w.dz, tmin);
                const double tc =
                    ex64 ? t64 : exact_t(S, cur_inst, slot, w.ox, w.oy, w.oz, w.dx, w.dy, w.dz, tmin);
                const bool better =
                    tc < tb || (tc == tb && (cur_inst < h.inst ||
                                             (cur_inst == h.inst &&
                                              __ldg(S.prim + slot) < __ldg(S.prim + h.slot))));
                if (better && tc < (double)tmax) {
                    h.t = (float)tc;
                    h.inst = cur_inst;
                    if constexpr (UV) {
                        h.u = uu;
                        h.v = vv;
                    }
                    h.slot = slot;
                    h_eps = sh.eps_t;
                }
                continue;
            }
            if (tt < h.t) {
                h.t = tt;
                h.inst = cur_inst;
                if constexpr (UV) {
                    h.u = uu;
                    h.v = vv;
                }
                h.slot = slot;
                h_eps = ex64 ? 0.f : sh.eps_t;
            } else if (tt == h.t) {
                if (cur_inst < h.inst ||
                    (cur_inst == h.inst && __ldg(S.prim + slot) < __ldg(S.prim + h.slot))) {
                    h.inst = cur_inst;
                    if constexpr (UV) {
                        h.u = uu;
                        h.v = vv;
                    }
                    h.slot = slot;
                    h_eps = ex64 ? 0.f : sh.eps_t;
                }
            }
        }
        return false;
    }
};

// Persistent warp-synchronous traversal loop over work items [0, count)
// claimed from *cursor.  Each lane holds one ray; start(k) sets item k up in
// T (T.init), done() consumes the finished ray in T, world() gives the world
// ray of the lane's current item; a ray may use cap (<=
// STACK) stack entries, a launch-wide value passed down rather than kept per
// ray.  A lane claims `batch`
// items at a time; the idle lanes of a warp claim theirs with one atomic
// (warp-aggregated), so a launch costs about one atomic per warp and
// refill round instead of one per thread.  Per outer iteration
// the warp first tests inner nodes together (lanes that reach a BLAS leaf
// postpone it and keep traversing; lanes waiting at instances enter them in
// groups) until few lanes are left with an inner node, then lanes enter
// instances or test one leaf each.  Finished lanes refill
// immediately, so no lane waits for the slowest ray of its warp.
template <bool ANY, int STACK, int FETCH, bool UV, class Idx, class Start, class Done, class World>
__device__ __forceinline__ void persistent_trace(const DevScene& S, Traversal<ANY, STACK, FETCH, UV>& T,
                                                 TraceStats& st, Idx* cursor, Idx count,
                                                 uint32_t batch, int cap, Start start, Done done,
                                                 World world) {
    const unsigned FULL = 0xFFFFFFFFu;
    const unsigned lane = threadIdx.x & 31u;
    // [next, end) = this lane's claimed items not yet started; a claim that
    // lands at or past count leaves end == count, which ends the claiming
    bool busy = false;
    Idx next = 0, end = 0;
    for (;;) {
        const bool need = !busy && next >= end && end < count;
        const unsigned want = __ballot_sync(FULL, need);
        if (want) {
            const int leader = __ffs(want) - 1;
            Idx base = 0;
            if ((int)lane == leader) base = atomicAdd(cursor, (Idx)batch * (Idx)__popc(want));
            base = __shfl_sync(FULL, base, leader);
            if (need) {
                next = base + (Idx)batch * (Idx)__popc(want & ((1u << lane) - 1u));
                end = min(next + (Idx)batch, count);
            }
        }
        if (!busy && next < end) {
            start(next++);
            busy = true;
        }
        if (__all_sync(FULL, !busy)) break;
        for (;;) {
            // Once eight or more lanes wait at an instance (TLAS leaf), they
            // enter it together and go on with the inner nodes of its BLAS
            // in this phase, instead of idling until the next outer
            // iteration.  Each such step enters at least eight instances.
            const bool wt = busy && T.at_instance();
            const unsigned bt = __ballot_sync(FULL, wt);
            if (__popc(bt) >= 8) {
                if (wt) T.instance_step(S, st, world);
                continue;
            }
            const bool w = busy && T.wants_inner();
            const unsigned bw = __ballot_sync(FULL, w);
            if (!bw) break;
            // Leave the inner-node phase early once the lanes still in it are
            // at most half as many as the lanes waiting at an instance or a
            // leaf (or finished): those then move on together instead of
            // idling until the warp's longest run of inner nodes ends.
            // bo != 0 keeps a lane that the next phase moves on, so every
            // outer iteration makes progress.
            const unsigned bo = __ballot_sync(FULL, busy && !w);
            if (bo && 2 * __popc(bw) <= __popc(bo)) break;
            if (w) T.inner_step(S, st, cap, world);
        }
        if (busy) {
            if (T.at_instance()) {
                T.instance_step(S, st, world);
            } else if (T.at_leaf()) {
                if (T.leaf_step(S, st, world)) {
                    T.have = false;
                    T.pleaf = 0;
                }
            }
            if (T.finished() || (ANY && T.h.inst != 0xFFFFFFFFu)) {
                T.resolve_prim(S);
                done();
                busy = false;
            }
        }
    }
}

// Closest hit (ANY = false) or any hit (ANY = true) of the world ray, run to
// completion.  Returns device error bits (0 = fine); h holds the best hit
// found (inst = 0xFFFFFFFF if none).
template <bool ANY, int STACK, int FETCH>
__device__ __forceinline__ uint32_t trace_ray(const DevScene& S, float wox, float woy, float woz,
                                              float wdx, float wdy, float wdz, float tmin,
                                              float tmax, uint32_t max_steps, Hit& h,
                                              TraceStats& st) {
    Traversal<ANY, STACK, FETCH> T;
    T.err = 0;
    T.init(S, wox, woy, woz, wdx, wdy, wdz, tmin, tmax, max_steps, st);
    const auto world = [=] { return WRay{wox, woy, woz, wdx, wdy, wdz}; };
    while (T.step(S, st, world)) {
    }
    T.resolve_prim(S);
    h = T.h;
    return T.err;
}

}  // namespace qrt

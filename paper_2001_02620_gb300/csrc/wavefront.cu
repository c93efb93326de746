// Wavefront path tracer: the same paths as the single-kernel renderer in
// render.cu, split into stages so the ray-tracing kernels stay lean and every
// lane stays busy.
//
// Per chunk of at most C paths (chunk boundaries fall on pixel boundaries):
//   gen        camera ray of every path; closest-ray queue of depth 1
//   for depth i = 1..D:
//     trace    persistent closest-hit kernel over queue i; each lane takes the
//              next ray as soon as its own is finished
//     shade    misses add beta*env; hits fetch albedo and normal, queue a
//              shadow ray toward the sun (pending term beta*a/pi*E*cos),
//              multiply beta by a and queue the bounce ray for depth i+1
//     shadow   persistent any-hit kernel over the shadow queue; an
//              unoccluded ray adds its pending term to the path (on a second
//              stream, beside the trace of depth i+1, unless the render is
//              timed stage by stage; shade i+1 waits for it)
//   accumulate mean over each pixel's samples, summed in sample order
// The adjoint runs the chunk twice: a primal pass that leaves each path's
// radiance in Ltot, then a replay pass whose shade stage adds
// w * (Ltot - sun terms before vertex i) / a_i into the albedo gradient.
// The primal also records which of the path's shadow rays of depths 1..32
// were unoccluded (bit i-1 in the spare w lane of its radiance), so the
// replay adds those sun terms in its shade stage instead of tracing the
// shadow rays again.
// Radiance is accumulated in the same order as render.cu, so the two
// renderers give bit-identical images.
#include <algorithm>
#include <mutex>

#include "launch.h"
#include "shading.cuh"
#include "traverse.cuh"
#include "wavefront.h"

namespace qrt {

__device__ __forceinline__ int find_view_by_path(const WaveArgs& A, uint64_t g) {
    int lo = 0, hi = (int)A.n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (A.views[mid].path_begin <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_view_by_item(const WaveArgs& A, uint64_t item) {
    int lo = 0, hi = (int)A.n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (A.views[mid].item_begin <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Appends j to a queue; lanes of a warp share one atomic.
__device__ __forceinline__ void push(uint32_t* queue, uint32_t* count, uint32_t j) {
    const unsigned m = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(m));
    base = __shfl_sync(m, base, leader);
    queue[base + __popc(m & ((1u << lane) - 1u))] = j;
}

__global__ void __launch_bounds__(256) wave_gen(const __grid_constant__ WaveArgs A, uint64_t P0,
                                                uint32_t n) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) A.B.ctr[kCtrStride * 1 + kCtrClosest] = n;  // queue of depth 1 holds every path
    if (j >= n) return;
    const uint64_t g = P0 + j;
    const ViewDev& V = A.views[find_view_by_path(A, g)];
    const uint64_t local = g - V.path_begin;
    const uint64_t pix = local / V.spp;
    const uint32_t smp = V.sample_base + (uint32_t)(local - pix * V.spp);  // global sample index
    uint32_t x, y;
    const uint64_t gpix = view_pixel(V, pix, &x, &y);
    const uint4 xi = draw(A.P.seed, gpix, smp, 0);
    const F3 d = camera_dir(V, x, y, u01(xi.x), u01(xi.y));
    A.B.ray_o[j] = make_float4(V.eye[0], V.eye[1], V.eye[2], 0.f);
    A.B.ray_d[j] = make_float4(d.x, d.y, d.z, kInfF);
    A.B.beta[j] = make_float4(1.f, 1.f, 1.f, 0.f);
    A.B.L[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (A.P.n_lights) A.B.lpend[j].w = 0.f;
    A.B.meta[j] = make_uint2((uint32_t)(V.item_begin + pix), smp);
    A.B.q[1][j] = j;  // depth 1 uses queue 1 & 1
    if (A.cost_on) A.B.cost[j] = 0;
    if (A.P.path_log) {
        uint32_t* log = A.P.path_log + g * path_log_words(A.P.max_depth);
        for (uint32_t k = 0; k < 2 * A.P.max_depth; ++k) log[k] = 0xFFFFFFFFu;
        log[2 * A.P.max_depth] = log[2 * A.P.max_depth + 1] = 0u;
    }
    if (A.P.ray_log) {
        float* rl = ray_log_rec(A.P, g, 1);
        clear_ray_log(rl, A.P.max_depth);
        log_ray(rl, f3(V.eye[0], V.eye[1], V.eye[2]), d);
    }
}

// Persistent trace over a queue.  ANY = false: closest hit of ray_o/ray_d of
// each queued path into hit[].  ANY = true: shadow ray from sray_o toward the
// sun; an unoccluded ray adds pend[] into L[].  Rays use at most stack_cap
// stack entries.  Work counters are kept only in the STATS variant: in the
// others they are dead code, which saves a dozen registers per thread.
// UV: closest-hit rays keep the hit's (u, v) (per-face textures need them)
template <bool ANY, int FETCH, int OCC, bool STATS, bool UV>
__global__ void __maxnreg__(occupancy_regs(OCC)) wave_trace(const __grid_constant__ WaveArgs A, int depth,
                                                        int stack_cap) {
    const uint32_t* ctr = A.B.ctr + kCtrStride * depth;
    const uint32_t count = ANY ? ctr[kCtrShadow] : ctr[kCtrClosest];
    uint32_t* fetch = A.B.ctr + kCtrStride * depth + (ANY ? kCtrFetchShadow : kCtrFetchClosest);
    const uint32_t* queue = ANY ? A.B.qs : A.B.q[depth & 1];
    const uint32_t batch = A.batch;
    TraceStats st{0, 0, 0, 0, 0, 0};
    Traversal<ANY, kMaxStack, FETCH, UV> T;
    T.err = 0;  // accumulated over this thread's rays
    uint32_t j = 0;
    // any-hit entries of key-light shadow rays carry kLightRay
    auto start_ray = [&](uint32_t k) {
        j = queue[k];
        if (ANY) {
            const float4 o = A.B.sray_o[j & ~kLightRay];
            if (j & kLightRay) {
                const float4 ld = A.B.lray_d[j & ~kLightRay];
                T.init(A.S, o.x, o.y, o.z, ld.x, ld.y, ld.z, 0.f, ld.w, A.P.max_steps, st);
            } else {
                T.init(A.S, o.x, o.y, o.z, A.P.sun_l[0], A.P.sun_l[1], A.P.sun_l[2], 0.f, kInfF,
                       A.P.max_steps, st);
            }
        } else {
            // path rays span (0, inf) (the spawn point is offset off the
            // surface): constant bounds fold into the traversal instead of
            // occupying two registers per ray
            const float4 o = A.B.ray_o[j], d = A.B.ray_d[j];
            T.init(A.S, o.x, o.y, o.z, d.x, d.y, d.z, 0.f, kInfF, A.P.max_steps, st);
        }
    };
    auto finish_ray = [&]() {
        const uint32_t jj = j & ~kLightRay;
        if constexpr (STATS) {
            if (A.cost_on) atomicAdd(A.B.cost + jj, A.P.max_steps - T.budget);
        }
        if (ANY) {
            const bool light = j & kLightRay;
            if (T.h.inst == 0xFFFFFFFFu) {
                if (light) {
                    // the sun's shadow ray of the same vertex may add into L
                    // in this launch: flag the term, fold_light adds it later
                    A.B.lpend[jj].w = 1.f;
                } else {
                    const float4 p = A.B.pend[jj];
                    float4 l = A.B.L[jj];
                    l.x = __fadd_rn(l.x, p.x);
                    l.y = __fadd_rn(l.y, p.y);
                    l.z = __fadd_rn(l.z, p.z);
                    if (depth <= kVisDepths) l.w = __uint_as_float(__float_as_uint(l.w) | (1u << (depth - 1)));
                    A.B.L[jj] = l;
                }
            } else if (A.P.path_log && depth <= 16) {
                const uint64_t g = A.P0 + jj;
                A.P.path_log[g * path_log_words(A.P.max_depth) + 2 * A.P.max_depth + (light ? 1 : 0)] |=
                    2u << (2 * (depth - 1));
            }
        } else {
            A.B.hit[j] = make_uint4(__float_as_uint(T.h.t), T.h.inst, T.h.prim, T.h.slot);
            if constexpr (UV) A.B.hit_uv[j] = make_float2(T.h.u, T.h.v);
        }
    };
    // the world ray is read back from the queue buffers where the traversal
    // needs it, not kept live per lane
    auto world_ray = [&]() {
        if (ANY) {
            const float4 o = __ldg(A.B.sray_o + (j & ~kLightRay));
            if (j & kLightRay) {
                const float4 ld = __ldg(A.B.lray_d + (j & ~kLightRay));
                return WRay{o.x, o.y, o.z, ld.x, ld.y, ld.z};
            }
            return WRay{o.x, o.y, o.z, A.P.sun_l[0], A.P.sun_l[1], A.P.sun_l[2]};
        }
        const float4 o = __ldg(A.B.ray_o + j), d = __ldg(A.B.ray_d + j);
        return WRay{o.x, o.y, o.z, d.x, d.y, d.z};
    };
    persistent_trace<ANY, kMaxStack, FETCH>(A.S, T, st, fetch, count, batch, stack_cap, start_ray,
                                            finish_ray, world_ray);
    if (T.err) atomicOr(A.S.err, T.err);
    if constexpr (STATS) add_stats(A.stats + (ANY ? 6 : 0), st);
}

// Adds path j's key-light term of the previous vertex into its radiance if
// its shadow ray found the light (flag in lpend.w): after the sun's term of
// that vertex, as the single-kernel renderer adds them.
__device__ __forceinline__ void fold_light(const WaveBufs& B, uint32_t j) {
    const float4 p = B.lpend[j];
    if (p.w != 0.f) {
        float4 l = B.L[j];
        l.x = __fadd_rn(l.x, p.x);
        l.y = __fadd_rn(l.y, p.y);
        l.z = __fadd_rn(l.z, p.z);
        B.L[j] = l;
        B.lpend[j].w = 0.f;
    }
}

__global__ void __launch_bounds__(256) wave_fold(const __grid_constant__ WaveArgs A, uint32_t n) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) fold_light(A.B, j);
}

// Shade stage of depth i (1-based).  replay = false: primal; true: replay
// pass of the adjoint (gradient into A.grad, no env term, L holds the
// next-event terms gathered so far).  The diffuse albedo is the quad's
// albedo times its per-face texture at the hit (when textures are given);
// next-event estimation queues the sun's shadow ray and one key-light
// shadow ray (tagged kLightRay) with their pending terms.
__global__ void __launch_bounds__(256) wave_shade(const __grid_constant__ WaveArgs A, int depth,
                                                  int replay) {
    const uint32_t* ctr = A.B.ctr + kCtrStride * depth;
    const uint32_t n = ctr[kCtrClosest];
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t j = A.B.q[depth & 1][k];
    if (A.P.n_lights && depth > 1) fold_light(A.B, j);
    const uint4 hb = A.B.hit[j];
    const float t = __uint_as_float(hb.x);
    const uint32_t inst = hb.y, prim = hb.z, slot = hb.w;
    const uint32_t D = A.P.max_depth;
    const uint64_t g = A.P0 + j;
    uint32_t* log = A.P.path_log ? A.P.path_log + g * path_log_words(D) : nullptr;
    if (log) {
        log[2 * (depth - 1)] = inst;
        log[2 * (depth - 1) + 1] = prim;
    }
    float4 b = A.B.beta[j];
    if (inst == 0xFFFFFFFFu) {
        if (!replay) {
            float4 l = A.B.L[j];
            l.x = __fmaf_rn(b.x, A.P.env[0], l.x);
            l.y = __fmaf_rn(b.y, A.P.env[1], l.y);
            l.z = __fmaf_rn(b.z, A.P.env[2], l.z);
            A.B.L[j] = l;
        }
        return;
    }
    const float4 o4 = A.B.ray_o[j], d4 = A.B.ray_d[j];
    const F3 o = f3(o4.x, o4.y, o4.z), d = f3(d4.x, d4.y, d4.z);
    uint32_t qbase;
    const F3 nrm = hit_normal(A.S, inst, slot, d, &qbase);
    const uint32_t row = qbase + prim;
    const float q0 = __ldg(A.albedo + 3 * (size_t)row);
    const float q1 = __ldg(A.albedo + 3 * (size_t)row + 1);
    const float q2 = __ldg(A.albedo + 3 * (size_t)row + 2);
    float a0 = q0, a1 = q1, a2 = q2;  // diffuse albedo at the hit
    if (A.P.tex_res) {
        const float2 uv = A.B.hit_uv[j];
        const F3 tx = tex_lookup(A.P.tex, A.P.tex_res, row, uv.x, uv.y);
        a0 = __fmul_rn(q0, tx.x);
        a1 = __fmul_rn(q1, tx.y);
        a2 = __fmul_rn(q2, tx.z);
    }
    const F3 sp = spawn_point(o, d, t, nrm);
    float* rlog = A.P.ray_log ? ray_log_rec(A.P, g, depth) : nullptr;
    if (rlog) log_spawn(rlog, sp);
    const uint2 mt = A.B.meta[j];
    const ViewDev& V = A.views[find_view_by_item(A, mt.x)];
    uint32_t px, py;
    const uint64_t gpix = view_pixel(V, mt.x - V.item_begin, &px, &py);
    if (replay) {
        // d L / d q_i = (radiance leaving vertex i) / q_i per channel, q_i the
        // quad's albedo (the texture factor is a constant of the path)
        const float* di = V.dimage + 3 * (mt.x - V.item_begin);
        const float inv_spp = __frcp_rn((float)V.spp);
        const float w0 = __fmul_rn(__ldg(di), inv_spp), w1 = __fmul_rn(__ldg(di + 1), inv_spp),
                    w2 = __fmul_rn(__ldg(di + 2), inv_spp);
        const float4 lt = A.B.Ltot[j], s = A.B.L[j];
        const float g0 = q0 != 0.f ? __fdiv_rn(__fmul_rn(w0, __fsub_rn(lt.x, s.x)), q0) : 0.f;
        const float g1 = q1 != 0.f ? __fdiv_rn(__fmul_rn(w1, __fsub_rn(lt.y, s.y)), q1) : 0.f;
        const float g2 = q2 != 0.f ? __fdiv_rn(__fmul_rn(w2, __fsub_rn(lt.z, s.z)), q2) : 0.f;
        if (g0 != 0.f || g1 != 0.f || g2 != 0.f) grad_add(A.grad, row, g0, g1, g2);
    }
    if (A.P.sun_on) {
        const float cl = dot3(nrm, f3(A.P.sun_l[0], A.P.sun_l[1], A.P.sun_l[2]));
        if (cl > 0.f) {
            if (log && depth <= 16) log[2 * D] |= 1u << (2 * (depth - 1));
            const float kk = __fmul_rn(cl, 0.318309886183790671538f);  // cos / pi
            const float4 p = make_float4(__fmul_rn(__fmul_rn(b.x, a0), __fmul_rn(A.P.sun_E[0], kk)),
                                         __fmul_rn(__fmul_rn(b.y, a1), __fmul_rn(A.P.sun_E[1], kk)),
                                         __fmul_rn(__fmul_rn(b.z, a2), __fmul_rn(A.P.sun_E[2], kk)), 0.f);
            if (replay && depth <= kVisDepths) {
                // the primal found this shadow ray unoccluded or not: add its
                // term after the gradient of this vertex, as the shadow stage
                // would have, without tracing it again
                if (__float_as_uint(A.B.Ltot[j].w) & (1u << (depth - 1))) {
                    float4 l = A.B.L[j];
                    l.x = __fadd_rn(l.x, p.x);
                    l.y = __fadd_rn(l.y, p.y);
                    l.z = __fadd_rn(l.z, p.z);
                    A.B.L[j] = l;
                }
            } else {
                A.B.pend[j] = p;
                push(A.B.qs, A.B.ctr + kCtrStride * depth + kCtrShadow, j);
            }
        }
    }
    if (A.P.sun_on || A.P.n_lights) A.B.sray_o[j] = make_float4(sp.x, sp.y, sp.z, 0.f);
    if (A.P.n_lights) {
        const uint4 xl = draw(A.P.seed, gpix, mt.y, kLightStream + (uint32_t)depth);
        F3 ld, w;
        float dist;
        if (light_sample(A.P, u01(xl.x), u01(xl.y), u01(xl.z), sp, nrm, &ld, &dist, &w)) {
            if (log && depth <= 16) log[2 * D + 1] |= 1u << (2 * (depth - 1));
            if (rlog) log_light_ray(rlog, ld, dist);
            const float ip = 0.318309886183790671538f;  // 1 / pi
            A.B.lpend[j] = make_float4(__fmul_rn(__fmul_rn(b.x, a0), __fmul_rn(w.x, ip)),
                                       __fmul_rn(__fmul_rn(b.y, a1), __fmul_rn(w.y, ip)),
                                       __fmul_rn(__fmul_rn(b.z, a2), __fmul_rn(w.z, ip)), 0.f);
            A.B.lray_d[j] = make_float4(ld.x, ld.y, ld.z, dist);
            push(A.B.qs, A.B.ctr + kCtrStride * depth + kCtrShadow, j | kLightRay);
        }
    }
    b.x = __fmul_rn(b.x, a0);
    b.y = __fmul_rn(b.y, a1);
    b.z = __fmul_rn(b.z, a2);
    A.B.beta[j] = b;
    if ((uint32_t)depth < D) {
        const uint4 xi = draw(A.P.seed, gpix, mt.y, (uint32_t)depth);
        const F3 nd = sample_cosine(nrm, u01(xi.x), u01(xi.y));
        if (A.P.ray_log) log_ray(ray_log_rec(A.P, g, depth + 1), sp, nd);
        A.B.ray_o[j] = make_float4(sp.x, sp.y, sp.z, 0.f);
        A.B.ray_d[j] = make_float4(nd.x, nd.y, nd.z, kInfF);
        push(A.B.q[(depth + 1) & 1], A.B.ctr + kCtrStride * (depth + 1) + kCtrClosest, j);
    }
    if (A.stats) atomicAdd(A.stats + 5, 1ull);  // shaded vertices (closest-hit counters)
}

// Mean over each pixel's samples (in sample order) for items [I0, I0 + n).
__global__ void __launch_bounds__(256) wave_accumulate(const __grid_constant__ WaveArgs A,
                                                       uint64_t I0, uint32_t n) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint64_t item = I0 + k;
    const ViewDev& V = A.views[find_view_by_item(A, item)];
    const uint64_t pix = item - V.item_begin;
    const uint64_t j0 = V.path_begin + pix * V.spp - A.P0;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (uint32_t s = 0; s < V.spp; ++s) {
        const float4 l = A.B.L[j0 + s];
        s0 = __fadd_rn(s0, l.x);
        s1 = __fadd_rn(s1, l.y);
        s2 = __fadd_rn(s2, l.z);
    }
    float* out = V.out + 3 * pix;
    out[0] = __fdiv_rn(s0, (float)V.spp);
    out[1] = __fdiv_rn(s1, (float)V.spp);
    out[2] = __fdiv_rn(s2, (float)V.spp);
    if (V.cost_out) {
        uint32_t c = 0;
        for (uint32_t s = 0; s < V.spp; ++s) c += A.B.cost[j0 + s];
        V.cost_out[pix] = (float)c / (float)V.spp;
    }
}

template <bool ANY, int FETCH, int OCC, bool STATS, bool UV>
static cudaError_t launch_wave_trace_v(const WaveArgs& A, int depth, const Tune& t, int sm_count,
                                       cudaStream_t s) {
    static ResidentBlocks resident;
    const int per_sm = t.blocks_per_sm > 0 ? t.blocks_per_sm
                                           : resident.get(wave_trace<ANY, FETCH, OCC, STATS, UV>, t.block);
    wave_trace<ANY, FETCH, OCC, STATS, UV><<<(unsigned)(sm_count * per_sm), t.block, 0, s>>>(
        A, depth, t.stack);
    return cudaGetLastError();
}

template <bool ANY, bool UV>
static cudaError_t launch_wave_trace_uv(const WaveArgs& A, int depth, const Tune& t, int sm_count,
                                        cudaStream_t s) {
    const bool st = A.stats != nullptr, f32 = t.fetch == 32;
#define QRT_WT(FE, OC, ST) return launch_wave_trace_v<ANY, FE, OC, ST, UV>(A, depth, t, sm_count, s)
#define QRT_WT_OCC(OC)                                          \
    if (t.occupancy == OC) {                                    \
        if (st) { if (f32) QRT_WT(32, OC, true); QRT_WT(16, OC, true); } \
        if (f32) QRT_WT(32, OC, false);                         \
        QRT_WT(16, OC, false);                                  \
    }
    QRT_WT_OCC(32)
    QRT_WT_OCC(40)
    QRT_WT_OCC(48)
    QRT_WT_OCC(24)
    QRT_WT_OCC(16)
#undef QRT_WT_OCC
#undef QRT_WT
    return cudaErrorInvalidValue;
}

// Closest-hit rays carry (u, v) only when the shading reads them.
template <bool ANY>
static cudaError_t launch_wave_trace(const WaveArgs& A, int depth, const Tune& t, int sm_count,
                                     cudaStream_t s) {
    if constexpr (!ANY) {
        if (A.P.tex_res) return launch_wave_trace_uv<false, true>(A, depth, t, sm_count, s);
    }
    return launch_wave_trace_uv<ANY, false>(A, depth, t, sm_count, s);
}

void wave_carve(void* base, uint64_t C, bool adjoint, WaveBufs& B) {
    char* p = static_cast<char*>(base);
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) & ~size_t(255);
        return r;
    };
    B.ray_o = reinterpret_cast<float4*>(take(16 * C));
    B.ray_d = reinterpret_cast<float4*>(take(16 * C));
    B.beta = reinterpret_cast<float4*>(take(16 * C));
    B.L = reinterpret_cast<float4*>(take(16 * C));
    B.pend = reinterpret_cast<float4*>(take(16 * C));
    B.sray_o = reinterpret_cast<float4*>(take(16 * C));
    B.lray_d = reinterpret_cast<float4*>(take(16 * C));
    B.lpend = reinterpret_cast<float4*>(take(16 * C));
    B.hit = reinterpret_cast<uint4*>(take(16 * C));
    B.hit_uv = reinterpret_cast<float2*>(take(8 * C));
    B.meta = reinterpret_cast<uint2*>(take(8 * C));
    B.q[0] = reinterpret_cast<uint32_t*>(take(4 * C));
    B.q[1] = reinterpret_cast<uint32_t*>(take(4 * C));
    B.qs = reinterpret_cast<uint32_t*>(take(4 * C));
    B.cost = reinterpret_cast<uint32_t*>(take(4 * C));
    B.Ltot = adjoint ? reinterpret_cast<float4*>(take(16 * C)) : nullptr;
    B.ctr = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * kCtrStride * 258));
}

// Scratch of qrt_render_spp_static.  It lives as long as the library is
// loaded on every device that runs it; concurrent calls share it.
static __device__ __align__(256) unsigned char g_static_workspace[kStaticWorkspaceBytes];

// The array's address is looked up once per device and context: a context
// made anew (after cudaDeviceReset, say) holds a new copy of the array at
// another address, so the cache is keyed by the context's unique id
// (cuCtxGetId, reached through the runtime's driver entry points; nothing is
// linked against the driver library).
namespace {
using CtxGetCurrent = int (*)(void**);
using CtxGetId = int (*)(void*, unsigned long long*);

cudaError_t current_context_id(unsigned long long* id) {
    static CtxGetCurrent get_current = nullptr;
    static CtxGetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrent>(f);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetId>(f);
    });
    if (!get_current || !get_id) return cudaErrorNotSupported;
    void* ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return cudaErrorDeviceUninitialized;
    return get_id(ctx, id) == 0 ? cudaSuccess : cudaErrorDeviceUninitialized;
}
}  // namespace

cudaError_t static_workspace(void** ptr) {
    constexpr int kMaxDevices = 64;
    struct Entry {
        unsigned long long ctx = 0;
        void* addr = nullptr;
    };
    static std::mutex mu;
    static Entry cache[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    // makes the device's primary context current (initialising it if needed)
    if ((e = cudaSetDevice(dev)) != cudaSuccess) return e;
    unsigned long long ctx = 0;
    if ((e = current_context_id(&ctx)) != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    Entry& c = cache[dev];
    if (!c.addr || c.ctx != ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_workspace);
        if (e != cudaSuccess) return e;
        c.addr = p;
        c.ctx = ctx;
    }
    *ptr = c.addr;
    return cudaSuccess;
}

// One pass over paths [P0, P0 + n) of the launch.
static cudaError_t wave_pass(WaveArgs& A, uint64_t P0, uint32_t n, int replay, const Tune& t,
                             int sm_count, cudaStream_t s, StageHook* hook, const WaveStreams* ov) {
    const bool overlap = ov && ov->aux && (A.P.sun_on || A.P.n_lights);
    A.P0 = P0;
    cudaError_t e = cudaMemsetAsync(A.B.ctr, 0, sizeof(uint32_t) * kCtrStride * (A.P.max_depth + 2), s);
    if (e != cudaSuccess) return e;
    if (hook) hook->begin(kStageGen, s);
    wave_gen<<<(n + 255) / 256, 256, 0, s>>>(A, P0, n);
    if (hook) hook->end(kStageGen, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    bool shadow_pending = false;
    for (uint32_t i = 1; i <= A.P.max_depth; ++i) {
        if (hook) hook->begin(kStageTrace, s);
        e = launch_wave_trace<false>(A, (int)i, t, sm_count, s);
        if (hook) hook->end(kStageTrace, s);
        if (e != cudaSuccess) return e;
        // shade(i) adds into the radiance that shadow(i - 1) adds into
        if (shadow_pending && (e = cudaStreamWaitEvent(s, ov->join, 0)) != cudaSuccess) return e;
        shadow_pending = false;
        if (hook) hook->begin(kStageShade, s);
        wave_shade<<<(n + 255) / 256, 256, 0, s>>>(A, (int)i, replay);
        if (hook) hook->end(kStageShade, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // the replay traces sun shadow rays only beyond the depths whose
        // visibility the primal recorded; key-light shadow rays every time
        if ((A.P.sun_on && !(replay && i <= (uint32_t)kVisDepths)) || A.P.n_lights) {
            cudaStream_t ss = s;
            if (overlap) {
                if ((e = cudaEventRecord(ov->fork, s)) != cudaSuccess) return e;
                if ((e = cudaStreamWaitEvent(ov->aux, ov->fork, 0)) != cudaSuccess) return e;
                ss = ov->aux;
            }
            if (hook) hook->begin(kStageShadow, ss);
            e = launch_wave_trace<true>(A, (int)i, t, sm_count, ss);
            if (hook) hook->end(kStageShadow, ss);
            if (e != cudaSuccess) return e;
            if (overlap) {
                if ((e = cudaEventRecord(ov->join, ss)) != cudaSuccess) return e;
                shadow_pending = true;
            }
        }
    }
    if (shadow_pending && (e = cudaStreamWaitEvent(s, ov->join, 0)) != cudaSuccess) return e;
    if (A.P.n_lights) {
        // key-light terms of the last vertices (no shade stage follows them)
        wave_fold<<<(n + 255) / 256, 256, 0, s>>>(A, n);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_wave(WaveArgs& A, const Tune& t, int sm_count, cudaStream_t s, StageHook* hook,
                        const WaveStreams* ov) {
    // chunks of at most A.capacity paths, cut at pixel boundaries
    uint64_t P_total = 0;
    for (uint32_t v = 0; v < A.n_views; ++v)
        P_total = A.views[v].path_begin + (uint64_t)A.views[v].w * A.views[v].h * A.views[v].spp;
    uint64_t P0 = A.views[0].path_begin;
    cudaError_t e = cudaSuccess;
    while (P0 < P_total) {
        // view containing P0 and the chunk end rounded down to a pixel boundary
        uint64_t P1 = std::min<uint64_t>(P_total, P0 + A.capacity);
        int v1 = 0;
        for (int v = 0; v < (int)A.n_views; ++v)
            if (A.views[v].path_begin < P1) v1 = v;
        const ViewDev& V1 = A.views[v1];
        if (P1 < P_total) {
            const uint64_t local = P1 - V1.path_begin;
            P1 = V1.path_begin + (local / V1.spp) * V1.spp;
        }
        const uint32_t n = (uint32_t)(P1 - P0);
        if (A.grad) {
            if ((e = wave_pass(A, P0, n, 0, t, sm_count, s, hook, ov)) != cudaSuccess) return e;
            // radiance of pass one becomes Ltot; L restarts at zero in the replay
            e = cudaMemcpyAsync(A.B.Ltot, A.B.L, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
            if ((e = wave_pass(A, P0, n, 1, t, sm_count, s, hook, ov)) != cudaSuccess) return e;
        } else {
            if ((e = wave_pass(A, P0, n, 0, t, sm_count, s, hook, ov)) != cudaSuccess) return e;
            // pixels of this chunk: items whose paths lie in [P0, P1)
            int v0 = 0;
            for (int v = 0; v < (int)A.n_views; ++v)
                if (A.views[v].path_begin <= P0) v0 = v;
            const ViewDev& V0 = A.views[v0];
            const uint64_t I0 = V0.item_begin + (P0 - V0.path_begin) / V0.spp;
            uint64_t I1;
            if (P1 >= P_total) {
                const ViewDev& VL = A.views[A.n_views - 1];
                I1 = VL.item_begin + (uint64_t)VL.w * VL.h;
            } else {
                I1 = V1.item_begin + (P1 - V1.path_begin) / V1.spp;
            }
            const uint32_t ni = (uint32_t)(I1 - I0);
            if (hook) hook->begin(kStageAccum, s);
            wave_accumulate<<<(ni + 255) / 256, 256, 0, s>>>(A, I0, ni);
            if (hook) hook->end(kStageAccum, s);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        P0 = P1;
    }
    return cudaSuccess;
}

}  // namespace qrt

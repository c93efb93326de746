// Path tracer (qrt_render_spp), its adjoint by path replay
// (qrt_render_adjoint) and the L2 image loss.
//
// One persistent kernel covers every (view, pixel) of a launch: each warp
// claims 32*batch consecutive pixels at a time from a global counter, each
// lane renders all spp samples of its pixel and writes the mean, so the
// primal needs no atomics and a pixel's value does not depend on how views
// are batched.  Random numbers: Philox4x32-10 keyed by the render seed with
// counter (global pixel lo, global pixel hi, sample, bounce).
//
// Per path (Section 5.4, "Shading": a path tracer with progressive
// one-sample-per-pixel refinement; Section 6: a maximum path depth):
//   camera ray through (x + xi1, y + xi2);
//   for i = 1..D: closest hit; on a miss add beta * env and stop; at a hit
//   take the per-quad albedo a and the geometric normal faced against the
//   ray, add the sun term beta * a/pi * E * (n.l) when the shadow ray toward
//   the sun is unoccluded, set beta *= a, and continue along a cosine-
//   distributed direction from an offset origin.
#include <math_constants.h>

#include "launch.h"
#include "shading.cuh"
#include "traverse.cuh"

namespace qrt {

// One path sample.  mode 0: returns its radiance in L.  mode 1 (replay):
// recomputes the identical path and adds w * dL/da into A.grad, where the
// radiance leaving vertex i is Ltot minus the sun terms gathered before i.
// Every floating-point operation on the path is an explicitly rounded
// intrinsic (nothing is left for the compiler to contract), so each inlined
// copy -- primal, replay pass 1, replay pass 2 -- computes bit-identical paths.
template <int STACK, int FETCH>
__device__ __forceinline__ uint32_t path_sample(const RenderArgs& A, const ViewDev& V, uint32_t x,
                                             uint32_t y, uint64_t gpix, uint32_t smp, int mode,
                                             float* L, const float* Ltot, const float* w,
                                             uint32_t* log, float* rlog, TraceStats* st) {
    const ParamsDev& P = A.P;
    const DevScene& S = A.S;
    uint32_t err = 0;
    TraceStats ls{0, 0, 0, 0, 0, 0};
    uint4 xi = draw(P.seed, gpix, smp, 0);
    F3 d = camera_dir(V, x, y, u01(xi.x), u01(xi.y));
    F3 o = f3(V.eye[0], V.eye[1], V.eye[2]);
    float b0 = 1.f, b1 = 1.f, b2 = 1.f;     // throughput
    float l0 = 0.f, l1 = 0.f, l2 = 0.f;     // radiance
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;     // next-event terms so far (replay)
    uint32_t shadow_bits = 0, light_bits = 0;
    const uint32_t D = P.max_depth;
    uint32_t i = 1;
    if (rlog) clear_ray_log(rlog, D);
    for (; i <= D; ++i) {
        Hit h;
        if (rlog) log_ray(rlog + (i - 1) * kRayLogFloats, o, d);
        err |= trace_ray<false, STACK, FETCH>(S, o.x, o.y, o.z, d.x, d.y, d.z, 0.0f, kInfF,
                                               P.max_steps, h, ls);
        if (log) {
            log[2 * (i - 1)] = h.inst;
            log[2 * (i - 1) + 1] = h.prim;
        }
        if (h.inst == 0xFFFFFFFFu) {
            l0 = __fmaf_rn(b0, P.env[0], l0);
            l1 = __fmaf_rn(b1, P.env[1], l1);
            l2 = __fmaf_rn(b2, P.env[2], l2);
            ++i;
            break;
        }
        ++ls.verts;
        uint32_t qbase;
        const F3 n = hit_normal(S, h.inst, h.slot, d, &qbase);
        const uint32_t row = qbase + h.prim;
        const float q0 = __ldg(A.albedo + 3 * (size_t)row);
        const float q1 = __ldg(A.albedo + 3 * (size_t)row + 1);
        const float q2 = __ldg(A.albedo + 3 * (size_t)row + 2);
        float a0 = q0, a1 = q1, a2 = q2;  // diffuse albedo: the quad's, times its texture
        if (P.tex_res) {
            const F3 tx = tex_lookup(P.tex, P.tex_res, row, h.u, h.v);
            a0 = __fmul_rn(q0, tx.x);
            a1 = __fmul_rn(q1, tx.y);
            a2 = __fmul_rn(q2, tx.z);
        }
        const F3 sp = spawn_point(o, d, h.t, n);
        if (rlog) log_spawn(rlog + (i - 1) * kRayLogFloats, sp);
        float n0 = 0.f, n1 = 0.f, n2 = 0.f;  // this vertex's sun term
        if (P.sun_on) {
            const float cl = dot3(n, f3(P.sun_l[0], P.sun_l[1], P.sun_l[2]));
            if (cl > 0.f) {
                if (i <= 16) shadow_bits |= 1u << (2 * (i - 1));
                Hit hs;
                err |= trace_ray<true, STACK, FETCH>(S, sp.x, sp.y, sp.z, P.sun_l[0], P.sun_l[1],
                                                      P.sun_l[2], 0.0f, kInfF, P.max_steps, hs, ls);
                if (hs.inst != 0xFFFFFFFFu) {
                    if (i <= 16) shadow_bits |= 2u << (2 * (i - 1));
                } else {
                    const float k = __fmul_rn(cl, 0.318309886183790671538f);  // cos / pi
                    n0 = __fmul_rn(__fmul_rn(b0, a0), __fmul_rn(P.sun_E[0], k));
                    n1 = __fmul_rn(__fmul_rn(b1, a1), __fmul_rn(P.sun_E[1], k));
                    n2 = __fmul_rn(__fmul_rn(b2, a2), __fmul_rn(P.sun_E[2], k));
                }
            }
        }
        if (mode == 1) {
            // d L / d q_i = (radiance leaving vertex i) / q_i, q_i the quad's
            // albedo (the texture factor is a constant of the path)
            const float g0 = q0 != 0.f ? __fdiv_rn(__fmul_rn(w[0], __fsub_rn(Ltot[0], s0)), q0) : 0.f;
            const float g1 = q1 != 0.f ? __fdiv_rn(__fmul_rn(w[1], __fsub_rn(Ltot[1], s1)), q1) : 0.f;
            const float g2 = q2 != 0.f ? __fdiv_rn(__fmul_rn(w[2], __fsub_rn(Ltot[2], s2)), q2) : 0.f;
            grad_add(A.grad, row, g0, g1, g2);
            s0 = __fadd_rn(s0, n0);
            s1 = __fadd_rn(s1, n1);
            s2 = __fadd_rn(s2, n2);
        }
        l0 = __fadd_rn(l0, n0);
        l1 = __fadd_rn(l1, n1);
        l2 = __fadd_rn(l2, n2);
        // key light: one sample, its shadow ray traced toward the sampled
        // point; added after the sun term, as the wavefront shadow stage
        // adds it after the sun's
        if (P.n_lights) {
            const uint4 xl = draw(P.seed, gpix, smp, kLightStream + i);
            F3 ld, wl;
            float dist;
            if (light_sample(P, u01(xl.x), u01(xl.y), u01(xl.z), sp, n, &ld, &dist, &wl)) {
                if (i <= 16) light_bits |= 1u << (2 * (i - 1));
                if (rlog) log_light_ray(rlog + (i - 1) * kRayLogFloats, ld, dist);
                Hit hl;
                err |= trace_ray<true, STACK, FETCH>(S, sp.x, sp.y, sp.z, ld.x, ld.y, ld.z, 0.0f, dist,
                                                      P.max_steps, hl, ls);
                if (hl.inst != 0xFFFFFFFFu) {
                    if (i <= 16) light_bits |= 2u << (2 * (i - 1));
                } else {
                    const float ip = 0.318309886183790671538f;  // 1 / pi
                    const float m0 = __fmul_rn(__fmul_rn(b0, a0), __fmul_rn(wl.x, ip));
                    const float m1 = __fmul_rn(__fmul_rn(b1, a1), __fmul_rn(wl.y, ip));
                    const float m2 = __fmul_rn(__fmul_rn(b2, a2), __fmul_rn(wl.z, ip));
                    l0 = __fadd_rn(l0, m0);
                    l1 = __fadd_rn(l1, m1);
                    l2 = __fadd_rn(l2, m2);
                    if (mode == 1) {
                        s0 = __fadd_rn(s0, m0);
                        s1 = __fadd_rn(s1, m1);
                        s2 = __fadd_rn(s2, m2);
                    }
                }
            }
        }
        b0 = __fmul_rn(b0, a0);
        b1 = __fmul_rn(b1, a1);
        b2 = __fmul_rn(b2, a2);
        if (i == D) {
            ++i;
            break;
        }
        xi = draw(P.seed, gpix, smp, i);
        d = sample_cosine(n, u01(xi.x), u01(xi.y));
        o = sp;
    }
    if (log) {
        for (uint32_t k = i - 1; k < D; ++k) {
            log[2 * k] = 0xFFFFFFFFu;
            log[2 * k + 1] = 0xFFFFFFFFu;
        }
        log[2 * D] = shadow_bits;
        log[2 * D + 1] = light_bits;
    }
    L[0] = l0;
    L[1] = l1;
    L[2] = l2;
    st->rays += ls.rays;
    st->nodes += ls.nodes;
    st->quads += ls.quads;
    st->insts += ls.insts;
    st->fallbacks += ls.fallbacks;
    st->verts += ls.verts;
    return err;
}

__device__ __forceinline__ int find_view(const RenderArgs& A, uint64_t item) {
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

template <int STACK, int FETCH, bool ADJ>
__global__ void __launch_bounds__(256) render_kernel(const __grid_constant__ RenderArgs A) {
    const int lane = threadIdx.x & 31;
    const uint32_t D = A.P.max_depth;
    uint32_t err = 0;
    uint64_t bad = ~0ull;
    TraceStats st{0, 0, 0, 0, 0, 0};
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(A.counter, 32ull * A.batch);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= A.n_items) break;
        for (uint32_t k = 0; k < A.batch; ++k) {
            const uint64_t item = base + 32ull * k + lane;
            if (item >= A.n_items) break;
            const ViewDev& V = A.views[find_view(A, item)];
            const uint64_t pix = item - V.item_begin;
            uint32_t x, y;
            const uint64_t gpix = view_pixel(V, pix, &x, &y);
            const float inv_spp = __frcp_rn((float)V.spp);
            if (!ADJ) {
                float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
                for (uint32_t s = 0; s < V.spp; ++s) {
                    float L[3];
                    const uint64_t g = V.path_begin + pix * V.spp + s;
                    uint32_t* log = A.P.path_log ? A.P.path_log + g * path_log_words(D) : nullptr;
                    float* rlog = A.P.ray_log ? ray_log_rec(A.P, g, 1) : nullptr;
                    const uint32_t e = path_sample<STACK, FETCH>(A, V, x, y, gpix, V.sample_base + s, 0, L, nullptr,
                                                                 nullptr, log, rlog, &st);
                    if (e) {
                        err |= e;
                        bad = min(bad, item);
                    }
                    acc0 = __fadd_rn(acc0, L[0]);
                    acc1 = __fadd_rn(acc1, L[1]);
                    acc2 = __fadd_rn(acc2, L[2]);
                }
                float* out = V.out + 3 * pix;
                out[0] = __fdiv_rn(acc0, (float)V.spp);
                out[1] = __fdiv_rn(acc1, (float)V.spp);
                out[2] = __fdiv_rn(acc2, (float)V.spp);
            } else {
                const float* di = V.dimage + 3 * pix;
                const float w[3] = {__fmul_rn(__ldg(di), inv_spp), __fmul_rn(__ldg(di + 1), inv_spp),
                                    __fmul_rn(__ldg(di + 2), inv_spp)};
                if (w[0] == 0.f && w[1] == 0.f && w[2] == 0.f) continue;
                for (uint32_t s = 0; s < V.spp; ++s) {
                    float L[3], L2[3];
                    uint32_t e = path_sample<STACK, FETCH>(A, V, x, y, gpix, V.sample_base + s, 0, L, nullptr,
                                                           nullptr, nullptr, nullptr, &st);
                    e |= path_sample<STACK, FETCH>(A, V, x, y, gpix, V.sample_base + s, 1, L2, L, w, nullptr,
                                                   nullptr, &st);
                    if (e) {
                        err |= e;
                        bad = min(bad, item);
                    }
                }
            }
        }
    }
    if (err) {
        atomicOr(A.S.err, err);
        atomicMin(A.S.err + 1, (uint32_t)min(bad, (uint64_t)0xFFFFFFFEu));
    }
    if (A.stats) add_stats(A.stats, st);
}

template <int STACK, int FETCH, bool ADJ>
static int occupancy_of(int block) {
    static ResidentBlocks resident;
    return resident.get(render_kernel<STACK, FETCH, ADJ>, block);
}

int render_occupancy(const Tune& t, bool adjoint) {
    const bool s32 = t.stack <= 32, f32 = t.fetch == 32;
    if (adjoint) {
        if (s32) return f32 ? occupancy_of<32, 32, true>(t.block) : occupancy_of<32, 16, true>(t.block);
        return f32 ? occupancy_of<64, 32, true>(t.block) : occupancy_of<64, 16, true>(t.block);
    }
    if (s32) return f32 ? occupancy_of<32, 32, false>(t.block) : occupancy_of<32, 16, false>(t.block);
    return f32 ? occupancy_of<64, 32, false>(t.block) : occupancy_of<64, 16, false>(t.block);
}

cudaError_t launch_render(const RenderArgs& A, const Tune& t, int sm_count, cudaStream_t s) {
    if (A.n_items == 0) return cudaSuccess;
    const bool adj = A.grad != nullptr;
    int per_sm = t.blocks_per_sm > 0 ? t.blocks_per_sm : render_occupancy(t, adj);
    if (per_sm < 1) per_sm = 1;
    uint64_t want = (A.n_items + (uint64_t)t.block - 1) / (uint64_t)t.block;
    uint64_t grid = (uint64_t)sm_count * (uint64_t)per_sm;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    const dim3 g((unsigned)grid), b((unsigned)t.block);
    const bool s32 = t.stack <= 32, f32 = t.fetch == 32;
    if (adj) {
        if (s32) {
            if (f32) render_kernel<32, 32, true><<<g, b, 0, s>>>(A);
            else render_kernel<32, 16, true><<<g, b, 0, s>>>(A);
        } else {
            if (f32) render_kernel<64, 32, true><<<g, b, 0, s>>>(A);
            else render_kernel<64, 16, true><<<g, b, 0, s>>>(A);
        }
    } else {
        if (s32) {
            if (f32) render_kernel<32, 32, false><<<g, b, 0, s>>>(A);
            else render_kernel<32, 16, false><<<g, b, 0, s>>>(A);
        } else {
            if (f32) render_kernel<64, 32, false><<<g, b, 0, s>>>(A);
            else render_kernel<64, 16, false><<<g, b, 0, s>>>(A);
        }
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// L2 loss: loss = sum (img - target)^2 / n (FP64 reduction), dimage = 2 (img - target) / n
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) l2_loss_kernel(const float* __restrict__ img,
                                                      const float* __restrict__ tgt, uint64_t n,
                                                      double* loss, float* __restrict__ dimg) {
    __shared__ double part[8];
    double acc = 0.0;
    const double inv_n = 1.0 / (double)n;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const double r = (double)img[i] - (double)tgt[i];  // exact for float inputs
        acc += r * r;
        if (dimg) dimg[i] = (float)(2.0 * r * inv_n);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += part[k];
        atomicAdd(loss, s * inv_n);
    }
}

cudaError_t launch_l2_loss(const float* img, const float* target, uint64_t n, double* loss,
                           float* dimage, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    uint64_t grid = (n + 255) / 256;
    if (grid > 4096) grid = 4096;
    l2_loss_kernel<<<(unsigned)grid, 256, 0, s>>>(img, target, n, loss, dimage);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Progressive accumulation: sum += frame; mean = sum / frames
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) accumulate_kernel(float* __restrict__ sum,
                                                         const float* frame, float* mean,
                                                         uint64_t n, float frames) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const float s = __fadd_rn(sum[i], frame[i]);
        sum[i] = s;
        if (mean) mean[i] = __fdiv_rn(s, frames);
    }
}

cudaError_t launch_accumulate(float* sum, const float* frame, float* mean, uint64_t n,
                              uint32_t frames, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    uint64_t grid = (n + 255) / 256;
    if (grid > 8192) grid = 8192;
    accumulate_kernel<<<(unsigned)grid, 256, 0, s>>>(sum, frame, mean, n, (float)frames);
    return cudaGetLastError();
}

}  // namespace qrt

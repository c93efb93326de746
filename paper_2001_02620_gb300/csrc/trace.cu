// Ray-query kernels behind qrt_trace_closest / qrt_trace_any.  Persistent:
// a grid of SMs x resident blocks running the warp-synchronous traversal loop
// (persistent_trace); each lane claims `batch` rays at a time from a global
// cursor and starts its next ray as soon as its own is done.
#include "launch.h"
#include "traverse.cuh"

namespace qrt {

template <bool ANY, int STACK, int FETCH, int MINB>
__global__ void __launch_bounds__(256, MINB) trace_kernel(const DevScene S, const float4* __restrict__ rays,
                                                       uint64_t n, uint4* __restrict__ hits,
                                                       uint32_t* __restrict__ occ, uint32_t max_steps,
                                                       unsigned long long* cursor, uint32_t batch,
                                                       unsigned long long* stats) {
    TraceStats st{0, 0, 0, 0, 0, 0};
    Traversal<ANY, STACK, FETCH> T;
    uint64_t next = 0, end = 0, i = 0;
    uint32_t err = 0;
    uint64_t bad = ~0ull;
    auto fetch_ray = [&]() -> bool {
        if (next >= end) {
            next = atomicAdd(cursor, (unsigned long long)batch);
            end = min(next + batch, n);
            if (next >= n) return false;
        }
        i = next++;
        const float4 a = __ldg(rays + 2 * i), b = __ldg(rays + 2 * i + 1);
        T.init(S, a.x, a.y, a.z, b.x, b.y, b.z, a.w, b.w, max_steps, st);
        return true;
    };
    auto finish_ray = [&]() {
        if (T.err) {
            err |= T.err;
            bad = min(bad, i);
        }
        if (ANY) {
            if (T.h.inst != 0xFFFFFFFFu) atomicOr(occ + (i >> 5), 1u << (i & 31));
        } else {
            const uint32_t uq = (uint32_t)__float2uint_rn(__saturatef(T.h.u) * 65535.f);
            const uint32_t vq = (uint32_t)__float2uint_rn(__saturatef(T.h.v) * 65535.f);
            const uint32_t uv = T.h.inst == 0xFFFFFFFFu ? 0u : (uq | (vq << 16));
            hits[i] = make_uint4(__float_as_uint(T.h.t), T.h.inst, T.h.prim, uv);
        }
    };
    persistent_trace<ANY, STACK, FETCH>(S, T, st, fetch_ray, finish_ray);
    if (err) {
        atomicOr(S.err, err);
        atomicMin(S.err + 1, (uint32_t)min(bad, (uint64_t)0xFFFFFFFEu));
    }
    if (stats) add_stats(stats, st);
}

template <bool ANY, int STACK, int FETCH, int MINB>
static cudaError_t launch_variant(const DevScene& S, const float4* rays, uint64_t n, uint4* hits,
                                  uint32_t* occ, uint32_t max_steps, unsigned long long* cursor,
                                  unsigned long long* stats, const Tune& t, int sm_count,
                                  cudaStream_t s) {
    int per_sm = t.blocks_per_sm;
    if (per_sm <= 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trace_kernel<ANY, STACK, FETCH, MINB>,
                                                      t.block, 0);
        if (per_sm < 1) per_sm = 1;
    }
    uint64_t grid = (uint64_t)sm_count * per_sm;
    const uint64_t want = (n + (uint64_t)t.block - 1) / (uint64_t)t.block;
    if (want < grid) grid = want;
    trace_kernel<ANY, STACK, FETCH, MINB><<<(unsigned)grid, t.block, 0, s>>>(
        S, rays, n, hits, occ, max_steps, cursor, (uint32_t)t.batch, stats);
    return cudaGetLastError();
}

template <bool ANY>
static cudaError_t launch_any_variant(const DevScene& S, const void* rays, uint64_t n, void* hits,
                                      uint32_t* occ, uint32_t max_steps, unsigned long long* cursor,
                                      unsigned long long* stats, const Tune& t, int sm_count,
                                      cudaStream_t s) {
    const float4* r = static_cast<const float4*>(rays);
    uint4* hp = static_cast<uint4*>(hits);
    const bool s32 = t.stack <= 32, f32 = t.fetch == 32, o24 = t.occupancy == 24;
#define QRT_TV(ST, FE, MB) \
    return launch_variant<ANY, ST, FE, MB>(S, r, n, hp, occ, max_steps, cursor, stats, t, sm_count, s)
    if (o24) {
        if (s32) { if (f32) QRT_TV(32, 32, 3); QRT_TV(32, 16, 3); }
        if (f32) QRT_TV(64, 32, 3);
        QRT_TV(64, 16, 3);
    }
    if (s32) { if (f32) QRT_TV(32, 32, 2); QRT_TV(32, 16, 2); }
    if (f32) QRT_TV(64, 32, 2);
    QRT_TV(64, 16, 2);
#undef QRT_TV
}

cudaError_t launch_trace(bool any, const DevScene& S, const void* rays, uint64_t n, void* hits,
                         uint32_t* occ_bits, uint32_t max_steps, unsigned long long* cursor,
                         unsigned long long* stats, const Tune& t, int sm_count, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (any) {
        e = cudaMemsetAsync(occ_bits, 0, sizeof(uint32_t) * ((n + 31) / 32), s);
        if (e != cudaSuccess) return e;
        return launch_any_variant<true>(S, rays, n, hits, occ_bits, max_steps, cursor, stats, t,
                                        sm_count, s);
    }
    return launch_any_variant<false>(S, rays, n, hits, occ_bits, max_steps, cursor, stats, t,
                                     sm_count, s);
}

}  // namespace qrt

// Ray-query kernels behind qrt_trace_closest / qrt_trace_any.  Persistent:
// a grid of SMs x resident blocks running the warp-synchronous traversal loop
// (persistent_trace); each lane claims `batch` rays at a time from a global
// cursor and starts its next ray as soon as its own is done.
#include "launch.h"
#include "traverse.cuh"

namespace qrt {

// Work counters are kept only in the STATS variant (dead code elsewhere).
template <bool ANY, int FETCH, int OCC, bool STATS>
__global__ void __maxnreg__(occupancy_regs(OCC)) trace_kernel(const DevScene S, const float4* __restrict__ rays,
                                                       uint64_t n, uint4* __restrict__ hits,
                                                       uint32_t* __restrict__ occ, uint32_t max_steps,
                                                       unsigned long long* cursor, uint32_t batch,
                                                       unsigned long long* stats, int stack_cap) {
    TraceStats st{0, 0, 0, 0, 0, 0};
    Traversal<ANY, kMaxStack, FETCH> T;
    uint64_t i = 0;
    uint32_t err = 0;
    uint64_t bad = ~0ull;
    WRay w{};  // kept per lane: reloading it from the ray array measured slower here
    auto start_ray = [&](unsigned long long k) {
        i = k;
        const float4 a = __ldg(rays + 2 * i), b = __ldg(rays + 2 * i + 1);
        w = WRay{a.x, a.y, a.z, b.x, b.y, b.z};
        T.err = 0;  // per ray: the first affected ray is reported
        T.init(S, a.x, a.y, a.z, b.x, b.y, b.z, a.w, b.w, max_steps, st);
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
    auto world_ray = [&]() { return w; };
    persistent_trace<ANY, kMaxStack, FETCH>(S, T, st, cursor, (unsigned long long)n, batch, stack_cap,
                                            start_ray, finish_ray, world_ray);
    if (err) {
        atomicOr(S.err, err);
        atomicMin(S.err + 1, (uint32_t)min(bad, (uint64_t)0xFFFFFFFEu));
    }
    if constexpr (STATS) add_stats(stats, st);
}

template <bool ANY, int FETCH, int OCC, bool STATS>
static cudaError_t launch_variant(const DevScene& S, const float4* rays, uint64_t n, uint4* hits,
                                  uint32_t* occ, uint32_t max_steps, unsigned long long* cursor,
                                  unsigned long long* stats, const Tune& t, int sm_count,
                                  cudaStream_t s) {
    static ResidentBlocks resident;
    const int per_sm = t.blocks_per_sm > 0 ? t.blocks_per_sm
                                           : resident.get(trace_kernel<ANY, FETCH, OCC, STATS>, t.block);
    uint64_t grid = (uint64_t)sm_count * per_sm;
    const uint64_t want = (n + (uint64_t)t.block - 1) / (uint64_t)t.block;
    if (want < grid) grid = want;
    trace_kernel<ANY, FETCH, OCC, STATS><<<(unsigned)grid, t.block, 0, s>>>(
        S, rays, n, hits, occ, max_steps, cursor, (uint32_t)t.batch, stats, t.stack);
    return cudaGetLastError();
}

template <bool ANY>
static cudaError_t launch_any_variant(const DevScene& S, const void* rays, uint64_t n, void* hits,
                                      uint32_t* occ, uint32_t max_steps, unsigned long long* cursor,
                                      unsigned long long* stats, const Tune& t, int sm_count,
                                      cudaStream_t s) {
    const float4* r = static_cast<const float4*>(rays);
    uint4* hp = static_cast<uint4*>(hits);
    const bool st = stats != nullptr, f32 = t.fetch == 32;
#define QRT_TV(FE, OC, ST) \
    return launch_variant<ANY, FE, OC, ST>(S, r, n, hp, occ, max_steps, cursor, stats, t, sm_count, s)
#define QRT_TV_OCC(OC)                                          \
    if (t.occupancy == OC) {                                    \
        if (st) { if (f32) QRT_TV(32, OC, true); QRT_TV(16, OC, true); } \
        if (f32) QRT_TV(32, OC, false);                         \
        QRT_TV(16, OC, false);                                  \
    }
    QRT_TV_OCC(32)
    QRT_TV_OCC(40)
    QRT_TV_OCC(48)
    QRT_TV_OCC(24)
    QRT_TV_OCC(16)
#undef QRT_TV_OCC
#undef QRT_TV
    return cudaErrorInvalidValue;
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

// Read-bandwidth sweep (a measurement helper, not part of the path): every
// thread reads 16-byte words of buf with L2-only loads, reps times over the
// whole buffer, and folds them into one word per warp so the loads stay live.
// With a buffer that fits in L2 this measures the L2 read bandwidth that
// bounds traversal of a cache-resident BVH.
__global__ void __launch_bounds__(256) read_sweep_kernel(const uint4* __restrict__ buf, uint64_t n16,
                                                         uint32_t reps, uint32_t* sink) {
    uint32_t acc = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint32_t r = 0; r < reps; ++r) {
#pragma unroll 4
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
            const uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicXor(sink, acc);
}

cudaError_t launch_read_sweep(const void* buf, uint64_t bytes, uint32_t reps, uint32_t* sink,
                              int sm_count, cudaStream_t s) {
    const uint64_t n16 = bytes / 16;
    if (n16 == 0 || reps == 0) return cudaSuccess;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, read_sweep_kernel, 256, 0);
    if (per_sm < 1) per_sm = 1;
    uint64_t grid = (uint64_t)sm_count * per_sm;
    const uint64_t want = (n16 + 255) / 256;
    if (want < grid) grid = want;
    read_sweep_kernel<<<(unsigned)grid, 256, 0, s>>>(static_cast<const uint4*>(buf), n16, reps, sink);
    return cudaGetLastError();
}

}  // namespace qrt

// Ray-query kernels behind qrt_trace_closest / qrt_trace_any: one ray per
// thread, 32 consecutive rays per warp so an any-hit warp writes its 32
// occlusion bits with a single ballot and store.
#include "launch.h"
#include "traverse.cuh"

namespace qrt {

template <bool ANY, int STACK, int FETCH>
__global__ void __launch_bounds__(256) trace_kernel(const DevScene S, const float4* __restrict__ rays,
                                                    uint64_t n, uint4* __restrict__ hits,
                                                    uint32_t* __restrict__ occ, uint32_t max_steps,
                                                    unsigned long long* stats) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    Hit h;
    h.inst = 0xFFFFFFFFu;
    uint32_t err = 0;
    TraceStats st{0, 0, 0, 0, 0, 0};
    if (valid) {
        const float4 a = __ldg(rays + 2 * i), b = __ldg(rays + 2 * i + 1);
        err = trace_ray<ANY, STACK, FETCH>(S, a.x, a.y, a.z, b.x, b.y, b.z, a.w, b.w, max_steps, h,
                                           st);
        if (!ANY) {
            const uint32_t uq = (uint32_t)__float2uint_rn(__saturatef(h.u) * 65535.f);
            const uint32_t vq = (uint32_t)__float2uint_rn(__saturatef(h.v) * 65535.f);
            const uint32_t uv = h.inst == 0xFFFFFFFFu ? 0u : (uq | (vq << 16));
            hits[i] = make_uint4(__float_as_uint(h.t), h.inst, h.prim, uv);
        }
    }
    if (ANY) {
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, valid && h.inst != 0xFFFFFFFFu);
        if ((threadIdx.x & 31) == 0 && (i < n)) occ[i >> 5] = bits;
    }
    if (err) {
        atomicOr(S.err, err);
        atomicMin(S.err + 1, (uint32_t)min(i, (uint64_t)0xFFFFFFFEu));
    }
    if (stats) add_stats(stats, st);
}

template <bool ANY>
static cudaError_t launch_any_variant(const DevScene& S, const void* rays, uint64_t n, void* hits,
                                      uint32_t* occ, uint32_t max_steps,
                                      unsigned long long* stats, const Tune& t, cudaStream_t s) {
    const int block = t.block;
    const uint64_t grid = (n + block - 1) / block;
    if (grid > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    const float4* r = static_cast<const float4*>(rays);
    uint4* hp = static_cast<uint4*>(hits);
    if (t.stack <= 32) {
        if (t.fetch == 32)
            trace_kernel<ANY, 32, 32><<<(unsigned)grid, block, 0, s>>>(S, r, n, hp, occ, max_steps, stats);
        else
            trace_kernel<ANY, 32, 16><<<(unsigned)grid, block, 0, s>>>(S, r, n, hp, occ, max_steps, stats);
    } else {
        if (t.fetch == 32)
            trace_kernel<ANY, 64, 32><<<(unsigned)grid, block, 0, s>>>(S, r, n, hp, occ, max_steps, stats);
        else
            trace_kernel<ANY, 64, 16><<<(unsigned)grid, block, 0, s>>>(S, r, n, hp, occ, max_steps, stats);
    }
    return cudaGetLastError();
}

cudaError_t launch_trace(bool any, const DevScene& S, const void* rays, uint64_t n, void* hits,
                         uint32_t* occ_bits, uint32_t max_steps, unsigned long long* stats,
                         const Tune& t, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    return any ? launch_any_variant<true>(S, rays, n, hits, occ_bits, max_steps, stats, t, s)
               : launch_any_variant<false>(S, rays, n, hits, occ_bits, max_steps, stats, t, s);
}

}  // namespace qrt

// Stable LSD radix sort of (64-bit key, 32-bit value) pairs (radix_sort.h).
#include "radix_sort.h"

namespace qrt {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;                             // items per thread and tile
constexpr uint32_t kSortTile = kSortThreads * kSortItems;  // 2048 items per tile
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kScanThreads = 1024;
constexpr uint32_t kScanTile = kScanThreads * 4;  // counts scanned per block
constexpr uint32_t kNoDigit = 256;                // digit of a position past the end
constexpr uint32_t kMaxSortItems = 0xFFFFFFFFu - kSortTile;

__device__ __forceinline__ uint32_t digit_of(uint64_t k, int shift, uint32_t dmask) {
    return (uint32_t)(k >> shift) & dmask;
}

// Exclusive scan of one value per thread over a block of NT threads; *total
// receives the block's sum.  wtot: NT / 32 words of shared memory.
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* wtot, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wtot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NT / 32 ? wtot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) wtot[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const uint32_t before = warp > 0 ? wtot[warp - 1] : 0u;
    *total = wtot[NT / 32 - 1];
    __syncthreads();  // wtot may be reused by the caller
    return before + inc - x;
}

// OR and AND of all keys: oa[0] |= key, oa[1] &= key.
__global__ void k_key_bits(const uint64_t* __restrict__ keys, uint32_t n, unsigned long long* oa) {
    unsigned long long o = 0ull, a = ~0ull;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        o |= k;
        a &= k;
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        o |= __shfl_xor_sync(0xFFFFFFFFu, o, s);
        a &= __shfl_xor_sync(0xFFFFFFFFu, a, s);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicOr(&oa[0], o);
        atomicAnd(&oa[1], a);
    }
}

// Digit counts of one tile, written digit-major: counts[d * tiles + tile].
__global__ void __launch_bounds__(kSortThreads)
    k_tile_counts(const uint64_t* __restrict__ keys, uint32_t n, int shift, uint32_t dmask,
                  uint32_t* __restrict__ counts, uint32_t tiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * kSortTile;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = base + r * kSortThreads + threadIdx.x;
        const uint32_t d = i < n ? digit_of(keys[i], shift, dmask) : kNoDigit;
        const uint32_t same = __match_any_sync(0xFFFFFFFFu, d);
        if (d != kNoDigit && (threadIdx.x & 31) == (uint32_t)(__ffs(same) - 1))
            atomicAdd(&h[d], (uint32_t)__popc(same));
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// In-place exclusive scan of each kScanTile-long block of counts; the block's
// total goes to sums[block].
__global__ void __launch_bounds__(kScanThreads)
    k_scan_blocks(uint32_t* __restrict__ c, uint32_t m, uint32_t* __restrict__ sums) {
    __shared__ uint32_t wtot[kScanThreads / 32];
    const uint32_t i0 = blockIdx.x * kScanTile + threadIdx.x * 4;
    uint32_t v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = i0 + k < m ? c[i0 + k] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan<kScanThreads>(s, wtot, &total);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (i0 + k < m) c[i0 + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// In-place exclusive scan of the block sums, one block looping over them.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint32_t* __restrict__ sums, uint32_t nb) {
    __shared__ uint32_t wtot[kScanThreads / 32];
    uint32_t carry = 0;
    for (uint32_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        const uint32_t i = b0 + threadIdx.x;
        const uint32_t v = i < nb ? sums[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan<kScanThreads>(v, wtot, &total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads)
    k_scan_add(uint32_t* __restrict__ c, uint32_t m, const uint32_t* __restrict__ sums) {
    const uint32_t add = sums[blockIdx.x];
    const uint32_t i0 = blockIdx.x * kScanTile + threadIdx.x * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (i0 + k < m) c[i0 + k] += add;
}

// One pass: every tile ranks its items by (digit, position) and writes them
// to offs[d * tiles + tile] + (rank among the tile's items of digit d).
// Items are read in rounds of kSortThreads consecutive positions, so the
// order (round, warp, lane) is the input order and equal digits stay in it.
__global__ void __launch_bounds__(kSortThreads)
    k_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
              uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, uint32_t n, int shift,
              uint32_t dmask, const uint32_t* __restrict__ offs, uint32_t tiles) {
    __shared__ uint64_t sk[kSortTile];
    __shared__ uint32_t sv[kSortTile];
    __shared__ uint32_t wcount[kSortWarps][256];  // this round's count per warp and digit
    __shared__ uint32_t wbase[kSortWarps][256];   // rank of a warp's first item of a digit
    __shared__ uint32_t run[256];                 // items of each digit in earlier rounds
    __shared__ uint32_t lstart[256];              // first tile-local position of each digit
    __shared__ uint32_t goff[256];                // first output position of each digit
    __shared__ uint32_t wtot[kSortWarps];
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t base = blockIdx.x * kSortTile;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) wcount[w][t] = 0;
    run[t] = 0;
    goff[t] = offs[(size_t)t * tiles + blockIdx.x];
    uint64_t key[kSortItems];
    uint32_t val[kSortItems], dig[kSortItems], rank[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = base + r * kSortThreads + t;
        key[r] = i < n ? kin[i] : 0ull;
        val[r] = i < n ? vin[i] : 0u;
        dig[r] = i < n ? digit_of(key[r], shift, dmask) : kNoDigit;
    }
    __syncthreads();
    const uint32_t below = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t same = __match_any_sync(0xFFFFFFFFu, dig[r]);
        const uint32_t before = (uint32_t)__popc(same & below);
        if (dig[r] != kNoDigit && before == 0) wcount[warp][dig[r]] = (uint32_t)__popc(same);
        __syncthreads();
        // thread t owns digit t: ranks of each warp's first item, counts reset
        uint32_t b = run[t];
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = wcount[w][t];
            wbase[w][t] = b;
            wcount[w][t] = 0;
            b += c;
        }
        run[t] = b;
        __syncthreads();
        rank[r] = dig[r] != kNoDigit ? wbase[warp][dig[r]] + before : 0u;
    }
    uint32_t total;
    const uint32_t ls = block_exclusive_scan<kSortThreads>(run[t], wtot, &total);
    lstart[t] = ls;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (dig[r] != kNoDigit) {
            const uint32_t p = lstart[dig[r]] + rank[r];
            sk[p] = key[r];
            sv[p] = val[r];
        }
    }
    __syncthreads();
    const uint32_t tile_n = n - base < kSortTile ? n - base : kSortTile;
    for (uint32_t p = t; p < tile_n; p += kSortThreads) {
        const uint64_t k = sk[p];
        const uint32_t d = digit_of(k, shift, dmask);
        const uint32_t g = goff[d] + (p - lstart[d]);
        kout[g] = k;
        vout[g] = sv[p];
    }
}

struct Scratch {
    unsigned long long* oa;
    uint32_t* counts;
    uint32_t* sums;
    uint32_t tiles, m, nb;
};

Scratch carve(void* scratch, uint32_t n) {
    Scratch s;
    s.tiles = (uint32_t)(((uint64_t)n + kSortTile - 1) / kSortTile);
    s.m = 256u * s.tiles;
    s.nb = (s.m + kScanTile - 1) / kScanTile;
    char* p = static_cast<char*>(scratch);
    s.oa = reinterpret_cast<unsigned long long*>(p);
    s.counts = reinterpret_cast<uint32_t*>(p + 16);
    s.sums = reinterpret_cast<uint32_t*>(p + 16 + (((size_t)s.m * 4 + 15) & ~(size_t)15));
    return s;
}

}  // namespace

size_t sort_pairs_scratch_bytes(uint32_t n) {
    const uint64_t tiles = ((uint64_t)n + kSortTile - 1) / kSortTile;
    const uint64_t m = 256u * tiles;
    const uint64_t nb = (m + kScanTile - 1) / kScanTile;
    return 16 + ((m * 4 + 15) & ~(uint64_t)15) + nb * 4;
}

cudaError_t sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_out, uint32_t* vals_out,
                       uint32_t n, int end_bit, void* scratch, cudaStream_t stream) {
    // positions inside the last tile must not wrap around 32 bits
    if (end_bit < 0 || end_bit > 64 || n > kMaxSortItems) return cudaErrorInvalidValue;
    const Scratch s = carve(scratch, n);
    unsigned long long oa[2] = {0ull, ~0ull};
    cudaError_t e;
    if (n > 1 && end_bit > 0) {
        if ((e = cudaMemcpyAsync(s.oa, oa, sizeof(oa), cudaMemcpyHostToDevice, stream))) return e;
        k_key_bits<<<1024, 256, 0, stream>>>(keys, n, s.oa);
        if ((e = cudaGetLastError())) return e;
        if ((e = cudaMemcpyAsync(oa, s.oa, sizeof(oa), cudaMemcpyDeviceToHost, stream))) return e;
        if ((e = cudaStreamSynchronize(stream))) return e;
    } else {
        oa[0] = oa[1] = 0ull;  // no pass
    }
    const uint64_t sort_mask = end_bit >= 64 ? ~0ull : ((1ull << end_bit) - 1ull);
    const uint64_t varies = (oa[0] ^ oa[1]) & sort_mask;
    uint64_t* ks[2] = {keys, keys_out};
    uint32_t* vs[2] = {vals, vals_out};
    int cur = 0;
    for (int shift = 0; shift < end_bit; shift += 8) {
        if (((varies >> shift) & 0xFFull) == 0) continue;
        const uint32_t dmask = end_bit - shift >= 8 ? 0xFFu : ((1u << (end_bit - shift)) - 1u);
        k_tile_counts<<<s.tiles, kSortThreads, 0, stream>>>(ks[cur], n, shift, dmask, s.counts, s.tiles);
        k_scan_blocks<<<s.nb, kScanThreads, 0, stream>>>(s.counts, s.m, s.sums);
        k_scan_sums<<<1, kScanThreads, 0, stream>>>(s.sums, s.nb);
        k_scan_add<<<s.nb, kScanThreads, 0, stream>>>(s.counts, s.m, s.sums);
        k_scatter<<<s.tiles, kSortThreads, 0, stream>>>(ks[cur], vs[cur], ks[cur ^ 1], vs[cur ^ 1], n,
                                                        shift, dmask, s.counts, s.tiles);
        if ((e = cudaGetLastError())) return e;
        cur ^= 1;
    }
    if (cur == 0 && n > 0) {
        if ((e = cudaMemcpyAsync(keys_out, keys, (size_t)n * 8, cudaMemcpyDeviceToDevice, stream)))
            return e;
        if ((e = cudaMemcpyAsync(vals_out, vals, (size_t)n * 4, cudaMemcpyDeviceToDevice, stream)))
            return e;
    }
    return cudaSuccess;
}

}  // namespace qrt

// Linear BVH build of the TLAS on the GPU (declared in lbvh.h).  Every step
// is a function of one node or one item, written once for host and device:
// the kernels call them per thread, and the host path runs the same functions
// in loops, so the index arithmetic is exercised without a GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cub/device/device_radix_sort.cuh>

#include "lbvh.h"

namespace qrt {
namespace {

constexpr uint32_t kLeafBit = 0x80000000u;  // binary child reference: leaf (sorted position)
constexpr uint32_t kNone = 0xFFFFFFFFu;

__host__ __device__ inline int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

__host__ __device__ inline int clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __clz((int)x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}

// 2^e for e in [-126, 127], built from its bit pattern (exact).
__host__ __device__ inline float pow2f(int e) {
    const uint32_t bits = (uint32_t)(e + 127) << 23;
    float f;
    memcpy(&f, &bits, 4);
    return f;
}

// Products and sums rounded one by one on both sides (no contraction into
// fused multiply-adds), so host and device pick the same child to open.
__host__ __device__ inline float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}

__host__ __device__ inline float add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}

// The low 21 bits of v spread to every third bit of a 63-bit word.
__host__ __device__ inline uint64_t spread21(uint32_t v) {
    uint64_t x = v & 0x1FFFFFu;
    x = (x | (x << 32)) & 0x1F00000000FFFFull;
    x = (x | (x << 16)) & 0x1F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Morton key of item i's box centre on a 2^21 grid over the centre bounds.
__host__ __device__ inline uint64_t morton_key(const FBox& b, const float* cmin, const float* scale) {
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        const float c = add_rn(mul_rn(0.5f, b.lo[a]), mul_rn(0.5f, b.hi[a]));
        const float u = mul_rn(c - cmin[a], scale[a]);
        q[a] = u >= 2097151.0f ? 2097151u : (u > 0.0f ? (uint32_t)u : 0u);
    }
    return (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
}

// Length of the common prefix of the augmented keys (key, position) at
// sorted positions i and j; -1 when j lies outside [0, n).  Positions break
// ties between equal keys, so all augmented keys are distinct.
__host__ __device__ inline int prefix(const uint64_t* k, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    const uint64_t a = k[i], b = k[j];
    if (a != b) return clz64(a ^ b);
    return 64 + clz32((uint32_t)i ^ (uint32_t)j);
}

// Children of internal node i (0 <= i < n-1) of the binary radix tree over
// the sorted keys: the node covers the key range from i to j, split where
// the common prefix of the range ends (Karras 2012).  A child reference is an
// internal node index, or kLeafBit | sorted position.
__host__ __device__ inline void radix_node(const uint64_t* k, int64_t n, int64_t i, uint32_t* left,
                                           uint32_t* right) {
    const int d = prefix(k, n, i, i + 1) > prefix(k, n, i, i - 1) ? 1 : -1;
    const int dmin = prefix(k, n, i, i - d);
    // upper bound on the range length by doubling (ends once i + lmax*d
    // leaves [0, n), where the prefix is -1 <= dmin)
    int64_t lmax = 2;
    while (prefix(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (prefix(k, n, i, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = prefix(k, n, i, j);
    // split: the last position s (0 <= s < l) whose prefix with i exceeds dnode
    int64_t s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (s + t < l && prefix(k, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int64_t g = i + s * d + (d < 0 ? -1 : 0);
    const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    *left = lo == g ? (kLeafBit | (uint32_t)g) : (uint32_t)g;
    *right = hi == g + 1 ? (kLeafBit | (uint32_t)(g + 1)) : (uint32_t)(g + 1);
}

__host__ __device__ inline void box_union(FBox& r, const FBox& a, const FBox& b) {
    for (int x = 0; x < 3; ++x) {
        r.lo[x] = fminf(a.lo[x], b.lo[x]);
        r.hi[x] = fmaxf(a.hi[x], b.hi[x]);
    }
}

__host__ __device__ inline float half_area(const FBox& b) {
    const float dx = b.hi[0] - b.lo[0], dy = b.hi[1] - b.lo[1], dz = b.hi[2] - b.lo[2];
    return add_rn(add_rn(mul_rn(dx, dy), mul_rn(dy, dz)), mul_rn(dz, dx));
}

__host__ __device__ inline float dequant_hd(int q, int e, float origin) {
    return fmaf((float)q, pow2f(e), origin);
}

// Conservative quantisation of nc child boxes against their union's lower
// corner: per axis the smallest power-of-two step (found from the extent,
// then raised while needed) at which every child box, rounded outward to
// 8-bit codes, still contains the exact box under the dequantisation
// fma(q, 2^e, origin).  The same rule as the host builder's.
__host__ __device__ inline bool quantize_node(QNode& q, const FBox* cb, int nc) {
    FBox u = cb[0];
    for (int i = 1; i < nc; ++i) box_union(u, u, cb[i]);
    int8_t ex[3];
    for (int a = 0; a < 3; ++a) {
        const float origin = u.lo[a];
        const double ext = (double)u.hi[a] - (double)origin;
        int e = -126;
        if (ext > 0.0) e = (int)ceil(log2(ext / 254.0));
        e = e < -126 ? -126 : (e > 127 ? 127 : e);
        for (;; ++e) {
            if (e > 127) return false;
            bool ok = true;
            const double step = ldexp(1.0, e);
            for (int i = 0; i < nc && ok; ++i) {
                const double fl = floor(((double)cb[i].lo[a] - origin) / step);
                int ql = (int)(fl < 0.0 ? 0.0 : (fl > 255.0 ? 255.0 : fl));
                while (ql > 0 && dequant_hd(ql, e, origin) > cb[i].lo[a]) --ql;
                if (dequant_hd(ql, e, origin) > cb[i].lo[a]) {
                    ok = false;
                    break;
                }
                const double ch = ceil(((double)cb[i].hi[a] - origin) / step);
                if (ch > 255.0) {
                    ok = false;
                    break;
                }
                int qh = (int)(ch < 0.0 ? 0.0 : ch);
                while (qh <= 255 && dequant_hd(qh, e, origin) < cb[i].hi[a]) ++qh;
                if (qh > 255) {
                    ok = false;
                    break;
                }
                q.qlo[a][i] = (uint8_t)ql;
                q.qhi[a][i] = (uint8_t)qh;
            }
            if (ok) break;
        }
        ex[a] = (int8_t)e;
    }
    q.ox = u.lo[0];
    q.oy = u.lo[1];
    q.oz = u.lo[2];
    q.ex = ex[0];
    q.ey = ex[1];
    q.ez = ex[2];
    return true;
}

__host__ __device__ inline FBox load_box(const FBox* p) {
#ifdef __CUDA_ARCH__
    // boxes written by other threads of this launch: read through L2
    const float* f = reinterpret_cast<const float*>(p);
    FBox b;
    for (int x = 0; x < 3; ++x) {
        b.lo[x] = __ldcg(f + x);
        b.hi[x] = __ldcg(f + 3 + x);
    }
    return b;
#else
    return *p;
#endif
}

__host__ __device__ inline FBox child_box(uint32_t c, const FBox* lbox, const FBox* ibox) {
    return (c & kLeafBit) ? lbox[c & ~kLeafBit] : load_box(ibox + c);
}

// Bottom-up box merge from leaf k: at each internal node the first of its two
// children to arrive stops; the second forms the node's box and goes on up.
// No thread waits for another, and each step moves one level up.
// A radix tree over distinct 96-bit augmented keys is at most 97 levels deep;
// the walk stops (and reports) if it ever gets further.
constexpr int kMaxRadixDepth = 128;

__host__ __device__ inline bool merge_up(uint32_t k, uint32_t n, const uint32_t* parent_leaf,
                                         const uint32_t* parent_int, const uint32_t* left,
                                         const uint32_t* right, const FBox* lbox, FBox* ibox,
                                         uint32_t* arrivals) {
    uint32_t node = parent_leaf[k];
    for (int level = 0; node != kNone; ++level) {
        if (level >= kMaxRadixDepth || node + 1 >= n) return false;
#ifdef __CUDA_ARCH__
        __threadfence();  // this child's box is visible before the arrival counts
        const uint32_t prior = atomicAdd(arrivals + node, 1u);
#else
        const uint32_t prior = arrivals[node]++;
#endif
        if (prior == 0) return true;
        box_union(ibox[node], child_box(left[node], lbox, ibox), child_box(right[node], lbox, ibox));
        node = parent_int[node];
    }
    return true;
}

// Children of the four-wide node made from binary internal node b: its two
// children, then repeatedly the internal child with the largest surface area
// replaced by its two children, up to four.  Returns the count.
__host__ __device__ inline int wide_children(uint32_t b, const uint32_t* left, const uint32_t* right,
                                             const FBox* ibox, uint32_t* c) {
    c[0] = left[b];
    c[1] = right[b];
    int nc = 2;
    while (nc < 4) {
        int best = -1;
        float best_area = -1.0f;
        for (int i = 0; i < nc; ++i) {
            if (c[i] & kLeafBit) continue;
            const float a = half_area(load_box(ibox + c[i]));
            if (a > best_area) {
                best_area = a;
                best = i;
            }
        }
        if (best < 0) break;
        const uint32_t x = c[best];
        c[best] = left[x];
        c[nc++] = right[x];
    }
    return nc;
}

// Writes four-wide node `wide` (made from binary node b); its inner children
// get consecutive indices after next_base, in the order of the next level's
// list.  Returns false if the child boxes cannot be quantised.
__host__ __device__ inline bool emit_wide(uint32_t b, uint32_t wide, uint32_t n, const uint32_t* left,
                                          const uint32_t* right, const FBox* lbox, const FBox* ibox,
                                          const uint32_t* ids, uint32_t* next, uint32_t* next_count,
                                          uint32_t next_base, QNode* nodes) {
    if (b + 1 >= n || wide + 1 >= n) return false;  // n - 1 binary and at most n - 1 wide nodes
    for (int h = 0; h < 2; ++h) {
        const uint32_t x = h ? right[b] : left[b];
        if ((x & kLeafBit) ? (x & ~kLeafBit) >= n : x + 1 >= n) return false;
    }
    uint32_t c[4];
    const int nc = wide_children(b, left, right, ibox, c);
    QNode q;
    memset(&q, 0, sizeof(q));
    FBox cb[4];
    for (int i = 0; i < nc; ++i) {
        cb[i] = child_box(c[i], lbox, ibox);
        if ((c[i] & kLeafBit) && (c[i] & ~kLeafBit) >= n) return false;
        if (c[i] & kLeafBit) {
            q.meta[i] = 1;  // a TLAS leaf holds one instance
            q.child[i] = ids[c[i] & ~kLeafBit];
        } else {
#ifdef __CUDA_ARCH__
            const uint32_t pos = atomicAdd(next_count, 1u);
#else
            const uint32_t pos = (*next_count)++;
#endif
            if (pos >= n || c[i] + 1 >= n) return false;
            next[pos] = c[i];
            q.meta[i] = kMetaInner;
            q.child[i] = next_base + pos;
        }
    }
    q.nchild = (uint8_t)nc;
    const bool ok = quantize_node(q, cb, nc);
    nodes[wide] = q;
    return ok;
}

// ---- kernels: one thread per item or node ----------------------------------

__global__ void k_morton(const FBox* boxes, uint32_t n, float cx, float cy, float cz, float sx,
                         float sy, float sz, uint64_t* keys, uint32_t* ids) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float cmin[3] = {cx, cy, cz}, scale[3] = {sx, sy, sz};
    keys[i] = morton_key(boxes[i], cmin, scale);
    ids[i] = i;
}

__global__ void k_radix(const uint64_t* keys, uint32_t n, uint32_t* left, uint32_t* right,
                        uint32_t* parent_int, uint32_t* parent_leaf, uint32_t* failed) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i + 1 >= n) return;  // n - 1 internal nodes
    uint32_t l, r;
    radix_node(keys, n, i, &l, &r);
    if (((l & kLeafBit) ? (l & ~kLeafBit) >= n : l + 1 >= n) ||
        ((r & kLeafBit) ? (r & ~kLeafBit) >= n : r + 1 >= n)) {
        atomicOr(failed, 1u);
        return;
    }
    left[i] = l;
    right[i] = r;
    if (l & kLeafBit) parent_leaf[l & ~kLeafBit] = i; else parent_int[l] = i;
    if (r & kLeafBit) parent_leaf[r & ~kLeafBit] = i; else parent_int[r] = i;
}

__global__ void k_gather(const FBox* boxes, const uint32_t* ids, uint32_t n, FBox* lbox) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) lbox[i] = boxes[ids[i]];
}

__global__ void k_merge(uint32_t n, const uint32_t* parent_leaf, const uint32_t* parent_int,
                        const uint32_t* left, const uint32_t* right, const FBox* lbox, FBox* ibox,
                        uint32_t* arrivals, uint32_t* failed) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n && !merge_up(k, n, parent_leaf, parent_int, left, right, lbox, ibox, arrivals))
        atomicOr(failed, 1u);
}

__global__ void k_collapse(uint32_t n, const uint32_t* cur, uint32_t cur_count, uint32_t cur_base,
                           uint32_t* next, uint32_t* next_count, uint32_t next_base,
                           const uint32_t* left, const uint32_t* right, const FBox* lbox,
                           const FBox* ibox, const uint32_t* ids, QNode* nodes, uint32_t* failed) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cur_count) return;
    if (!emit_wide(cur[t], cur_base + t, n, left, right, lbox, ibox, ids, next, next_count, next_base,
                   nodes))
        atomicOr(failed, 1u);
}

// ---- host side -------------------------------------------------------------

struct Grid {
    float cmin[3], scale[3];
};

// Centre bounds of the items and the scale that maps them onto the 2^21 grid:
// one scale for all three axes (cubic cells), so a flat scene's thin axis does
// not get as many splits as its wide ones (on the mid scene this made the
// tree's render speed 656 instead of 584 Mrays/s, against 678 for SAH).
Grid centre_grid(const std::vector<FBox>& boxes) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (const FBox& b : boxes)
        for (int a = 0; a < 3; ++a) {
            const float c = 0.5f * b.lo[a] + 0.5f * b.hi[a];
            lo[a] = std::min(lo[a], c);
            hi[a] = std::max(hi[a], c);
        }
    Grid g;
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) ext = std::max(ext, (double)hi[a] - (double)lo[a]);
    for (int a = 0; a < 3; ++a) {
        g.cmin[a] = lo[a];
        g.scale[a] = ext > 0.0 ? (float)(2097152.0 / ext) : 0.0f;
    }
    return g;
}

// The per-node functions in host loops (no GPU needed).
bool build_on_host(const std::vector<FBox>& boxes, const Grid& g, TlasResult& out, std::string& err) {
    const uint32_t n = (uint32_t)boxes.size();
    std::vector<std::pair<uint64_t, uint32_t>> kv(n);
    for (uint32_t i = 0; i < n; ++i) kv[i] = {morton_key(boxes[i], g.cmin, g.scale), i};
    std::sort(kv.begin(), kv.end());
    std::vector<uint64_t> keys(n);
    std::vector<uint32_t> ids(n);
    for (uint32_t i = 0; i < n; ++i) {
        keys[i] = kv[i].first;
        ids[i] = kv[i].second;
    }
    std::vector<uint32_t> left(n - 1), right(n - 1), parent_int(n - 1, kNone), parent_leaf(n, kNone);
    for (uint32_t i = 0; i + 1 < n; ++i) {
        radix_node(keys.data(), n, i, &left[i], &right[i]);
        const uint32_t l = left[i], r = right[i];
        if (((l & kLeafBit) ? (l & ~kLeafBit) >= n : l + 1 >= n) ||
            ((r & kLeafBit) ? (r & ~kLeafBit) >= n : r + 1 >= n)) {
            err = "internal: radix tree child out of range";
            return false;
        }
        if (l & kLeafBit) parent_leaf[l & ~kLeafBit] = i; else parent_int[l] = i;
        if (r & kLeafBit) parent_leaf[r & ~kLeafBit] = i; else parent_int[r] = i;
    }
    std::vector<FBox> lbox(n), ibox(n - 1);
    for (uint32_t i = 0; i < n; ++i) lbox[i] = boxes[ids[i]];
    std::vector<uint32_t> arrivals(n - 1, 0);
    for (uint32_t k = 0; k < n; ++k)
        if (!merge_up(k, n, parent_leaf.data(), parent_int.data(), left.data(), right.data(),
                      lbox.data(), ibox.data(), arrivals.data())) {
            err = "internal: radix tree is not a tree";
            return false;
        }
    out.nodes.assign(n - 1, QNode{});
    std::vector<uint32_t> cur{0}, next(n);
    uint32_t base = 0, depth = 0;
    while (!cur.empty()) {
        uint32_t count = 0;
        const uint32_t next_base = base + (uint32_t)cur.size();
        if (next_base > n - 1 || depth >= (uint32_t)kMaxRadixDepth) {
            err = "internal: collapse left the binary tree";
            return false;
        }
        for (uint32_t t = 0; t < cur.size(); ++t)
            if (!emit_wide(cur[t], base + t, n, left.data(), right.data(), lbox.data(), ibox.data(),
                           ids.data(), next.data(), &count, next_base, out.nodes.data())) {
                err = "child boxes cannot be quantised, or the tree is broken";
                return false;
            }
        base = next_base;
        cur.assign(next.begin(), next.begin() + count);
        ++depth;
    }
    out.nodes.resize(base);
    out.depth = depth;
    return true;
}

// Device buffers of one build, freed on every path out.
struct DeviceBuffers {
    std::vector<void*> ptrs;
    ~DeviceBuffers() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <class T>
    cudaError_t alloc(T** p, size_t count) {
        void* v = nullptr;
        const cudaError_t e = cudaMalloc(&v, std::max<size_t>(1, count) * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(v);
        *p = static_cast<T*>(v);
        return e;
    }
};

#define QRT_LBVH_TRY(x)                                                    \
    do {                                                                   \
        const cudaError_t e_ = (x);                                        \
        if (e_ != cudaSuccess) {                                           \
            err = std::string("CUDA: ") + cudaGetErrorString(e_) + " (" #x ")"; \
            return false;                                                  \
        }                                                                  \
    } while (0)

bool build_on_device(const std::vector<FBox>& boxes, const Grid& g, TlasResult& out, std::string& err) {
    const uint32_t n = (uint32_t)boxes.size();
    constexpr int B = 256;
    const unsigned blocks = (n + B - 1) / B;
    DeviceBuffers buf;
    FBox *d_boxes, *d_lbox, *d_ibox;
    uint64_t *d_keys, *d_keys_sorted;
    uint32_t *d_ids, *d_ids_sorted, *d_left, *d_right, *d_pint, *d_pleaf, *d_arrivals;
    uint32_t *d_list[2], *d_counts, *d_failed;
    QNode* d_nodes;
    QRT_LBVH_TRY(buf.alloc(&d_boxes, n));
    QRT_LBVH_TRY(buf.alloc(&d_lbox, n));
    QRT_LBVH_TRY(buf.alloc(&d_ibox, n - 1));
    QRT_LBVH_TRY(buf.alloc(&d_keys, n));
    QRT_LBVH_TRY(buf.alloc(&d_keys_sorted, n));
    QRT_LBVH_TRY(buf.alloc(&d_ids, n));
    QRT_LBVH_TRY(buf.alloc(&d_ids_sorted, n));
    QRT_LBVH_TRY(buf.alloc(&d_left, n - 1));
    QRT_LBVH_TRY(buf.alloc(&d_right, n - 1));
    QRT_LBVH_TRY(buf.alloc(&d_pint, n - 1));
    QRT_LBVH_TRY(buf.alloc(&d_pleaf, n));
    QRT_LBVH_TRY(buf.alloc(&d_arrivals, n - 1));
    QRT_LBVH_TRY(buf.alloc(&d_list[0], n));
    QRT_LBVH_TRY(buf.alloc(&d_list[1], n));
    QRT_LBVH_TRY(buf.alloc(&d_counts, 2));
    QRT_LBVH_TRY(buf.alloc(&d_failed, 1));
    QRT_LBVH_TRY(cudaMemset(d_failed, 0, sizeof(uint32_t)));
    QRT_LBVH_TRY(buf.alloc(&d_nodes, n - 1));
    QRT_LBVH_TRY(cudaMemcpy(d_boxes, boxes.data(), n * sizeof(FBox), cudaMemcpyHostToDevice));

    k_morton<<<blocks, B>>>(d_boxes, n, g.cmin[0], g.cmin[1], g.cmin[2], g.scale[0], g.scale[1],
                            g.scale[2], d_keys, d_ids);
    QRT_LBVH_TRY(cudaGetLastError());
    size_t tmp_bytes = 0;
    QRT_LBVH_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, d_keys, d_keys_sorted, d_ids,
                                                 d_ids_sorted, (int)n, 0, 63));
    void* d_tmp = nullptr;
    QRT_LBVH_TRY(buf.alloc(reinterpret_cast<char**>(&d_tmp), tmp_bytes));
    QRT_LBVH_TRY(cub::DeviceRadixSort::SortPairs(d_tmp, tmp_bytes, d_keys, d_keys_sorted, d_ids,
                                                 d_ids_sorted, (int)n, 0, 63));
    QRT_LBVH_TRY(cudaMemset(d_pint, 0xFF, (n - 1) * sizeof(uint32_t)));
    QRT_LBVH_TRY(cudaMemset(d_pleaf, 0xFF, n * sizeof(uint32_t)));
    QRT_LBVH_TRY(cudaMemset(d_arrivals, 0, (n - 1) * sizeof(uint32_t)));
    k_radix<<<blocks, B>>>(d_keys_sorted, n, d_left, d_right, d_pint, d_pleaf, d_failed);
    QRT_LBVH_TRY(cudaGetLastError());
    k_gather<<<blocks, B>>>(d_boxes, d_ids_sorted, n, d_lbox);
    QRT_LBVH_TRY(cudaGetLastError());
    uint32_t failed = 0;
    QRT_LBVH_TRY(cudaMemcpy(&failed, d_failed, sizeof(failed), cudaMemcpyDeviceToHost));
    if (failed) {
        err = "internal: radix tree child out of range";
        return false;
    }
    k_merge<<<blocks, B>>>(n, d_pleaf, d_pint, d_left, d_right, d_lbox, d_ibox, d_arrivals, d_failed);
    QRT_LBVH_TRY(cudaGetLastError());
    QRT_LBVH_TRY(cudaMemcpy(&failed, d_failed, sizeof(failed), cudaMemcpyDeviceToHost));
    if (failed) {
        err = "internal: radix tree is not a tree";
        return false;
    }

    // top-down collapse, one launch per level of the four-wide tree
    const uint32_t root = 0;
    QRT_LBVH_TRY(cudaMemcpy(d_list[0], &root, sizeof(root), cudaMemcpyHostToDevice));
    uint32_t cur_count = 1, base = 0, depth = 0;
    int side = 0;
    while (cur_count > 0) {
        if (base + cur_count > n - 1 || depth >= (uint32_t)kMaxRadixDepth) {
            err = "internal: collapse produced more nodes than the binary tree has";
            return false;
        }
        const uint32_t next_base = base + cur_count;
        QRT_LBVH_TRY(cudaMemset(d_counts, 0, 2 * sizeof(uint32_t)));
        k_collapse<<<(cur_count + B - 1) / B, B>>>(n, d_list[side], cur_count, base, d_list[side ^ 1],
                                                    d_counts, next_base, d_left, d_right, d_lbox,
                                                    d_ibox, d_ids_sorted, d_nodes, d_counts + 1);
        QRT_LBVH_TRY(cudaGetLastError());
        uint32_t counts[2];
        QRT_LBVH_TRY(cudaMemcpy(counts, d_counts, sizeof(counts), cudaMemcpyDeviceToHost));
        failed |= counts[1];
        base = next_base;
        cur_count = counts[0];
        side ^= 1;
        ++depth;
    }
    if (failed) {
        err = "child boxes cannot be quantised, or the tree is broken";
        return false;
    }
    out.nodes.resize(base);
    QRT_LBVH_TRY(cudaMemcpy(out.nodes.data(), d_nodes, base * sizeof(QNode), cudaMemcpyDeviceToHost));
    out.depth = depth;
    return true;
}

#undef QRT_LBVH_TRY

}  // namespace

bool build_tlas_lbvh(const std::vector<FBox>& inst_boxes, bool on_device, TlasResult& out,
                     std::string& err) {
    out.nodes.clear();
    out.depth = 0;
    const size_t n = inst_boxes.size();
    if (n == 0) return true;
    if (n > kMaxLocalIndex) {
        err = "more than 2^27 instances";
        return false;
    }
    for (const FBox& b : inst_boxes)
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(b.lo[a]) || !std::isfinite(b.hi[a]) || !(b.lo[a] <= b.hi[a])) {
                err = "non-finite or empty instance bounds";
                return false;
            }
    if (n == 1) {  // a root with one leaf
        QNode q;
        std::memset(&q, 0, sizeof(q));
        q.meta[0] = 1;
        q.child[0] = 0;
        q.nchild = 1;
        if (!quantize_node(q, inst_boxes.data(), 1)) {
            err = "child boxes cannot be quantised";
            return false;
        }
        out.nodes.push_back(q);
        out.depth = 1;
        return true;
    }
    const Grid g = centre_grid(inst_boxes);
    return on_device ? build_on_device(inst_boxes, g, out, err) : build_on_host(inst_boxes, g, out, err);
}

}  // namespace qrt

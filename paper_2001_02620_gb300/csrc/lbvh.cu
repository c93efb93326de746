// Linear BVH builds of the TLAS and the BLASes on the GPU (declared in
// lbvh.h).  Every step is a function of one node or one item, written once
// for host and device: the kernels call them per thread, and the host path
// runs the same functions in loops, so the index arithmetic is exercised
// without a GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "lbvh.h"
#include "radix_sort.h"

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
                                           uint32_t* right, uint32_t* range_lo = nullptr,
                                           uint32_t* range_hi = nullptr) {
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
    if (range_lo) *range_lo = (uint32_t)lo;
    if (range_hi) *range_hi = (uint32_t)hi;
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
    char* d_tmp = nullptr;
    QRT_LBVH_TRY(buf.alloc(&d_tmp, sort_pairs_scratch_bytes(n)));
    QRT_LBVH_TRY(sort_pairs(d_keys, d_ids, d_keys_sorted, d_ids_sorted, n, 63, d_tmp, 0));
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

// ---- BLAS: every mesh's tree in one pass ------------------------------------
// All quads are sorted by (mesh, Morton code of the quad centre on the mesh's
// own grid); with the mesh index in the key's top bits each mesh's quads form
// one contiguous range and one subtree of the radix tree, whose root is the
// node covering exactly that range.  Sorted order is slot order, so a subtree
// of at most max_leaf quads is a leaf of contiguous slots.

namespace {

constexpr int kMeshShift = 50;                 // key = mesh << 50 | 48-bit Morton code
constexpr uint32_t kMaxMeshes = 1u << 13;

struct MeshDev {
    uint64_t quad_off;   // first global quad (= first sorted position) of the mesh
    uint64_t vert_off;   // first global vertex
    uint32_t n_quads;
    uint32_t node_off;   // first slot of the mesh's node region (n_quads - 1 slots, at least 1)
    float cmin[3];
    float scale;         // one scale for all axes: cubic cells
};

__host__ __device__ inline FBox quad_box(const float* verts, const uint32_t* quads, uint64_t q,
                                         uint64_t vert_off) {
    FBox b;
    for (int k = 0; k < 4; ++k) {
        const float* v = verts + 3 * (vert_off + quads[4 * q + k]);
        for (int a = 0; a < 3; ++a) {
            b.lo[a] = k ? fminf(b.lo[a], v[a]) : v[a];
            b.hi[a] = k ? fmaxf(b.hi[a], v[a]) : v[a];
        }
    }
    return b;
}

__host__ __device__ inline uint64_t quad_key(const FBox& b, uint32_t m, const MeshDev& md) {
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        const float c = add_rn(mul_rn(0.5f, b.lo[a]), mul_rn(0.5f, b.hi[a]));
        const float u = mul_rn(c - md.cmin[a], md.scale);
        q[a] = u >= 65535.0f ? 65535u : (u > 0.0f ? (uint32_t)u : 0u);
    }
    return ((uint64_t)m << kMeshShift) | (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
}

// Mesh of global quad q (quad_off ascending): binary search.
__host__ __device__ inline uint32_t mesh_of(const MeshDev* md, uint32_t n_mesh, uint64_t q) {
    uint32_t lo = 0, hi = n_mesh;  // md[lo].quad_off <= q < md[hi].quad_off
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (md[mid].quad_off <= q) lo = mid; else hi = mid;
    }
    return lo;
}

// Leaf of a BLAS: a binary leaf, or an internal node over at most max_leaf
// quads; returns its first sorted position and count, or count 0 if c is an
// inner node of the BLAS.
__host__ __device__ inline uint32_t leaf_span(uint32_t c, const uint32_t* rlo, const uint32_t* rhi,
                                              uint32_t max_leaf, uint32_t* first) {
    if (c & kLeafBit) {
        *first = c & ~kLeafBit;
        return 1;
    }
    const uint32_t size = rhi[c] - rlo[c] + 1;
    if (size > max_leaf) return 0;
    *first = rlo[c];
    return size;
}

// Children of the BLAS node made from binary node b (a binary leaf stands for
// a one-quad mesh): as wide_children, but subtrees of at most max_leaf quads
// are leaves and are not opened.
__host__ __device__ inline int blas_children(uint32_t b, const uint32_t* left, const uint32_t* right,
                                             const uint32_t* rlo, const uint32_t* rhi,
                                             uint32_t max_leaf, const FBox* ibox, uint32_t* c) {
    uint32_t f;
    if ((b & kLeafBit) || leaf_span(b, rlo, rhi, max_leaf, &f)) {
        c[0] = b;  // the whole mesh is one leaf
        return 1;
    }
    c[0] = left[b];
    c[1] = right[b];
    int nc = 2;
    while (nc < 4) {
        int best = -1;
        float best_area = -1.0f;
        for (int i = 0; i < nc; ++i) {
            if (leaf_span(c[i], rlo, rhi, max_leaf, &f)) continue;
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

// Writes BLAS node `local` of mesh m (made from binary node b) into the
// mesh's node region; its inner children get the next local indices of the
// mesh (one counter per mesh) and join the next level's list.
__host__ __device__ inline bool emit_blas(uint32_t b, uint32_t m, uint32_t local, uint32_t n,
                                          const MeshDev* md, const uint32_t* left,
                                          const uint32_t* right, const uint32_t* rlo,
                                          const uint32_t* rhi, uint32_t max_leaf, const FBox* lbox,
                                          const FBox* ibox, uint32_t* mesh_nodes, uint32_t* next_b,
                                          uint32_t* next_m, uint32_t* next_w, uint32_t* next_count,
                                          QNode* nodes) {
    const MeshDev& d = md[m];
    const uint32_t cap = d.n_quads > 1 ? d.n_quads - 1 : 1;
    if (local >= cap) return false;
    uint32_t c[4];
    const int nc = blas_children(b, left, right, rlo, rhi, max_leaf, ibox, c);
    QNode q;
    memset(&q, 0, sizeof(q));
    FBox cb[4];
    for (int i = 0; i < nc; ++i) {
        if ((c[i] & kLeafBit) ? (c[i] & ~kLeafBit) >= n : c[i] + 1 >= n) return false;
        cb[i] = child_box(c[i], lbox, ibox);
        uint32_t first;
        const uint32_t cnt = leaf_span(c[i], rlo, rhi, max_leaf, &first);
        if (cnt) {
            if (first < d.quad_off || first + cnt > d.quad_off + d.n_quads) return false;
            q.meta[i] = (uint8_t)cnt;
            q.child[i] = (uint32_t)(first - d.quad_off);  // slot within the mesh
        } else {
#ifdef __CUDA_ARCH__
            const uint32_t w = atomicAdd(mesh_nodes + m, 1u);
            const uint32_t pos = atomicAdd(next_count, 1u);
#else
            const uint32_t w = mesh_nodes[m]++;
            const uint32_t pos = (*next_count)++;
#endif
            if (w >= cap || pos >= n) return false;
            next_b[pos] = c[i];
            next_m[pos] = m;
            next_w[pos] = w;
            q.meta[i] = kMetaInner;
            q.child[i] = w;
        }
    }
    q.nchild = (uint8_t)nc;
    const bool ok = quantize_node(q, cb, nc);
    nodes[d.node_off + local] = q;
    return ok;
}

__global__ void k_quad_keys(const float* verts, const uint32_t* quads, const MeshDev* md,
                            uint32_t n_mesh, uint32_t n, uint64_t* keys, uint32_t* ids) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint32_t m = mesh_of(md, n_mesh, q);
    keys[q] = quad_key(quad_box(verts, quads, q, md[m].vert_off), m, md[m]);
    ids[q] = q;
}

// Sorted position p: the quad's box (for the tree), its vertices in slot
// order and its index within its mesh.
__global__ void k_quad_gather(const float* verts, const uint32_t* quads, const MeshDev* md,
                              uint32_t n_mesh, const uint32_t* ids, uint32_t n, FBox* lbox,
                              QuadDev* out_quads, uint32_t* out_prim) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t q = ids[p];
    const uint32_t m = mesh_of(md, n_mesh, q);
    lbox[p] = quad_box(verts, quads, q, md[m].vert_off);
    QuadDev o;
    for (int k = 0; k < 4; ++k) {
        const float* v = verts + 3 * (md[m].vert_off + quads[4 * (uint64_t)q + k]);
        o.v[3 * k] = v[0];
        o.v[3 * k + 1] = v[1];
        o.v[3 * k + 2] = v[2];
    }
    out_quads[p] = o;
    out_prim[p] = (uint32_t)(q - md[m].quad_off);
}

__global__ void k_radix_blas(const uint64_t* keys, uint32_t n, const MeshDev* md, uint32_t* left,
                             uint32_t* right, uint32_t* rlo, uint32_t* rhi, uint32_t* parent_int,
                             uint32_t* parent_leaf, uint32_t* roots, uint32_t* failed) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i + 1 >= n) return;
    uint32_t l, r, lo, hi;
    radix_node(keys, n, i, &l, &r, &lo, &hi);
    if (((l & kLeafBit) ? (l & ~kLeafBit) >= n : l + 1 >= n) ||
        ((r & kLeafBit) ? (r & ~kLeafBit) >= n : r + 1 >= n) || lo >= n || hi >= n) {
        atomicOr(failed, 1u);
        return;
    }
    left[i] = l;
    right[i] = r;
    rlo[i] = lo;
    rhi[i] = hi;
    if (l & kLeafBit) parent_leaf[l & ~kLeafBit] = i; else parent_int[l] = i;
    if (r & kLeafBit) parent_leaf[r & ~kLeafBit] = i; else parent_int[r] = i;
    const uint32_t m = (uint32_t)(keys[lo] >> kMeshShift);
    if ((uint32_t)(keys[hi] >> kMeshShift) == m && lo == md[m].quad_off &&
        hi + 1 == md[m].quad_off + md[m].n_quads)
        roots[m] = i;
}

__global__ void k_collapse_blas(uint32_t n, const MeshDev* md, const uint32_t* cur_b,
                                const uint32_t* cur_m, const uint32_t* cur_w, uint32_t cur_count,
                                uint32_t* next_b, uint32_t* next_m, uint32_t* next_w,
                                uint32_t* next_count, const uint32_t* left, const uint32_t* right,
                                const uint32_t* rlo, const uint32_t* rhi, uint32_t max_leaf,
                                const FBox* lbox, const FBox* ibox, uint32_t* mesh_nodes,
                                uint32_t* mesh_depth, uint32_t level, QNode* nodes, uint32_t* failed) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cur_count) return;
    const uint32_t m = cur_m[t];
    atomicMax(mesh_depth + m, level + 1);
    if (!emit_blas(cur_b[t], m, cur_w[t], n, md, left, right, rlo, rhi, max_leaf, lbox, ibox,
                   mesh_nodes, next_b, next_m, next_w, next_count, nodes))
        atomicOr(failed, 1u);
}

}  // namespace

namespace {

// fn(i) for i in [0, n) on all host cores (items claimed one at a time).
template <class Fn>
void parallel_for(size_t n, Fn fn) {
    const unsigned nt = (unsigned)std::min<size_t>(n, std::max(1u, std::thread::hardware_concurrency()));
    std::atomic<size_t> next{0};
    auto work = [&]() {
        for (size_t i; (i = next.fetch_add(1)) < n;) fn(i);
    };
    std::vector<std::thread> th;
    for (unsigned k = 1; k < nt; ++k) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
}

// Mesh table: offsets, node regions and each mesh's Morton grid (the box of
// its referenced vertices, one scale for all axes).  Also checks the input
// as the host builder does; meshes are scanned in parallel.
bool mesh_table(const std::vector<MeshView>& meshes, std::vector<MeshDev>& md, uint64_t& total_q,
                uint64_t& total_v, std::string& err) {
    md.resize(meshes.size());
    total_q = total_v = 0;
    uint64_t nodes = 0;
    std::vector<std::string> errs(meshes.size());
    std::vector<FBox> vbox(meshes.size());
    parallel_for(meshes.size(), [&](size_t m) {
        const MeshView& mv = meshes[m];
        if (mv.n_quads == 0) {
            errs[m] = "mesh has no quads";
            return;
        }
        if (mv.n_quads > kMaxLocalIndex) {
            errs[m] = "mesh has more than 2^27 quads";
            return;
        }
        FBox b{{INFINITY, INFINITY, INFINITY}, {-INFINITY, -INFINITY, -INFINITY}};
        for (uint64_t k = 0; k < 4ull * mv.n_quads; ++k) {
            const uint32_t vi = mv.quads[k];
            if (vi >= mv.n_verts) {
                errs[m] = "quad vertex index out of range";
                return;
            }
            const float* v = mv.verts + 3 * (size_t)vi;
            for (int a = 0; a < 3; ++a) {
                if (!std::isfinite(v[a])) {
                    errs[m] = "non-finite vertex";
                    return;
                }
                b.lo[a] = std::min(b.lo[a], v[a]);
                b.hi[a] = std::max(b.hi[a], v[a]);
            }
        }
        vbox[m] = b;
    });
    for (size_t m = 0; m < meshes.size(); ++m) {
        if (!errs[m].empty()) {
            err = "mesh " + std::to_string(m) + ": " + errs[m];
            return false;
        }
        const MeshView& mv = meshes[m];
        const float* lo = vbox[m].lo;
        const float* hi = vbox[m].hi;
        MeshDev& d = md[m];
        d.quad_off = total_q;
        d.vert_off = total_v;
        d.n_quads = mv.n_quads;
        d.node_off = (uint32_t)nodes;
        double ext = 0.0;
        for (int a = 0; a < 3; ++a) {
            d.cmin[a] = lo[a];
            ext = std::max(ext, (double)hi[a] - (double)lo[a]);
        }
        d.scale = ext > 0.0 ? (float)(65536.0 / ext) : 0.0f;
        total_q += mv.n_quads;
        total_v += mv.n_verts;
        nodes += mv.n_quads > 1 ? mv.n_quads - 1 : 1;
    }
    if (total_q >= 0x7FFFFFFFull || nodes >= 0xFFFFFFFFull) {
        err = "more than 2^31 quads in all meshes";
        return false;
    }
    return true;
}

// Exact box of the vertices of a mesh's quads.
FBox quads_box(const std::vector<QuadDev>& quads) {
    FBox b{{INFINITY, INFINITY, INFINITY}, {-INFINITY, -INFINITY, -INFINITY}};
    for (const QuadDev& q : quads)
        for (int k = 0; k < 4; ++k)
            for (int a = 0; a < 3; ++a) {
                b.lo[a] = std::min(b.lo[a], q.v[3 * k + a]);
                b.hi[a] = std::max(b.hi[a], q.v[3 * k + a]);
            }
    return b;
}

// Splits the per-mesh results out of the global arrays.
void split_blases(const std::vector<MeshDev>& md, const std::vector<QNode>& nodes,
                  const std::vector<uint32_t>& mesh_nodes, const std::vector<uint32_t>& mesh_depth,
                  const std::vector<QuadDev>& quads, const std::vector<uint32_t>& prim,
                  std::vector<BlasResult>& out) {
    out.resize(md.size());
    for (size_t m = 0; m < md.size(); ++m) {
        BlasResult& r = out[m];
        const MeshDev& d = md[m];
        r.nodes.assign(nodes.begin() + d.node_off, nodes.begin() + d.node_off + mesh_nodes[m]);
        r.quads.assign(quads.begin() + d.quad_off, quads.begin() + d.quad_off + d.n_quads);
        r.prim.assign(prim.begin() + d.quad_off, prim.begin() + d.quad_off + d.n_quads);
        r.depth = mesh_depth[m];
        r.box = quads_box(r.quads);
    }
}

bool blases_on_host(const std::vector<MeshView>& meshes, const std::vector<MeshDev>& md,
                    uint32_t n, uint32_t max_leaf, std::vector<BlasResult>& out, std::string& err) {
    const uint32_t n_mesh = (uint32_t)md.size();
    std::vector<float> verts;
    std::vector<uint32_t> quads;
    for (const MeshView& mv : meshes) {
        verts.insert(verts.end(), mv.verts, mv.verts + 3 * (size_t)mv.n_verts);
        quads.insert(quads.end(), mv.quads, mv.quads + 4 * (size_t)mv.n_quads);
    }
    std::vector<std::pair<uint64_t, uint32_t>> kv(n);
    for (uint32_t q = 0; q < n; ++q) {
        const uint32_t m = mesh_of(md.data(), n_mesh, q);
        kv[q] = {quad_key(quad_box(verts.data(), quads.data(), q, md[m].vert_off), m, md[m]), q};
    }
    std::sort(kv.begin(), kv.end());
    std::vector<uint64_t> keys(n);
    std::vector<uint32_t> ids(n);
    for (uint32_t p = 0; p < n; ++p) {
        keys[p] = kv[p].first;
        ids[p] = kv[p].second;
    }
    std::vector<FBox> lbox(n);
    std::vector<QuadDev> oq(n);
    std::vector<uint32_t> prim(n);
    for (uint32_t p = 0; p < n; ++p) {
        const uint32_t q = ids[p], m = mesh_of(md.data(), n_mesh, q);
        lbox[p] = quad_box(verts.data(), quads.data(), q, md[m].vert_off);
        for (int k = 0; k < 4; ++k)
            for (int a = 0; a < 3; ++a)
                oq[p].v[3 * k + a] = verts[3 * (md[m].vert_off + quads[4 * (uint64_t)q + k]) + a];
        prim[p] = (uint32_t)(q - md[m].quad_off);
    }
    const uint32_t ni = n > 1 ? n - 1 : 1;
    std::vector<uint32_t> left(ni), right(ni), rlo(ni), rhi(ni), pint(ni, kNone), pleaf(n, kNone);
    std::vector<uint32_t> roots(n_mesh, kNone);
    for (uint32_t m = 0; m < n_mesh; ++m)
        if (md[m].n_quads == 1) roots[m] = kLeafBit | (uint32_t)md[m].quad_off;
    for (uint32_t i = 0; i + 1 < n; ++i) {
        uint32_t l, r, lo, hi;
        radix_node(keys.data(), n, i, &l, &r, &lo, &hi);
        if (((l & kLeafBit) ? (l & ~kLeafBit) >= n : l + 1 >= n) ||
            ((r & kLeafBit) ? (r & ~kLeafBit) >= n : r + 1 >= n) || lo >= n || hi >= n) {
            err = "internal: radix tree child out of range";
            return false;
        }
        left[i] = l;
        right[i] = r;
        rlo[i] = lo;
        rhi[i] = hi;
        if (l & kLeafBit) pleaf[l & ~kLeafBit] = i; else pint[l] = i;
        if (r & kLeafBit) pleaf[r & ~kLeafBit] = i; else pint[r] = i;
        const uint32_t m = (uint32_t)(keys[lo] >> kMeshShift);
        if ((uint32_t)(keys[hi] >> kMeshShift) == m && lo == md[m].quad_off &&
            hi + 1 == md[m].quad_off + md[m].n_quads)
            roots[m] = i;
    }
    std::vector<FBox> ibox(ni);
    std::vector<uint32_t> arrivals(ni, 0);
    for (uint32_t k = 0; k < n; ++k)
        if (!merge_up(k, n, pleaf.data(), pint.data(), left.data(), right.data(), lbox.data(),
                      ibox.data(), arrivals.data())) {
            err = "internal: radix tree is not a tree";
            return false;
        }
    uint64_t node_slots = 0;
    for (const MeshDev& d : md) node_slots += d.n_quads > 1 ? d.n_quads - 1 : 1;
    std::vector<QNode> nodes(node_slots);
    std::vector<uint32_t> mesh_nodes(n_mesh, 1), mesh_depth(n_mesh, 0);
    std::vector<uint32_t> cb, cm, cw, nb(n), nm(n), nw(n);
    for (uint32_t m = 0; m < n_mesh; ++m) {
        if (roots[m] == kNone) {
            err = "internal: mesh " + std::to_string(m) + " has no subtree";
            return false;
        }
        cb.push_back(roots[m]);
        cm.push_back(m);
        cw.push_back(0);
    }
    for (uint32_t level = 0; !cb.empty(); ++level) {
        if (level >= (uint32_t)kMaxRadixDepth) {
            err = "internal: collapse left the binary tree";
            return false;
        }
        uint32_t count = 0;
        for (size_t t = 0; t < cb.size(); ++t) {
            mesh_depth[cm[t]] = std::max(mesh_depth[cm[t]], level + 1);
            if (!emit_blas(cb[t], cm[t], cw[t], n, md.data(), left.data(), right.data(), rlo.data(),
                           rhi.data(), max_leaf, lbox.data(), ibox.data(), mesh_nodes.data(),
                           nb.data(), nm.data(), nw.data(), &count, nodes.data())) {
                err = "child boxes cannot be quantised, or the tree is broken";
                return false;
            }
        }
        cb.assign(nb.begin(), nb.begin() + count);
        cm.assign(nm.begin(), nm.begin() + count);
        cw.assign(nw.begin(), nw.begin() + count);
    }
    split_blases(md, nodes, mesh_nodes, mesh_depth, oq, prim, out);
    return true;
}

}  // namespace

namespace {

#define QRT_LBVH_TRY(x)                                                         \
    do {                                                                        \
        const cudaError_t e_ = (x);                                             \
        if (e_ != cudaSuccess) {                                                \
            err = std::string("CUDA: ") + cudaGetErrorString(e_) + " (" #x ")"; \
            return false;                                                       \
        }                                                                       \
    } while (0)

bool blases_on_device(const std::vector<MeshView>& meshes, const std::vector<MeshDev>& md,
                      uint64_t total_v, uint32_t n, uint32_t max_leaf, std::vector<BlasResult>& out,
                      std::string& err) {
    const uint32_t n_mesh = (uint32_t)md.size();
    constexpr int B = 256;
    const unsigned blocks = (n + B - 1) / B;
    const uint32_t ni = n > 1 ? n - 1 : 1;
    uint64_t node_slots = 0;
    for (const MeshDev& d : md) node_slots += d.n_quads > 1 ? d.n_quads - 1 : 1;
    DeviceBuffers buf;
    float* d_verts;
    uint32_t *d_quads, *d_ids, *d_ids_sorted, *d_prim, *d_left, *d_right, *d_rlo, *d_rhi, *d_pint,
        *d_pleaf, *d_arrivals, *d_roots, *d_mesh_nodes, *d_mesh_depth, *d_counts, *d_failed;
    uint32_t *d_lb[2], *d_lm[2], *d_lw[2];
    uint64_t *d_keys, *d_keys_sorted;
    FBox *d_lbox, *d_ibox;
    QuadDev* d_oq;
    QNode* d_nodes;
    MeshDev* d_md;
    QRT_LBVH_TRY(buf.alloc(&d_verts, 3 * total_v));
    QRT_LBVH_TRY(buf.alloc(&d_quads, 4 * (uint64_t)n));
    QRT_LBVH_TRY(buf.alloc(&d_md, n_mesh));
    for (uint32_t m = 0; m < n_mesh; ++m) {
        QRT_LBVH_TRY(cudaMemcpy(d_verts + 3 * md[m].vert_off, meshes[m].verts,
                                12 * (size_t)meshes[m].n_verts, cudaMemcpyHostToDevice));
        QRT_LBVH_TRY(cudaMemcpy(d_quads + 4 * md[m].quad_off, meshes[m].quads,
                                16 * (size_t)meshes[m].n_quads, cudaMemcpyHostToDevice));
    }
    QRT_LBVH_TRY(cudaMemcpy(d_md, md.data(), n_mesh * sizeof(MeshDev), cudaMemcpyHostToDevice));
    QRT_LBVH_TRY(buf.alloc(&d_keys, n));
    QRT_LBVH_TRY(buf.alloc(&d_keys_sorted, n));
    QRT_LBVH_TRY(buf.alloc(&d_ids, n));
    QRT_LBVH_TRY(buf.alloc(&d_ids_sorted, n));
    QRT_LBVH_TRY(buf.alloc(&d_prim, n));
    QRT_LBVH_TRY(buf.alloc(&d_lbox, n));
    QRT_LBVH_TRY(buf.alloc(&d_oq, n));
    QRT_LBVH_TRY(buf.alloc(&d_ibox, ni));
    QRT_LBVH_TRY(buf.alloc(&d_left, ni));
    QRT_LBVH_TRY(buf.alloc(&d_right, ni));
    QRT_LBVH_TRY(buf.alloc(&d_rlo, ni));
    QRT_LBVH_TRY(buf.alloc(&d_rhi, ni));
    QRT_LBVH_TRY(buf.alloc(&d_pint, ni));
    QRT_LBVH_TRY(buf.alloc(&d_pleaf, n));
    QRT_LBVH_TRY(buf.alloc(&d_arrivals, ni));
    QRT_LBVH_TRY(buf.alloc(&d_roots, n_mesh));
    QRT_LBVH_TRY(buf.alloc(&d_mesh_nodes, n_mesh));
    QRT_LBVH_TRY(buf.alloc(&d_mesh_depth, n_mesh));
    QRT_LBVH_TRY(buf.alloc(&d_counts, 1));
    QRT_LBVH_TRY(buf.alloc(&d_failed, 1));
    for (int k = 0; k < 2; ++k) {
        QRT_LBVH_TRY(buf.alloc(&d_lb[k], n));
        QRT_LBVH_TRY(buf.alloc(&d_lm[k], n));
        QRT_LBVH_TRY(buf.alloc(&d_lw[k], n));
    }
    QRT_LBVH_TRY(buf.alloc(&d_nodes, node_slots));
    QRT_LBVH_TRY(cudaMemset(d_failed, 0, 4));

    k_quad_keys<<<blocks, B>>>(d_verts, d_quads, d_md, n_mesh, n, d_keys, d_ids);
    QRT_LBVH_TRY(cudaGetLastError());
    char* d_tmp = nullptr;
    QRT_LBVH_TRY(buf.alloc(&d_tmp, sort_pairs_scratch_bytes(n)));
    QRT_LBVH_TRY(sort_pairs(d_keys, d_ids, d_keys_sorted, d_ids_sorted, n, 63, d_tmp, 0));
    k_quad_gather<<<blocks, B>>>(d_verts, d_quads, d_md, n_mesh, d_ids_sorted, n, d_lbox, d_oq, d_prim);
    QRT_LBVH_TRY(cudaGetLastError());
    std::vector<uint32_t> roots(n_mesh, kNone);
    for (uint32_t m = 0; m < n_mesh; ++m)
        if (md[m].n_quads == 1) roots[m] = kLeafBit | (uint32_t)md[m].quad_off;
    QRT_LBVH_TRY(cudaMemcpy(d_roots, roots.data(), 4 * (size_t)n_mesh, cudaMemcpyHostToDevice));
    QRT_LBVH_TRY(cudaMemset(d_pint, 0xFF, 4 * (size_t)ni));
    QRT_LBVH_TRY(cudaMemset(d_pleaf, 0xFF, 4 * (size_t)n));
    QRT_LBVH_TRY(cudaMemset(d_arrivals, 0, 4 * (size_t)ni));
    uint32_t failed = 0;
    if (n > 1) {
        k_radix_blas<<<blocks, B>>>(d_keys_sorted, n, d_md, d_left, d_right, d_rlo, d_rhi, d_pint,
                                    d_pleaf, d_roots, d_failed);
        QRT_LBVH_TRY(cudaGetLastError());
        QRT_LBVH_TRY(cudaMemcpy(&failed, d_failed, 4, cudaMemcpyDeviceToHost));
        if (failed) {
            err = "internal: radix tree child out of range";
            return false;
        }
        k_merge<<<blocks, B>>>(n, d_pleaf, d_pint, d_left, d_right, d_lbox, d_ibox, d_arrivals, d_failed);
        QRT_LBVH_TRY(cudaGetLastError());
        QRT_LBVH_TRY(cudaMemcpy(&failed, d_failed, 4, cudaMemcpyDeviceToHost));
        if (failed) {
            err = "internal: radix tree is not a tree";
            return false;
        }
    }
    QRT_LBVH_TRY(cudaMemcpy(roots.data(), d_roots, 4 * (size_t)n_mesh, cudaMemcpyDeviceToHost));
    std::vector<uint32_t> cm(n_mesh), cw(n_mesh, 0), ones(n_mesh, 1);
    for (uint32_t m = 0; m < n_mesh; ++m) {
        if (roots[m] == kNone) {
            err = "internal: mesh " + std::to_string(m) + " has no subtree";
            return false;
        }
        cm[m] = m;
    }
    QRT_LBVH_TRY(cudaMemcpy(d_lb[0], roots.data(), 4 * (size_t)n_mesh, cudaMemcpyHostToDevice));
    QRT_LBVH_TRY(cudaMemcpy(d_lm[0], cm.data(), 4 * (size_t)n_mesh, cudaMemcpyHostToDevice));
    QRT_LBVH_TRY(cudaMemcpy(d_lw[0], cw.data(), 4 * (size_t)n_mesh, cudaMemcpyHostToDevice));
    QRT_LBVH_TRY(cudaMemcpy(d_mesh_nodes, ones.data(), 4 * (size_t)n_mesh, cudaMemcpyHostToDevice));
    QRT_LBVH_TRY(cudaMemset(d_mesh_depth, 0, 4 * (size_t)n_mesh));
    uint32_t cur_count = n_mesh;
    int side = 0;
    for (uint32_t level = 0; cur_count > 0; ++level) {
        if (level >= (uint32_t)kMaxRadixDepth) {
            err = "internal: collapse left the binary tree";
            return false;
        }
        QRT_LBVH_TRY(cudaMemset(d_counts, 0, 4));
        k_collapse_blas<<<(cur_count + B - 1) / B, B>>>(
            n, d_md, d_lb[side], d_lm[side], d_lw[side], cur_count, d_lb[side ^ 1], d_lm[side ^ 1],
            d_lw[side ^ 1], d_counts, d_left, d_right, d_rlo, d_rhi, max_leaf, d_lbox, d_ibox,
            d_mesh_nodes, d_mesh_depth, level, d_nodes, d_failed);
        QRT_LBVH_TRY(cudaGetLastError());
        QRT_LBVH_TRY(cudaMemcpy(&cur_count, d_counts, 4, cudaMemcpyDeviceToHost));
        side ^= 1;
    }
    QRT_LBVH_TRY(cudaMemcpy(&failed, d_failed, 4, cudaMemcpyDeviceToHost));
    if (failed) {
        err = "child boxes cannot be quantised, or the tree is broken";
        return false;
    }
    // each mesh's used nodes, quads and indices straight into its result
    std::vector<uint32_t> mesh_nodes(n_mesh), mesh_depth(n_mesh);
    QRT_LBVH_TRY(cudaMemcpy(mesh_nodes.data(), d_mesh_nodes, 4 * (size_t)n_mesh, cudaMemcpyDeviceToHost));
    QRT_LBVH_TRY(cudaMemcpy(mesh_depth.data(), d_mesh_depth, 4 * (size_t)n_mesh, cudaMemcpyDeviceToHost));
    out.resize(n_mesh);
    for (uint32_t m = 0; m < n_mesh; ++m) {
        const MeshDev& d = md[m];
        BlasResult& r = out[m];
        const uint32_t cap = d.n_quads > 1 ? d.n_quads - 1 : 1;
        if (mesh_nodes[m] > cap) {
            err = "internal: mesh node region overflow";
            return false;
        }
        r.nodes.resize(mesh_nodes[m]);
        r.quads.resize(d.n_quads);
        r.prim.resize(d.n_quads);
        QRT_LBVH_TRY(cudaMemcpy(r.nodes.data(), d_nodes + d.node_off, mesh_nodes[m] * sizeof(QNode),
                                cudaMemcpyDeviceToHost));
        QRT_LBVH_TRY(cudaMemcpy(r.quads.data(), d_oq + d.quad_off, d.n_quads * sizeof(QuadDev),
                                cudaMemcpyDeviceToHost));
        QRT_LBVH_TRY(cudaMemcpy(r.prim.data(), d_prim + d.quad_off, 4 * (size_t)d.n_quads,
                                cudaMemcpyDeviceToHost));
        r.depth = mesh_depth[m];
    }
    parallel_for(n_mesh, [&](size_t m) { out[m].box = quads_box(out[m].quads); });
    return true;
}

#undef QRT_LBVH_TRY

}  // namespace

bool build_blases_lbvh(const std::vector<MeshView>& meshes, uint32_t max_leaf, bool on_device,
                       std::vector<BlasResult>& out, std::string& err) {
    out.clear();
    if (meshes.empty()) return true;
    if (meshes.size() > kMaxMeshes) {
        err = "the linear BLAS build takes at most 8192 meshes";
        return false;
    }
    if (max_leaf < 1 || max_leaf > kMaxLeaf) {
        err = "max_leaf out of range";
        return false;
    }
    std::vector<MeshDev> md;
    uint64_t total_q = 0, total_v = 0;
    if (!mesh_table(meshes, md, total_q, total_v, err)) return false;
    return on_device ? blases_on_device(meshes, md, total_v, (uint32_t)total_q, max_leaf, out, err)
                     : blases_on_host(meshes, md, (uint32_t)total_q, max_leaf, out, err);
}

}  // namespace qrt

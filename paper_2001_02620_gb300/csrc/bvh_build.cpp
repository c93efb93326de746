// Host BVH builder (see bvh_build.h).  Binned SAH on item centroids, leaves of
// up to max_leaf items, collapsed greedily to four children per node (the
// child with the largest surface area is opened first), child boxes quantised
// to 8 bits per plane against a power-of-two grid anchored at the node's lower
// corner and widened until the dequantised box contains the exact one.
#include "bvh_build.h"

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <limits>
#include <thread>

namespace qrt {
namespace {

const float kFInf = std::numeric_limits<float>::infinity();

void box_empty(FBox& b) {
    for (int a = 0; a < 3; ++a) {
        b.lo[a] = kFInf;
        b.hi[a] = -kFInf;
    }
}
void box_grow(FBox& b, const FBox& c) {
    for (int a = 0; a < 3; ++a) {
        b.lo[a] = std::min(b.lo[a], c.lo[a]);
        b.hi[a] = std::max(b.hi[a], c.hi[a]);
    }
}
double box_area(const FBox& b) {
    if (b.lo[0] > b.hi[0]) return 0.0;
    double dx = (double)b.hi[0] - b.lo[0], dy = (double)b.hi[1] - b.lo[1],
           dz = (double)b.hi[2] - b.lo[2];
    return 2.0 * (dx * dy + dy * dz + dz * dx);
}

struct BinNode {
    FBox box;
    int32_t left = -1, right = -1;
    uint32_t first = 0, count = 0;  // leaf when left < 0
};

struct Centroid {
    float c[3];
};

// Helper threads that binary builds may start, shared by all builds running
// at once (the BLAS builds of one scene run concurrently, one per core).
std::atomic<int> g_helpers{0};

// Binned-SAH binary build over items [0, n); ids receives the leaf order.
// Subtrees of at least kForkItems items may be handed to a helper thread
// while fewer than max_helpers helpers run.  Node slots are allocated
// atomically, so their numbering depends on thread timing, but the tree --
// every split, and the four-wide tree collapsed from it by following child
// links from the root -- does not.
class BinaryBuilder {
  public:
    static constexpr uint32_t kForkItems = 1u << 15;

    BinaryBuilder(const std::vector<FBox>& boxes, std::vector<uint32_t>& ids, uint32_t max_leaf,
                  uint32_t bins, std::vector<BinNode>& nodes, int max_helpers)
        : boxes_(boxes), ids_(ids), max_leaf_(max_leaf), bins_(bins), nodes_(nodes),
          max_helpers_(max_helpers) {}

    void build() {
        const uint32_t n = (uint32_t)boxes_.size();
        ids_.resize(n);
        cen_.resize(n);
        for (uint32_t i = 0; i < n; ++i) {
            ids_[i] = i;
            for (int a = 0; a < 3; ++a) cen_[i].c[a] = 0.5f * boxes_[i].lo[a] + 0.5f * boxes_[i].hi[a];
        }
        nodes_.assign(2 * (size_t)std::max(1u, n), BinNode{});  // a binary tree has < 2n nodes
        next_.store(1);
        run(Task{0, 0, n});
        nodes_.resize(next_.load());
    }

  private:
    struct Task {
        int32_t node;
        uint32_t first, count;
    };

    void run(Task root) {
        std::vector<Task> work{root};
        std::vector<std::thread> helpers;
        std::vector<uint32_t> bcnt(bins_);
        std::vector<FBox> bbox(bins_);
        std::vector<double> right_area(bins_);
        std::vector<uint32_t> right_cnt(bins_);
        std::vector<uint32_t> bcnt3(3 * bins_);
        std::vector<FBox> bbox3(3 * bins_);
        while (!work.empty()) {
            Task tk = work.back();
            work.pop_back();
            FBox b, cb;
            bounds(tk.first, tk.first + tk.count, b, cb);
            nodes_[tk.node].box = b;
            if (tk.count <= max_leaf_) {
                nodes_[tk.node].first = tk.first;
                nodes_[tk.node].count = tk.count;
                continue;
            }
            int best_axis = -1;
            uint32_t best_split = 0;
            double best_cost = std::numeric_limits<double>::infinity();
            double scale3[3];
            for (int a = 0; a < 3; ++a) {
                const double ext = (double)cb.hi[a] - cb.lo[a];
                scale3[a] = ext > 0.0 ? (double)bins_ / ext : 0.0;
            }
            bin3(tk.first, tk.first + tk.count, cb, scale3, bcnt3, bbox3);
            for (int a = 0; a < 3; ++a) {
                if (!(scale3[a] > 0.0)) continue;
                std::copy(bcnt3.begin() + a * bins_, bcnt3.begin() + (a + 1) * bins_, bcnt.begin());
                std::copy(bbox3.begin() + a * bins_, bbox3.begin() + (a + 1) * bins_, bbox.begin());
                FBox acc;
                box_empty(acc);
                uint32_t cnt = 0;
                for (int bi = (int)bins_ - 1; bi >= 1; --bi) {
                    box_grow(acc, bbox[bi]);
                    cnt += bcnt[bi];
                    right_area[bi] = box_area(acc);
                    right_cnt[bi] = cnt;
                }
                box_empty(acc);
                cnt = 0;
                for (uint32_t sp = 0; sp + 1 < bins_; ++sp) {  // left = bins [0, sp]
                    box_grow(acc, bbox[sp]);
                    cnt += bcnt[sp];
                    uint32_t rc = right_cnt[sp + 1];
                    if (cnt == 0 || rc == 0) continue;
                    double cost = box_area(acc) * cnt + right_area[sp + 1] * rc;
                    if (cost < best_cost) {
                        best_cost = cost;
                        best_axis = a;
                        best_split = sp;
                    }
                }
            }
            uint32_t mid;
            if (best_axis < 0) {
                mid = tk.first + tk.count / 2;  // all centroids coincide: split by count
            } else {
                double ext = (double)cb.hi[best_axis] - cb.lo[best_axis];
                double scale = (double)bins_ / ext;
                float lo = cb.lo[best_axis];
                auto it = std::partition(ids_.begin() + tk.first, ids_.begin() + tk.first + tk.count,
                                         [&](uint32_t i) {
                                             int bi = (int)(((double)cen_[i].c[best_axis] - lo) * scale);
                                             bi = std::min(std::max(bi, 0), (int)bins_ - 1);
                                             return (uint32_t)bi <= best_split;
                                         });
                mid = (uint32_t)(it - ids_.begin());
                if (mid == tk.first || mid == tk.first + tk.count) mid = tk.first + tk.count / 2;
            }
            const int32_t l = (int32_t)next_.fetch_add(2);
            nodes_[tk.node].left = l;
            nodes_[tk.node].right = l + 1;
            const Task kids[2] = {Task{l + 1, mid, tk.first + tk.count - mid},
                                  Task{l, tk.first, mid - tk.first}};
            for (const Task& c : kids) {
                if (c.count >= kForkItems && take_helper()) {
                    helpers.emplace_back([this, c] {
                        run(c);
                        g_helpers.fetch_sub(1);
                    });
                } else {
                    work.push_back(c);
                }
            }
        }
        for (std::thread& t : helpers) t.join();
    }

    // Items [k0, k1) split into chunks processed on threads when the range is
    // large (the first splits of a big tree would otherwise be one long
    // sequential pass each); merging counts and min/max boxes is exact, so
    // the result does not depend on the chunking.
    static constexpr uint32_t kParItems = 1u << 20;

    template <class F>
    void chunks(uint32_t k0, uint32_t k1, F f) {
        const uint32_t n = k1 - k0;
        const int nt = n >= kParItems ? std::max(1, max_helpers_) : 1;
        if (nt == 1) {
            f(0, k0, k1);
            return;
        }
        std::vector<std::thread> th;
        const uint32_t step = (n + nt - 1) / nt;
        for (int t = 1; t < nt; ++t) {
            const uint32_t a = k0 + std::min(n, t * step), b = k0 + std::min(n, (t + 1) * step);
            th.emplace_back([&f, t, a, b] { f(t, a, b); });
        }
        f(0, k0, k0 + std::min(n, step));
        for (std::thread& x : th) x.join();
    }

    void bounds(uint32_t k0, uint32_t k1, FBox& b, FBox& cb) {
        const int nt = (k1 - k0) >= kParItems ? std::max(1, max_helpers_) : 1;
        std::vector<FBox> pb(nt), pc(nt);
        for (int t = 0; t < nt; ++t) {
            box_empty(pb[t]);
            box_empty(pc[t]);
        }
        chunks(k0, k1, [&](int t, uint32_t a, uint32_t e) {
            for (uint32_t k = a; k < e; ++k) {
                box_grow(pb[t], boxes_[ids_[k]]);
                const Centroid& c = cen_[ids_[k]];
                FBox p{{c.c[0], c.c[1], c.c[2]}, {c.c[0], c.c[1], c.c[2]}};
                box_grow(pc[t], p);
            }
        });
        box_empty(b);
        box_empty(cb);
        for (int t = 0; t < nt; ++t) {
            box_grow(b, pb[t]);
            box_grow(cb, pc[t]);
        }
    }

    // Bins every item once for all three axes (axes with scale 0 are
    // skipped): one gather of its box and centroid per item and pass.
    void bin3(uint32_t k0, uint32_t k1, const FBox& cb, const double* scale, std::vector<uint32_t>& bcnt,
              std::vector<FBox>& bbox) {
        const int nt = (k1 - k0) >= kParItems ? std::max(1, max_helpers_) : 1;
        const uint32_t nb = 3 * bins_;
        std::vector<std::vector<uint32_t>> pc(nt, std::vector<uint32_t>(nb, 0u));
        std::vector<std::vector<FBox>> pb(nt, std::vector<FBox>(nb));
        for (auto& v : pb)
            for (auto& x : v) box_empty(x);
        chunks(k0, k1, [&](int t, uint32_t s, uint32_t e) {
            uint32_t* cnt = pc[t].data();
            FBox* bx = pb[t].data();
            for (uint32_t k = s; k < e; ++k) {
                const uint32_t i = ids_[k];
                const FBox& box = boxes_[i];
                const Centroid& c = cen_[i];
                for (int a = 0; a < 3; ++a) {
                    if (!(scale[a] > 0.0)) continue;
                    int bi = (int)(((double)c.c[a] - cb.lo[a]) * scale[a]);
                    bi = std::min(std::max(bi, 0), (int)bins_ - 1);
                    cnt[a * bins_ + bi]++;
                    box_grow(bx[a * bins_ + bi], box);
                }
            }
        });
        std::fill(bcnt.begin(), bcnt.end(), 0u);
        for (auto& x : bbox) box_empty(x);
        for (int t = 0; t < nt; ++t)
            for (uint32_t bi = 0; bi < nb; ++bi) {
                bcnt[bi] += pc[t][bi];
                box_grow(bbox[bi], pb[t][bi]);
            }
    }

    bool take_helper() {
        int h = g_helpers.load();
        while (h < max_helpers_)
            if (g_helpers.compare_exchange_weak(h, h + 1)) return true;
        return false;
    }

    const std::vector<FBox>& boxes_;
    std::vector<uint32_t>& ids_;
    uint32_t max_leaf_, bins_;
    std::vector<BinNode>& nodes_;
    int max_helpers_;
    std::vector<Centroid> cen_;
    std::atomic<uint32_t> next_{1};
};

void build_binary(const std::vector<FBox>& boxes, std::vector<uint32_t>& ids, uint32_t max_leaf,
                  uint32_t bins, std::vector<BinNode>& nodes, int max_helpers) {
    BinaryBuilder b(boxes, ids, max_leaf, bins, nodes, max_helpers);
    b.build();
}

// Helper threads a build may start: one per core (opts.threads, 0 = all).
int helper_budget(const BuildOpts& opts) {
    const unsigned hw = opts.threads ? opts.threads : std::max(1u, std::thread::hardware_concurrency());
    return (int)hw;
}

// Chain-shaped binary tree (test aid): every inner node has one leaf of one
// item and the rest of the chain; after collapsing, each wide node holds the
// chain continuation in slot 0 and three single-item leaves after it.
void build_chain(const std::vector<FBox>& boxes, std::vector<uint32_t>& ids,
                 std::vector<BinNode>& nodes) {
    const uint32_t n = (uint32_t)boxes.size();
    ids.resize(n);
    for (uint32_t i = 0; i < n; ++i) ids[i] = i;
    nodes.clear();
    // node for suffix [k, n): inner(leaf k, suffix k+1) until one item remains
    std::vector<FBox> suffix(n);
    FBox acc;
    box_empty(acc);
    for (int64_t k = (int64_t)n - 1; k >= 0; --k) {
        box_grow(acc, boxes[k]);
        suffix[k] = acc;
    }
    nodes.emplace_back();
    int32_t cur = 0;
    for (uint32_t k = 0; k < n; ++k) {
        nodes[cur].box = suffix[k];
        if (k + 1 == n) {
            nodes[cur].first = k;
            nodes[cur].count = 1;
            break;
        }
        int32_t rest = (int32_t)nodes.size();
        nodes.emplace_back();
        int32_t leaf = (int32_t)nodes.size();
        nodes.emplace_back();
        nodes[leaf].box = boxes[k];
        nodes[leaf].first = k;
        nodes[leaf].count = 1;
        nodes[cur].left = rest;  // continuation first, so it sorts first on ties
        nodes[cur].right = leaf;
        cur = rest;
    }
}

bool quantize(QNode& q, const FBox* cb, int nc) {
    FBox u;
    box_empty(u);
    for (int i = 0; i < nc; ++i) box_grow(u, cb[i]);
    float origin[3] = {u.lo[0], u.lo[1], u.lo[2]};
    int8_t ex[3];
    for (int a = 0; a < 3; ++a) {
        double ext = (double)u.hi[a] - (double)origin[a];
        int e = -126;
        if (ext > 0.0) e = (int)std::ceil(std::log2(ext / 254.0));
        e = std::max(-126, std::min(127, e));
        for (;; ++e) {
            if (e > 127) return false;
            bool ok = true;
            const double s = std::ldexp(1.0, e);
            for (int i = 0; i < nc && ok; ++i) {
                double fl = std::floor(((double)cb[i].lo[a] - origin[a]) / s);
                int ql = (int)std::max(0.0, std::min(255.0, fl));
                while (ql > 0 && dequant((uint8_t)ql, (int8_t)e, origin[a]) > cb[i].lo[a]) --ql;
                if (dequant((uint8_t)ql, (int8_t)e, origin[a]) > cb[i].lo[a]) {
                    ok = false;
                    break;
                }
                double ch = std::ceil(((double)cb[i].hi[a] - origin[a]) / s);
                if (ch > 255.0) {
                    ok = false;
                    break;
                }
                int qh = (int)std::max(0.0, ch);
                while (qh <= 255 && dequant((uint8_t)qh, (int8_t)e, origin[a]) < cb[i].hi[a]) ++qh;
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
    q.ox = origin[0];
    q.oy = origin[1];
    q.oz = origin[2];
    q.ex = ex[0];
    q.ey = ex[1];
    q.ez = ex[2];
    return true;
}

// Collapses the binary tree to four-wide nodes in two passes: emit() lays
// the wide nodes out depth first (children and leaf references; it fixes
// every index), then quantise() fills in the child boxes of all nodes in
// parallel (each node's quantisation depends only on its own child boxes).
struct Collapser {
    const std::vector<BinNode>& bn;
    const std::vector<uint32_t>& ids;
    bool leaf_holds_id;  // TLAS: leaf child = instance id; BLAS: leaf child = slot
    std::vector<QNode>& out;
    uint32_t max_depth = 0;
    std::string err;
    std::vector<std::array<int32_t, 4>> kids;  // binary node of each child slot

    bool quantise(int threads) {
        const size_t n = out.size();
        const size_t chunk = 4096;
        std::atomic<size_t> next{0};
        std::atomic<bool> bad{false};
        auto work = [&]() {
            for (;;) {
                const size_t c0 = next.fetch_add(chunk);
                if (c0 >= n || bad.load()) break;
                for (size_t k = c0; k < std::min(n, c0 + chunk); ++k) {
                    FBox cb[4];
                    const int nc = out[k].nchild;
                    for (int i = 0; i < nc; ++i) cb[i] = bn[kids[k][i]].box;
                    if (!quantize(out[k], cb, nc)) bad.store(true);
                }
            }
        };
        const int nt = (int)std::max<size_t>(1, std::min<size_t>((size_t)std::max(1, threads), n / chunk + 1));
        std::vector<std::thread> th;
        for (int t = 1; t < nt; ++t) th.emplace_back(work);
        work();
        for (std::thread& t : th) t.join();
        if (bad.load()) {
            err = "box quantisation failed (coordinates out of range)";
            return false;
        }
        return true;
    }

    // Emits the wide node for binary node b; returns its local index or -1.
    int64_t emit(int32_t b, uint32_t depth) {
        max_depth = std::max(max_depth, depth);
        int64_t idx = (int64_t)out.size();
        if (idx > (int64_t)kMaxLocalIndex) {
            err = "too many nodes in one object (limit 2^27)";
            return -1;
        }
        out.emplace_back();
        kids.emplace_back();
        int32_t ch[4];
        int nc = 0;
        if (bn[b].left < 0) {
            ch[nc++] = b;
        } else {
            ch[nc++] = bn[b].left;
            ch[nc++] = bn[b].right;
            while (nc < 4) {
                int pick = -1;
                double best = -1.0;
                for (int i = 0; i < nc; ++i) {
                    if (bn[ch[i]].left < 0) continue;
                    double a = box_area(bn[ch[i]].box);
                    if (a > best) {
                        best = a;
                        pick = i;
                    }
                }
                if (pick < 0) break;
                int32_t c = ch[pick];
                for (int i = nc; i > pick + 1; --i) ch[i] = ch[i - 1];
                ch[pick] = bn[c].left;
                ch[pick + 1] = bn[c].right;
                ++nc;
            }
        }
        QNode q;
        std::memset(&q, 0, sizeof(q));
        uint32_t childv[4] = {0, 0, 0, 0};
        uint8_t meta[4] = {0, 0, 0, 0};
        std::array<int32_t, 4> kb = {-1, -1, -1, -1};
        for (int i = 0; i < nc; ++i) {
            const BinNode& c = bn[ch[i]];
            kb[i] = ch[i];
            if (c.left < 0) {
                if (c.count == 0 || c.count > kMaxLeaf) {
                    err = "leaf size out of range";
                    return -1;
                }
                uint32_t first = leaf_holds_id ? ids[c.first] : c.first;
                if (first > kMaxLocalIndex) {
                    err = "item index beyond 2^27 within one object";
                    return -1;
                }
                childv[i] = first;
                meta[i] = (uint8_t)c.count;
            } else {
                int64_t k = emit(ch[i], depth + 1);
                if (k < 0) return -1;
                childv[i] = (uint32_t)k;
                meta[i] = kMetaInner;
            }
        }
        for (int i = 0; i < 4; ++i) {
            q.child[i] = childv[i];
            q.meta[i] = meta[i];
        }
        q.nchild = (uint8_t)nc;
        out[idx] = q;
        kids[idx] = kb;
        return idx;
    }
};

bool finite_box(const FBox& b) {
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(b.lo[a]) || !std::isfinite(b.hi[a])) return false;
    return true;
}

}  // namespace

float dequant(uint8_t q, int8_t e, float origin) {
    return std::fmaf((float)q, std::ldexp(1.0f, e), origin);
}

FBox transform_box(const FBox& b, const float* x) {
    FBox out;
    for (int r = 0; r < 3; ++r) {
        double wc = (double)x[4 * r + 3], wh = 0.0, mag = std::fabs(wc);
        for (int c = 0; c < 3; ++c) {
            const double ctr = 0.5 * ((double)b.lo[c] + (double)b.hi[c]);
            const double half = 0.5 * ((double)b.hi[c] - (double)b.lo[c]);
            const double a = (double)x[4 * r + c];
            wc += a * ctr;
            wh += std::fabs(a) * half;
            mag += std::fabs(a * ctr) + std::fabs(a) * half;
        }
        // every product and sum above is exact to within 2^-52 of mag;
        // 1e-12 mag covers their accumulated rounding many times over
        const double pad = 1e-12 * mag + 1e-300;
        const double l = wc - wh - pad, h = wc + wh + pad;
        float fl = (float)l, fh = (float)h;
        if ((double)fl > l) fl = std::nextafter(fl, -kFInf);
        if ((double)fh < h) fh = std::nextafter(fh, kFInf);
        out.lo[r] = fl;
        out.hi[r] = fh;
    }
    return out;
}

static void level_boxes_rec(const std::vector<QNode>& nodes, uint32_t n, uint32_t level,
                            std::vector<FBox>& out) {
    const QNode& q = nodes[n];
    const float o[3] = {q.ox, q.oy, q.oz};
    const int8_t e[3] = {q.ex, q.ey, q.ez};
    for (int i = 0; i < 4; ++i) {
        const uint8_t m = q.meta[i];
        if (m == 0) continue;
        if (m == kMetaInner && level > 1) {
            level_boxes_rec(nodes, q.child[i], level - 1, out);
            continue;
        }
        FBox b;
        for (int a = 0; a < 3; ++a) {
            b.lo[a] = dequant(q.qlo[a][i], e[a], o[a]);
            b.hi[a] = dequant(q.qhi[a][i], e[a], o[a]);
        }
        out.push_back(b);
    }
}

std::vector<FBox> level_boxes(const std::vector<QNode>& nodes, uint32_t level) {
    std::vector<FBox> out;
    if (level == 0 || nodes.empty()) return out;
    level_boxes_rec(nodes, 0, level, out);
    return out;
}

bool build_blas(const float* verts, uint32_t n_verts, const uint32_t* quads, uint32_t n_quads,
                const BuildOpts& opts, BlasResult& out, std::string& err) {
    if (n_quads == 0) {
        err = "mesh has no quads";
        return false;
    }
    if (n_quads > kMaxLocalIndex) {
        err = "mesh has more than 2^27 quads";
        return false;
    }
    std::vector<FBox> boxes(n_quads);
    for (uint32_t q = 0; q < n_quads; ++q) {
        FBox b;
        box_empty(b);
        for (int k = 0; k < 4; ++k) {
            uint32_t vi = quads[4 * (size_t)q + k];
            if (vi >= n_verts) {
                err = "quad vertex index out of range";
                return false;
            }
            const float* v = verts + 3 * (size_t)vi;
            if (!std::isfinite(v[0]) || !std::isfinite(v[1]) || !std::isfinite(v[2])) {
                err = "non-finite vertex";
                return false;
            }
            FBox p{{v[0], v[1], v[2]}, {v[0], v[1], v[2]}};
            box_grow(b, p);
        }
        if (!finite_box(b)) {
            err = "non-finite vertex";
            return false;
        }
        boxes[q] = b;
    }
    std::vector<BinNode> bn;
    std::vector<uint32_t> ids;
    if (opts.degenerate)
        build_chain(boxes, ids, bn);
    else
        build_binary(boxes, ids, std::max(1u, std::min(opts.max_leaf, 8u)),
                     std::max(4u, std::min(opts.sah_bins, 64u)), bn, helper_budget(opts));
    out.nodes.clear();
    Collapser col{bn, ids, false, out.nodes};
    if (col.emit(0, 1) < 0 || !col.quantise(1)) {
        err = col.err;
        return false;
    }
    out.depth = col.max_depth;
    out.quads.resize(n_quads);
    out.prim.resize(n_quads);
    for (uint32_t s = 0; s < n_quads; ++s) {
        uint32_t q = ids[s];
        out.prim[s] = q;
        for (int k = 0; k < 4; ++k) {
            const float* v = verts + 3 * (size_t)quads[4 * (size_t)q + k];
            out.quads[s].v[3 * k] = v[0];
            out.quads[s].v[3 * k + 1] = v[1];
            out.quads[s].v[3 * k + 2] = v[2];
        }
    }
    out.box = bn[0].box;
    return true;
}

bool build_tlas(const std::vector<FBox>& inst_boxes, const BuildOpts& opts, TlasResult& out,
                std::string& err) {
    out.nodes.clear();
    out.depth = 0;
    if (inst_boxes.empty()) return true;
    if (inst_boxes.size() > kMaxLocalIndex) {
        err = "more than 2^27 instances";
        return false;
    }
    for (const FBox& b : inst_boxes)
        if (!finite_box(b)) {
            err = "non-finite instance bounds";
            return false;
        }
    std::vector<BinNode> bn;
    std::vector<uint32_t> ids;
    build_binary(inst_boxes, ids, 1, std::max(4u, std::min(opts.sah_bins, 64u)), bn,
                 helper_budget(opts));
    Collapser col{bn, ids, true, out.nodes};
    if (col.emit(0, 1) < 0 || !col.quantise(helper_budget(opts))) {
        err = col.err;
        return false;
    }
    out.depth = col.max_depth;
    return true;
}

namespace {
// Checks subtrees recursively; the subtrees two levels below the root of a
// large tree are checked on their own threads (items are marked seen with
// atomic increments, so an item referenced from two subtrees is still found).
struct Checker {
    const std::vector<QNode>& nodes;
    const std::vector<FBox>& items;
    std::vector<uint8_t>& seen;
    std::string err;
    uint32_t depth = 0;
    uint32_t fork_depth = 0;  // nodes at depths < fork_depth check inner children on threads

    bool rec(uint32_t idx, uint32_t d, FBox& box) {
        depth = std::max(depth, d);
        if (d < fork_depth && idx < nodes.size()) return rec_forked(idx, d, box);
        if (idx >= nodes.size()) {
            err = "child node index out of range";
            return false;
        }
        const QNode& n = nodes[idx];
        box_empty(box);
        const float org[3] = {n.ox, n.oy, n.oz};
        const int8_t ex[3] = {n.ex, n.ey, n.ez};
        int valid = 0;
        for (int i = 0; i < 4; ++i) {
            if (n.meta[i] == 0) continue;
            ++valid;
            FBox cb;
            if (n.meta[i] == kMetaInner) {
                if (!rec(n.child[i], d + 1, cb)) return false;
            } else {
                if (n.meta[i] > kMaxLeaf) {
                    err = "leaf count too large";
                    return false;
                }
                box_empty(cb);
                for (uint32_t k = 0; k < n.meta[i]; ++k) {
                    uint32_t it = n.child[i] + k;
                    if (it >= items.size()) {
                        err = "leaf item out of range";
                        return false;
                    }
                    if (__atomic_fetch_add(&seen[it], (uint8_t)1, __ATOMIC_RELAXED)) {
                        err = "item referenced twice";
                        return false;
                    }
                    box_grow(cb, items[it]);
                }
            }
            for (int a = 0; a < 3; ++a) {
                float lo = dequant(n.qlo[a][i], ex[a], org[a]);
                float hi = dequant(n.qhi[a][i], ex[a], org[a]);
                if (!(lo <= cb.lo[a] && hi >= cb.hi[a])) {
                    err = "quantised child box does not contain its subtree";
                    return false;
                }
            }
            box_grow(box, cb);
        }
        if (valid == 0 || valid != n.nchild) {
            err = "node child count inconsistent";
            return false;
        }
        return true;
    }

    // As rec(), with each inner child checked by its own Checker on a thread.
    bool rec_forked(uint32_t idx, uint32_t d, FBox& box) {
        const QNode& n = nodes[idx];
        std::vector<Checker> sub;
        sub.reserve(4);
        FBox cbs[4];
        bool ok[4] = {true, true, true, true};
        std::vector<std::thread> th;
        for (int i = 0; i < 4; ++i)
            if (n.meta[i] == kMetaInner) sub.push_back(Checker{nodes, items, seen, {}, 0, fork_depth});
        int s = 0;
        for (int i = 0; i < 4; ++i) {
            if (n.meta[i] != kMetaInner) continue;
            Checker* c = &sub[s++];
            th.emplace_back([c, &n, i, d, &cbs, &ok] { ok[i] = c->rec(n.child[i], d + 1, cbs[i]); });
        }
        for (std::thread& t : th) t.join();
        s = 0;
        for (int i = 0; i < 4; ++i) {
            if (n.meta[i] != kMetaInner) continue;
            Checker& c = sub[s++];
            depth = std::max(depth, c.depth);
            if (!ok[i]) {
                err = c.err;
                return false;
            }
        }
        // the node itself, with the children's boxes already known
        Checker self{nodes, items, seen, {}, 0, 0};
        if (!self.node(idx, d, box, cbs)) {
            err = self.err;
            return false;
        }
        depth = std::max(depth, self.depth);
        return true;
    }

    // Checks node idx given the boxes of its inner children (leaves are
    // checked here).
    bool node(uint32_t idx, uint32_t d, FBox& box, const FBox* inner_boxes) {
        depth = std::max(depth, d);
        const QNode& n = nodes[idx];
        box_empty(box);
        const float org[3] = {n.ox, n.oy, n.oz};
        const int8_t ex[3] = {n.ex, n.ey, n.ez};
        int valid = 0;
        for (int i = 0; i < 4; ++i) {
            if (n.meta[i] == 0) continue;
            ++valid;
            FBox cb;
            if (n.meta[i] == kMetaInner) {
                cb = inner_boxes[i];
            } else {
                if (n.meta[i] > kMaxLeaf) {
                    err = "leaf count too large";
                    return false;
                }
                box_empty(cb);
                for (uint32_t k = 0; k < n.meta[i]; ++k) {
                    uint32_t it = n.child[i] + k;
                    if (it >= items.size()) {
                        err = "leaf item out of range";
                        return false;
                    }
                    if (__atomic_fetch_add(&seen[it], (uint8_t)1, __ATOMIC_RELAXED)) {
                        err = "item referenced twice";
                        return false;
                    }
                    box_grow(cb, items[it]);
                }
            }
            for (int a = 0; a < 3; ++a) {
                float lo = dequant(n.qlo[a][i], ex[a], org[a]);
                float hi = dequant(n.qhi[a][i], ex[a], org[a]);
                if (!(lo <= cb.lo[a] && hi >= cb.hi[a])) {
                    err = "quantised child box does not contain its subtree";
                    return false;
                }
            }
            box_grow(box, cb);
        }
        if (valid == 0 || valid != n.nchild) {
            err = "node child count inconsistent";
            return false;
        }
        return true;
    }
};
}  // namespace

bool check_wide(const std::vector<QNode>& nodes, const std::vector<FBox>& item_boxes,
                std::string& err, uint32_t* depth) {
    if (nodes.empty()) {
        if (!item_boxes.empty()) {
            err = "no nodes for a non-empty item set";
            return false;
        }
        return true;
    }
    std::vector<uint8_t> seen(item_boxes.size(), 0);
    // large trees: the root's and its children's inner subtrees on threads
    Checker c{nodes, item_boxes, seen, {}, 0, nodes.size() > (1u << 16) ? 3u : 0u};
    FBox b;
    if (!c.rec(0, 1, b)) {
        err = c.err;
        return false;
    }
    for (size_t i = 0; i < seen.size(); ++i)
        if (seen[i] != 1) {
            err = "item not referenced";
            return false;
        }
    if (depth) *depth = c.depth;
    return true;
}

}  // namespace qrt

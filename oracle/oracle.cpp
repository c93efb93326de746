// FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h for scope,
// citations and the parity status of each function).
//
// Plain and slow on purpose: binary BVHs with median splits, exact FP64
// boxes, Moller-Trumbore per triangle, one std::thread per slice of work.
#include "oracle.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <thread>
#include <vector>

namespace {

const double kPi = 3.14159265358979323846;
const double kInf = std::numeric_limits<double>::infinity();
const uint32_t kNone = 0xFFFFFFFFu;

struct V3 {
    double x, y, z;
};
inline V3 mk(double x, double y, double z) { return V3{x, y, z}; }
inline V3 operator+(V3 a, V3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
inline V3 operator-(V3 a, V3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
inline V3 operator*(double s, V3 a) { return mk(s * a.x, s * a.y, s * a.z); }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
inline V3 normalize(V3 a) { return (1.0 / std::sqrt(dot(a, a))) * a; }
inline double comp(V3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

// ---------------------------------------------------------------------------
// Philox4x32-10, from its definition (Salmon, Moraes, Dror and Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC 2011): ten rounds of two 32x32->64
// multiplies with S-box constants 0xD2511F53 / 0xCD9E8D57, the key bumped by
// the Weyl constants 0x9E3779B9 / 0xBB67AE85 between rounds.
// ---------------------------------------------------------------------------
void philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// Uniform in [0,1) with 24 bits: exact in both float and double.
inline double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

// Four uniforms keyed by (global pixel, sample, bounce).
void draw4(uint64_t seed, uint64_t pixel, uint32_t sample, uint32_t bounce, double xi[4]) {
    uint32_t ctr[4] = {(uint32_t)pixel, (uint32_t)(pixel >> 32), sample, bounce};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    philox(ctr, key, out);
    for (int i = 0; i < 4; ++i) xi[i] = u01(out[i]);
}

// ---------------------------------------------------------------------------
// Ray / triangle: Moller-Trumbore in double, both sides, inclusive edges.
// ---------------------------------------------------------------------------
bool tri_hit(V3 o, V3 d, V3 a, V3 b, V3 c, double tmin, double tmax, double* t, double* bu,
             double* bv) {
    V3 e1 = b - a, e2 = c - a;
    V3 p = cross(d, e2);
    double det = dot(e1, p);
    if (det == 0.0) return false;
    double inv = 1.0 / det;
    V3 s = o - a;
    double u = dot(s, p) * inv;
    if (u < 0.0 || u > 1.0) return false;
    V3 q = cross(s, e1);
    double v = dot(d, q) * inv;
    if (v < 0.0 || u + v > 1.0) return false;
    double tt = dot(e2, q) * inv;
    if (!(tt > tmin && tt < tmax)) return false;
    *t = tt;
    *bu = u;
    *bv = v;
    return true;
}

// Quad (v0,v1,v2,v3) = triangles (v0,v1,v2) and (v0,v2,v3).  Quad-space
// (u,v): triangle 0 gives (b1+b2, b2), triangle 1 gives (b1, b1+b2).
bool quad_hit(V3 o, V3 d, const V3 v[4], double tmin, double tmax, double* t, double* u,
              double* w) {
    bool hit = false;
    double tt, b1, b2;
    double best = tmax;
    if (tri_hit(o, d, v[0], v[1], v[2], tmin, best, &tt, &b1, &b2)) {
        hit = true;
        best = tt;
        *t = tt;
        *u = b1 + b2;
        *w = b2;
    }
    if (tri_hit(o, d, v[0], v[2], v[3], tmin, best, &tt, &b1, &b2)) {
        hit = true;
        best = tt;
        *t = tt;
        *u = b1;
        *w = b1 + b2;
    }
    return hit;
}

// ---------------------------------------------------------------------------
// Boxes and a plain binary BVH (median split along the longest centroid axis).
// ---------------------------------------------------------------------------
struct Box {
    V3 lo, hi;
};
Box empty_box() { return Box{mk(kInf, kInf, kInf), mk(-kInf, -kInf, -kInf)}; }
void grow(Box& b, V3 p) {
    b.lo = mk(std::min(b.lo.x, p.x), std::min(b.lo.y, p.y), std::min(b.lo.z, p.z));
    b.hi = mk(std::max(b.hi.x, p.x), std::max(b.hi.y, p.y), std::max(b.hi.z, p.z));
}
void grow(Box& b, const Box& c) {
    grow(b, c.lo);
    grow(b, c.hi);
}
// Pad so that rounding in the slab test can never drop a true hit.
Box padded(Box b) {
    double m = std::max({std::fabs(b.lo.x), std::fabs(b.lo.y), std::fabs(b.lo.z),
                         std::fabs(b.hi.x), std::fabs(b.hi.y), std::fabs(b.hi.z)});
    double e = 1e-9 * (m + 1.0);
    return Box{b.lo - mk(e, e, e), b.hi + mk(e, e, e)};
}

// Slab test on [t0, t1] (inclusive).
bool box_hit(const Box& b, V3 o, V3 d, double t0, double t1) {
    for (int a = 0; a < 3; ++a) {
        double oa = comp(o, a), da = comp(d, a), lo = comp(b.lo, a), hi = comp(b.hi, a);
        if (da == 0.0) {
            if (oa < lo || oa > hi) return false;
            continue;
        }
        double ta = (lo - oa) / da, tb = (hi - oa) / da;
        if (ta > tb) std::swap(ta, tb);
        t0 = std::max(t0, ta);
        t1 = std::min(t1, tb);
        if (t0 > t1) return false;
    }
    return true;
}

struct Node {
    Box box;
    int left = -1, right = -1;  // children (internal)
    int first = 0, count = 0;   // items (leaf, count > 0)
};

struct Bvh {
    std::vector<Node> nodes;
    std::vector<uint32_t> items;  // item ids in leaf order
};

// Nodes of the tree over m items: a node over m > 4 items splits them
// m/2 : m - m/2, so the subtree sizes on one level take at most two values.
uint64_t tree_nodes(uint64_t m) {
    std::map<uint64_t, uint64_t> level{{m, 1}};
    uint64_t nodes = 0;
    while (!level.empty()) {
        std::map<uint64_t, uint64_t> next;
        for (const auto& sc : level) {
            nodes += sc.second;
            if (sc.first > 4) {
                next[sc.first / 2] += sc.second;
                next[sc.first - sc.first / 2] += sc.second;
            }
        }
        level.swap(next);
    }
    return nodes;
}

// Builds the subtree over ids[lo, hi) into bvh.nodes[node ...] in preorder
// (left subtree first): its size is known in advance, so the two halves of a
// large node are built on two threads without changing the tree.
void build_rec(Bvh& bvh, const std::vector<Box>& boxes, std::vector<uint32_t>& ids, int64_t lo,
               int64_t hi, uint64_t node, int fork_levels) {
    Box b = empty_box(), cb = empty_box();
    for (int64_t i = lo; i < hi; ++i) {
        grow(b, boxes[ids[i]]);
        grow(cb, 0.5 * (boxes[ids[i]].lo + boxes[ids[i]].hi));
    }
    bvh.nodes[node].box = padded(b);
    if (hi - lo <= 4) {
        bvh.nodes[node].first = (int)lo;
        bvh.nodes[node].count = (int)(hi - lo);
        return;
    }
    V3 ext = cb.hi - cb.lo;
    int axis = (ext.x >= ext.y && ext.x >= ext.z) ? 0 : (ext.y >= ext.z ? 1 : 2);
    int64_t mid = (lo + hi) / 2;
    std::nth_element(ids.begin() + lo, ids.begin() + mid, ids.begin() + hi,
                     [&](uint32_t a, uint32_t c) {
                         double ca = comp(boxes[a].lo, axis) + comp(boxes[a].hi, axis);
                         double cc = comp(boxes[c].lo, axis) + comp(boxes[c].hi, axis);
                         return ca < cc || (ca == cc && a < c);
                     });
    const uint64_t l = node + 1, r = node + 1 + tree_nodes((uint64_t)(mid - lo));
    bvh.nodes[node].left = (int)l;
    bvh.nodes[node].right = (int)r;
    if (fork_levels > 0 && hi - lo >= (1 << 16)) {
        std::thread t([&] { build_rec(bvh, boxes, ids, lo, mid, l, fork_levels - 1); });
        build_rec(bvh, boxes, ids, mid, hi, r, fork_levels - 1);
        t.join();
    } else {
        build_rec(bvh, boxes, ids, lo, mid, l, 0);
        build_rec(bvh, boxes, ids, mid, hi, r, 0);
    }
}

Bvh build_bvh(const std::vector<Box>& boxes) {
    Bvh bvh;
    std::vector<uint32_t> ids(boxes.size());
    for (size_t i = 0; i < ids.size(); ++i) ids[i] = (uint32_t)i;
    bvh.nodes.resize(boxes.empty() ? 1 : tree_nodes(boxes.size()));
    if (!boxes.empty()) build_rec(bvh, boxes, ids, 0, (int64_t)boxes.size(), 0, 4);
    bvh.items = ids;
    return bvh;
}

// ---------------------------------------------------------------------------
// Scene
// ---------------------------------------------------------------------------
struct Mesh {
    std::vector<V3> verts;
    std::vector<uint32_t> quads;  // 4 per quad
    uint64_t albedo_base = 0;
    Bvh bvh;
    Box box;
    void quad(uint32_t q, V3 v[4]) const {
        for (int k = 0; k < 4; ++k) v[k] = verts[quads[4 * q + k]];
    }
};

struct Instance {
    double A[9];     // object->world linear part (row-major)
    double b[3];     // translation
    double Ainv[9];  // world->object linear part
    uint32_t mesh;
    Box world_box;
};

V3 mul3(const double* M, V3 v) {
    return mk(M[0] * v.x + M[1] * v.y + M[2] * v.z, M[3] * v.x + M[4] * v.y + M[5] * v.z,
              M[6] * v.x + M[7] * v.y + M[8] * v.z);
}
V3 mul3T(const double* M, V3 v) {  // M^T v
    return mk(M[0] * v.x + M[3] * v.y + M[6] * v.z, M[1] * v.x + M[4] * v.y + M[7] * v.z,
              M[2] * v.x + M[5] * v.y + M[8] * v.z);
}

// 3x3 inverse by the adjugate.
void inverse3(const double* m, double* r) {
    double c00 = m[4] * m[8] - m[5] * m[7];
    double c01 = m[5] * m[6] - m[3] * m[8];
    double c02 = m[3] * m[7] - m[4] * m[6];
    double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
    double id = 1.0 / det;
    r[0] = c00 * id;
    r[1] = (m[2] * m[7] - m[1] * m[8]) * id;
    r[2] = (m[1] * m[5] - m[2] * m[4]) * id;
    r[3] = c01 * id;
    r[4] = (m[0] * m[8] - m[2] * m[6]) * id;
    r[5] = (m[2] * m[3] - m[0] * m[5]) * id;
    r[6] = c02 * id;
    r[7] = (m[1] * m[6] - m[0] * m[7]) * id;
    r[8] = (m[0] * m[4] - m[1] * m[3]) * id;
}

}  // namespace

struct ora_scene {
    std::vector<Mesh> meshes;
    std::vector<Instance> inst;
    Bvh tlas;
    uint64_t n_quads = 0;
};

namespace {

struct HitRec {
    double t;
    uint32_t inst, prim;
    double u, v;
};

inline bool better(double t, uint32_t inst, uint32_t prim, const HitRec& h) {
    if (t != h.t) return t < h.t;
    if (inst != h.inst) return inst < h.inst;
    return prim < h.prim;
}

void object_ray(const Instance& I, V3 o, V3 d, V3* oo, V3* od) {
    *oo = mul3(I.Ainv, o - mk(I.b[0], I.b[1], I.b[2]));
    *od = mul3(I.Ainv, d);
}

// Closest hit within one mesh (object space), updating h with tie-break.
void mesh_closest(const Mesh& m, uint32_t inst_id, V3 o, V3 d, double tmin, double tmax,
                  HitRec& h, bool brute) {
    V3 v[4];
    double t, u, w;
    if (brute) {
        for (uint32_t q = 0; q < (uint32_t)(m.quads.size() / 4); ++q) {
            m.quad(q, v);
            if (quad_hit(o, d, v, tmin, tmax, &t, &u, &w) && t <= h.t &&
                better(t, inst_id, q, h))
                h = HitRec{t, inst_id, q, u, w};
        }
        return;
    }
    std::vector<int> stack;
    stack.push_back(0);
    while (!stack.empty()) {
        const Node& n = m.bvh.nodes[stack.back()];
        stack.pop_back();
        if (!box_hit(n.box, o, d, tmin, h.t)) continue;
        if (n.count > 0) {
            for (int i = 0; i < n.count; ++i) {
                uint32_t q = m.bvh.items[n.first + i];
                m.quad(q, v);
                if (quad_hit(o, d, v, tmin, tmax, &t, &u, &w) && t <= h.t &&
                    better(t, inst_id, q, h))
                    h = HitRec{t, inst_id, q, u, w};
            }
        } else {
            stack.push_back(n.left);
            stack.push_back(n.right);
        }
    }
}

bool mesh_any(const Mesh& m, V3 o, V3 d, double tmin, double tmax, bool brute) {
    V3 v[4];
    double t, u, w;
    if (brute) {
        for (uint32_t q = 0; q < (uint32_t)(m.quads.size() / 4); ++q) {
            m.quad(q, v);
            if (quad_hit(o, d, v, tmin, tmax, &t, &u, &w)) return true;
        }
        return false;
    }
    std::vector<int> stack;
    stack.push_back(0);
    while (!stack.empty()) {
        const Node& n = m.bvh.nodes[stack.back()];
        stack.pop_back();
        if (!box_hit(n.box, o, d, tmin, tmax)) continue;
        if (n.count > 0) {
            for (int i = 0; i < n.count; ++i) {
                m.quad(m.bvh.items[n.first + i], v);
                if (quad_hit(o, d, v, tmin, tmax, &t, &u, &w)) return true;
            }
        } else {
            stack.push_back(n.left);
            stack.push_back(n.right);
        }
    }
    return false;
}

// World ray through the whole scene.  mode 0: TLAS + BLAS BVHs; 1: every
// instance and every quad; 2: every quad moved to world space (flattened).
HitRec closest(const ora_scene& s, V3 o, V3 d, double tmin, double tmax, int mode) {
    HitRec h{tmax, kNone, kNone, 0.0, 0.0};
    if (mode == 2) {
        V3 v[4];
        double t, u, w;
        for (uint32_t i = 0; i < (uint32_t)s.inst.size(); ++i) {
            const Instance& I = s.inst[i];
            const Mesh& m = s.meshes[I.mesh];
            for (uint32_t q = 0; q < (uint32_t)(m.quads.size() / 4); ++q) {
                m.quad(q, v);
                for (int k = 0; k < 4; ++k) v[k] = mul3(I.A, v[k]) + mk(I.b[0], I.b[1], I.b[2]);
                if (quad_hit(o, d, v, tmin, tmax, &t, &u, &w) && t <= h.t && better(t, i, q, h))
                    h = HitRec{t, i, q, u, w};
            }
        }
        return h;
    }
    if (mode == 1) {
        for (uint32_t i = 0; i < (uint32_t)s.inst.size(); ++i) {
            V3 oo, od;
            object_ray(s.inst[i], o, d, &oo, &od);
            mesh_closest(s.meshes[s.inst[i].mesh], i, oo, od, tmin, tmax, h, true);
        }
        return h;
    }
    if (s.inst.empty()) return h;
    std::vector<int> stack;
    stack.push_back(0);
    while (!stack.empty()) {
        const Node& n = s.tlas.nodes[stack.back()];
        stack.pop_back();
        if (!box_hit(n.box, o, d, tmin, h.t)) continue;
        if (n.count > 0) {
            for (int k = 0; k < n.count; ++k) {
                uint32_t i = s.tlas.items[n.first + k];
                if (!box_hit(s.inst[i].world_box, o, d, tmin, h.t)) continue;
                V3 oo, od;
                object_ray(s.inst[i], o, d, &oo, &od);
                mesh_closest(s.meshes[s.inst[i].mesh], i, oo, od, tmin, tmax, h, false);
            }
        } else {
            stack.push_back(n.left);
            stack.push_back(n.right);
        }
    }
    return h;
}

bool any_hit(const ora_scene& s, V3 o, V3 d, double tmin, double tmax, int mode) {
    if (mode == 2) return closest(s, o, d, tmin, tmax, 2).inst != kNone;
    if (mode == 1) {
        for (uint32_t i = 0; i < (uint32_t)s.inst.size(); ++i) {
            V3 oo, od;
            object_ray(s.inst[i], o, d, &oo, &od);
            if (mesh_any(s.meshes[s.inst[i].mesh], oo, od, tmin, tmax, true)) return true;
        }
        return false;
    }
    if (s.inst.empty()) return false;
    std::vector<int> stack;
    stack.push_back(0);
    while (!stack.empty()) {
        const Node& n = s.tlas.nodes[stack.back()];
        stack.pop_back();
        if (!box_hit(n.box, o, d, tmin, tmax)) continue;
        if (n.count > 0) {
            for (int k = 0; k < n.count; ++k) {
                uint32_t i = s.tlas.items[n.first + k];
                if (!box_hit(s.inst[i].world_box, o, d, tmin, tmax)) continue;
                V3 oo, od;
                object_ray(s.inst[i], o, d, &oo, &od);
                if (mesh_any(s.meshes[s.inst[i].mesh], oo, od, tmin, tmax, false)) return true;
            }
        } else {
            stack.push_back(n.left);
            stack.push_back(n.right);
        }
    }
    return false;
}

template <class F>
void parallel_for(uint64_t n, int nthreads, F f) {
    if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
    std::atomic<uint64_t> next{0};
    const uint64_t chunk = 64;
    auto work = [&]() {
        for (;;) {
            uint64_t b = next.fetch_add(chunk);
            if (b >= n) break;
            uint64_t e = std::min(n, b + chunk);
            for (uint64_t i = b; i < e; ++i) f(i);
        }
    };
    std::vector<std::thread> th;
    for (int k = 1; k < nthreads; ++k) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
}

// ---------------------------------------------------------------------------
// Camera and sampling
// ---------------------------------------------------------------------------
// Pinhole through (x + xi1, y + xi2); y = 0 is the top row; vfov is vertical.
void camera_ray(const ora_view& v, double px, double py, V3* o, V3* d) {
    V3 eye = mk(v.eye[0], v.eye[1], v.eye[2]);
    V3 f = normalize(mk(v.look[0], v.look[1], v.look[2]) - eye);
    V3 r = normalize(cross(f, mk(v.up[0], v.up[1], v.up[2])));
    V3 u = cross(r, f);
    double th = std::tan(0.5 * (double)v.vfov_deg * kPi / 180.0);
    double aspect = (double)v.w / (double)v.h;
    double sx = (2.0 * px / (double)v.w - 1.0) * th * aspect;
    double sy = (1.0 - 2.0 * py / (double)v.h) * th;
    *o = eye;
    *d = normalize(f + sx * r + sy * u);
}

// Cosine-weighted hemisphere (Malley's method: a uniform disk sample lifted
// onto the hemisphere) in the orthonormal basis of Duff et al., "Building an
// Orthonormal Basis, Revisited", JCGT 2017.
V3 sample_cosine(V3 n, double xi1, double xi2) {
    double r = std::sqrt(xi1);
    double phi = 2.0 * kPi * xi2;
    double lx = r * std::cos(phi), ly = r * std::sin(phi);
    double lz = std::sqrt(std::max(0.0, 1.0 - xi1));
    double sign = std::copysign(1.0, n.z);
    double a = -1.0 / (sign + n.z);
    double b = n.x * n.y * a;
    V3 b1 = mk(1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x);
    V3 b2 = mk(b, sign + n.y * n.y * a, -n.y);
    return lx * b1 + ly * b2 + lz * n;
}

// Geometric normal of quad q of instance i in world space: the cross product of
// the two diagonals (independent of which of the two triangles was hit), moved
// by the inverse transpose of the object->world linear part.
V3 world_normal(const ora_scene& s, uint32_t i, uint32_t q) {
    const Instance& I = s.inst[i];
    V3 v[4];
    s.meshes[I.mesh].quad(q, v);
    V3 n = cross(v[2] - v[0], v[3] - v[1]);
    return normalize(mul3T(I.Ainv, n));
}

// Self-intersection offset along the (faced) normal, scaled with |p|.
V3 spawn_point(V3 p, V3 n) {
    double m = std::max({std::fabs(p.x), std::fabs(p.y), std::fabs(p.z)});
    return p + (1e-4 + 1e-5 * m) * n;
}

struct PathVertex {
    uint64_t albedo_row;
    double tex[3];  // texture factor of the diffuse albedo at the hit (1 without textures)
    double nee[3];  // light arriving by next-event estimation, over pi (sun and key light)
};

// Per-face texture (the stand-in for a Ptex texture: a texel grid baked on
// each face, looked up by face id and the hit's position on the face): quad
// row's R x R RGB texels (row-major in v, then u) cover quad-space
// [i/R, (i+1)/R] x [j/R, (j+1)/R]; the value at (u, v) is bilinear between
// texel centres, clamped to the face.
void tex_lookup(const float* tex, uint32_t R, uint64_t row, double u, double v, double out[3]) {
    const double s = std::min(std::max(u * R - 0.5, 0.0), (double)(R - 1));
    const double t = std::min(std::max(v * R - 0.5, 0.0), (double)(R - 1));
    const uint32_t i0 = (uint32_t)std::floor(s), j0 = (uint32_t)std::floor(t);
    const uint32_t i1 = std::min(i0 + 1, R - 1), j1 = std::min(j0 + 1, R - 1);
    const double fs = s - i0, ft = t - j0;
    const float* T = tex + row * R * R * 3;
    for (int c = 0; c < 3; ++c)
        out[c] = (1.0 - fs) * (1.0 - ft) * T[3 * (j0 * R + i0) + c] + fs * (1.0 - ft) * T[3 * (j0 * R + i1) + c] +
                 (1.0 - fs) * ft * T[3 * (j1 * R + i0) + c] + fs * ft * T[3 * (j1 * R + i1) + c];
}

// One sample of the key lights seen from x with unit normal nx.  Light k
// (corner c, edges e1, e2, radiance Le; 12 floats) is a parallelogram
// emitting on the side of e1 x e2.  xi picks a light uniformly and a point
// uniformly on it; the estimator of the light arriving at x is
// Le cos_x cos_l |e1 x e2| n / d^2 (n lights).  Writes the unit direction
// toward the point, its distance and that estimator; false when the point
// faces away from x or lies below x's horizon.
bool light_sample(const float* lights, uint32_t n, const double xi[3], V3 x, V3 nx, V3* dir,
                  double* dist, double w[3]) {
    const uint32_t k = std::min((uint32_t)(xi[0] * n), n - 1);
    const float* Lk = lights + 12 * (size_t)k;
    const V3 c = mk(Lk[0], Lk[1], Lk[2]), e1 = mk(Lk[3], Lk[4], Lk[5]), e2 = mk(Lk[6], Lk[7], Lk[8]);
    const V3 y = c + xi[1] * e1 + xi[2] * e2;
    const V3 q = y - x;
    const double d2 = dot(q, q);
    if (!(d2 > 0.0)) return false;
    const double d = std::sqrt(d2);
    const V3 om = (1.0 / d) * q;
    const V3 cr = cross(e1, e2);
    const double A = std::sqrt(dot(cr, cr));
    if (!(A > 0.0)) return false;
    const double cx = dot(nx, om), cl = -dot(cr, om) / A;
    if (!(cx > 0.0) || !(cl > 0.0)) return false;
    const double g = cx * cl * A * (double)n / d2;
    for (int ch = 0; ch < 3; ++ch) w[ch] = Lk[9 + ch] * g;
    *dir = om;
    *dist = d;
    return true;
}

// Philox counter word of the key-light sample drawn at bounce i.
const uint32_t kLightStream = 0x40000000u;

// Optional per-path logs of trace_path.
struct PathLogs {
    uint32_t* inst = nullptr;   // max_depth hit instances
    uint32_t* prim = nullptr;   // max_depth hit quads
    uint32_t* shadow = nullptr; // sun shadow bits
    uint32_t* light = nullptr;  // key-light shadow bits
    double* rays = nullptr;     // max_depth records of kRayRec doubles
};
const int kRayRec = 13;  // ray origin, direction; spawn point; light direction, distance

struct PathRecord {
    std::vector<PathVertex> verts;
    bool escaped = false;  // the ray after the last vertex left the scene
};

// One path sample (the view's sample sample_base + k); returns radiance
// (with the given albedo) and its record.
void trace_path(const ora_scene& s, const ora_view& view, const float* albedo,
                const ora_params& p, uint32_t x, uint32_t y, uint32_t k, double L[3],
                PathRecord* rec, const PathLogs& lg) {
    uint32_t* log_inst = lg.inst;
    uint32_t* log_prim = lg.prim;
    uint32_t* log_shadow = lg.shadow;
    double* log_rays = lg.rays;
    const uint64_t pix = view.pixel_base + (uint64_t)y * view.w + x;
    const uint32_t smp = view.sample_base + k;  // Philox counter: (pixel, sample, bounce)
    double xi[4];
    draw4(p.seed, pix, smp, 0, xi);
    V3 o, d;
    camera_ray(view, x + xi[0], y + xi[1], &o, &d);
    double beta[3] = {1.0, 1.0, 1.0};
    L[0] = L[1] = L[2] = 0.0;
    const bool sun = p.sun_E[0] != 0.0f || p.sun_E[1] != 0.0f || p.sun_E[2] != 0.0f;
    V3 l = normalize(mk(p.sun_dir[0], p.sun_dir[1], p.sun_dir[2]));
    uint32_t shadow_bits = 0, light_bits = 0;
    if (rec) {
        rec->verts.clear();
        rec->escaped = false;
    }
    for (uint32_t i = 1; i <= p.max_depth; ++i) {
        if (log_rays) {
            // the ray traced at depth i: origin, direction (spawn point and
            // key-light sample below)
            double* r = log_rays + kRayRec * (i - 1);
            r[0] = o.x, r[1] = o.y, r[2] = o.z, r[3] = d.x, r[4] = d.y, r[5] = d.z;
        }
        HitRec h = closest(s, o, d, 0.0, kInf, 0);
        if (log_inst) {
            log_inst[i - 1] = h.inst;
            log_prim[i - 1] = h.prim;
        }
        if (h.inst == kNone) {
            for (int c = 0; c < 3; ++c) L[c] += beta[c] * p.env[c];
            if (rec) rec->escaped = true;
            break;
        }
        const Instance& I = s.inst[h.inst];
        uint64_t row = s.meshes[I.mesh].albedo_base + h.prim;
        PathVertex pv{row, {1.0, 1.0, 1.0}, {0.0, 0.0, 0.0}};
        if (p.tex_res > 0) tex_lookup(p.tex, p.tex_res, row, h.u, h.v, pv.tex);
        // diffuse albedo: the quad's albedo modulated by its texture
        double a[3];
        for (int c = 0; c < 3; ++c) a[c] = albedo[3 * row + c] * pv.tex[c];
        V3 n = world_normal(s, h.inst, h.prim);
        if (dot(n, d) > 0.0) n = -1.0 * n;
        V3 hp = o + h.t * d;
        V3 sp = spawn_point(hp, n);
        if (log_rays) {
            double* r = log_rays + kRayRec * (i - 1) + 6;
            r[0] = sp.x, r[1] = sp.y, r[2] = sp.z;
        }
        if (sun) {
            double cl = dot(n, l);
            if (cl > 0.0) {
                if (i <= 16) shadow_bits |= 1u << (2 * (i - 1));
                bool occ = any_hit(s, sp, l, 0.0, kInf, 0);
                if (occ) {
                    if (i <= 16) shadow_bits |= 2u << (2 * (i - 1));
                } else {
                    for (int c = 0; c < 3; ++c) {
                        pv.nee[c] = p.sun_E[c] * cl / kPi;
                        L[c] += beta[c] * a[c] * pv.nee[c];
                    }
                }
            }
        }
        if (p.n_lights > 0) {
            double xl[4], w[3], dist;
            V3 ld;
            draw4(p.seed, pix, smp, kLightStream + i, xl);
            if (light_sample(p.lights, p.n_lights, xl, sp, n, &ld, &dist, w)) {
                if (i <= 16) light_bits |= 1u << (2 * (i - 1));
                if (log_rays) {
                    double* r = log_rays + kRayRec * (i - 1) + 9;
                    r[0] = ld.x, r[1] = ld.y, r[2] = ld.z, r[3] = dist;
                }
                if (any_hit(s, sp, ld, 0.0, dist, 0)) {
                    if (i <= 16) light_bits |= 2u << (2 * (i - 1));
                } else {
                    for (int c = 0; c < 3; ++c) {
                        pv.nee[c] += w[c] / kPi;
                        L[c] += beta[c] * a[c] * (w[c] / kPi);
                    }
                }
            }
        }
        if (rec) rec->verts.push_back(pv);
        for (int c = 0; c < 3; ++c) beta[c] *= a[c];
        if (i == p.max_depth) break;
        draw4(p.seed, pix, smp, i, xi);
        d = sample_cosine(n, xi[0], xi[1]);
        o = sp;
    }
    if (log_shadow) *log_shadow = shadow_bits;
    if (lg.light) *lg.light = light_bits;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void ora_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    philox(ctr, key, out);
}

ora_scene* ora_scene_new(uint32_t n_mesh, const float* const* verts, const uint32_t* n_verts,
                         const uint32_t* const* quads, const uint32_t* n_quads, uint64_t n_inst,
                         const float* xforms, const uint32_t* mesh_ids) {
    ora_scene* s = new ora_scene();
    s->meshes.resize(n_mesh);
    std::vector<int> ids(n_mesh);
    for (uint32_t m = 0; m < n_mesh; ++m) ids[m] = (int)m;
    uint64_t base = 0;
    for (uint32_t m = 0; m < n_mesh; ++m) {
        Mesh& M = s->meshes[m];
        M.albedo_base = base;
        base += n_quads[m];
        M.verts.resize(n_verts[m]);
        for (uint32_t k = 0; k < n_verts[m]; ++k)
            M.verts[k] = mk(verts[m][3 * k], verts[m][3 * k + 1], verts[m][3 * k + 2]);
        M.quads.assign(quads[m], quads[m] + 4 * (size_t)n_quads[m]);
    }
    s->n_quads = base;
    parallel_for(n_mesh, 0, [&](uint64_t m) {
        Mesh& M = s->meshes[m];
        uint32_t nq = (uint32_t)(M.quads.size() / 4);
        std::vector<Box> boxes(nq);
        V3 v[4];
        M.box = empty_box();
        for (uint32_t q = 0; q < nq; ++q) {
            M.quad(q, v);
            boxes[q] = empty_box();
            for (int k = 0; k < 4; ++k) grow(boxes[q], v[k]);
            grow(M.box, boxes[q]);
        }
        M.bvh = build_bvh(boxes);
    });
    s->inst.resize(n_inst);
    std::vector<Box> wboxes(n_inst);
    parallel_for(n_inst, 0, [&](uint64_t i) {
        Instance& I = s->inst[i];
        const float* x = xforms + 12 * i;
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) I.A[3 * r + c] = x[4 * r + c];
            I.b[r] = x[4 * r + 3];
        }
        inverse3(I.A, I.Ainv);
        I.mesh = mesh_ids[i];
        const Box& mb = s->meshes[I.mesh].box;
        Box wb = empty_box();
        for (int k = 0; k < 8; ++k) {
            V3 c = mk((k & 1) ? mb.hi.x : mb.lo.x, (k & 2) ? mb.hi.y : mb.lo.y,
                      (k & 4) ? mb.hi.z : mb.lo.z);
            grow(wb, mul3(I.A, c) + mk(I.b[0], I.b[1], I.b[2]));
        }
        I.world_box = padded(wb);
        wboxes[i] = I.world_box;
    });
    s->tlas = build_bvh(wboxes);
    return s;
}

void ora_scene_free(ora_scene* s) { delete s; }

uint64_t ora_scene_n_quads(const ora_scene* s) { return s->n_quads; }

int ora_intersect_quad(const double o[3], const double d[3], double tmin, double tmax,
                       const double v[12], double* t, double* u, double* w) {
    V3 q[4];
    for (int k = 0; k < 4; ++k) q[k] = mk(v[3 * k], v[3 * k + 1], v[3 * k + 2]);
    return quad_hit(mk(o[0], o[1], o[2]), mk(d[0], d[1], d[2]), q, tmin, tmax, t, u, w) ? 1 : 0;
}

void ora_trace_closest(const ora_scene* s, const float* rays, uint64_t n, int mode, double* t,
                       uint32_t* inst, uint32_t* prim, double* u, double* v, int nthreads) {
    parallel_for(n, nthreads, [&](uint64_t i) {
        const float* r = rays + 8 * i;
        HitRec h = closest(*s, mk(r[0], r[1], r[2]), mk(r[4], r[5], r[6]), r[3], r[7], mode);
        t[i] = h.t;
        inst[i] = h.inst;
        prim[i] = h.prim;
        if (u) u[i] = h.u;
        if (v) v[i] = h.v;
    });
}

void ora_trace_any(const ora_scene* s, const float* rays, uint64_t n, int mode,
                   uint8_t* occluded, int nthreads) {
    parallel_for(n, nthreads, [&](uint64_t i) {
        const float* r = rays + 8 * i;
        occluded[i] =
            any_hit(*s, mk(r[0], r[1], r[2]), mk(r[4], r[5], r[6]), r[3], r[7], mode) ? 1 : 0;
    });
}

void ora_camera_ray(const ora_view* v, uint32_t x, uint32_t y, double xi1, double xi2,
                    double o[3], double d[3]) {
    V3 oo, dd;
    camera_ray(*v, x + xi1, y + xi2, &oo, &dd);
    o[0] = oo.x;
    o[1] = oo.y;
    o[2] = oo.z;
    d[0] = dd.x;
    d[1] = dd.y;
    d[2] = dd.z;
}

void ora_tex_lookup(const float* tex, uint32_t res, uint64_t row, double u, double v, double out[3]) {
    tex_lookup(tex, res, row, u, v, out);
}

int ora_light_sample(const float* lights, uint32_t n, const double xi[3], const double x[3],
                     const double nx[3], double dir[3], double* dist, double w[3]) {
    V3 d;
    if (!light_sample(lights, n, xi, mk(x[0], x[1], x[2]), mk(nx[0], nx[1], nx[2]), &d, dist, w)) return 0;
    dir[0] = d.x;
    dir[1] = d.y;
    dir[2] = d.z;
    return 1;
}

void ora_sample_cosine(const double n[3], double xi1, double xi2, double out[3]) {
    V3 r = sample_cosine(mk(n[0], n[1], n[2]), xi1, xi2);
    out[0] = r.x;
    out[1] = r.y;
    out[2] = r.z;
}

int ora_render(const ora_scene* s, const ora_view* view, const float* albedo,
               const ora_params* p, const int64_t* pixels, uint64_t n_pix, double* rgb,
               uint32_t* log_inst, uint32_t* log_prim, uint32_t* log_shadow, uint32_t* log_light,
               double* log_rays, uint64_t* n_escaped, uint64_t* n_truncated, int nthreads) {
    if (p->max_depth == 0 || p->max_depth > 256) return -1;
    if ((p->tex_res > 0 && !p->tex) || (p->n_lights > 0 && !p->lights)) return -1;
    std::atomic<uint64_t> esc{0}, trunc{0};
    const uint32_t D = p->max_depth, spp = view->spp;
    parallel_for(n_pix, nthreads, [&](uint64_t k) {
        int64_t idx = pixels ? pixels[k] : (int64_t)k;
        uint32_t x = (uint32_t)(idx % view->w), y = (uint32_t)(idx / view->w);
        double acc[3] = {0.0, 0.0, 0.0};
        PathRecord rec;
        for (uint32_t smp = 0; smp < spp; ++smp) {
            uint64_t path = k * spp + smp;
            double L[3];
            PathLogs lg;
            lg.inst = log_inst ? log_inst + path * D : nullptr;
            lg.prim = log_prim ? log_prim + path * D : nullptr;
            lg.shadow = log_shadow ? log_shadow + path : nullptr;
            lg.light = log_light ? log_light + path : nullptr;
            lg.rays = log_rays ? log_rays + path * D * kRayRec : nullptr;
            trace_path(*s, *view, albedo, *p, x, y, smp, L, &rec, lg);
            if (log_inst) {
                for (uint32_t i = (uint32_t)rec.verts.size() + (rec.escaped ? 1 : 0); i < D; ++i) {
                    log_inst[path * D + i] = kNone;
                    log_prim[path * D + i] = kNone;
                }
            }
            if (rec.escaped)
                esc++;
            else
                trunc++;
            for (int c = 0; c < 3; ++c) acc[c] += L[c];
        }
        for (int c = 0; c < 3; ++c) rgb[3 * k + c] = acc[c] / (double)spp;
    });
    if (n_escaped) *n_escaped = esc.load();
    if (n_truncated) *n_truncated = trunc.load();
    return 0;
}

int ora_render_grad(const ora_scene* s, const ora_view* view, const float* albedo,
                    const ora_params* p, const int64_t* pixels, uint64_t n_pix,
                    const double* dimage, double* grad, int nthreads) {
    if (p->max_depth == 0 || p->max_depth > 256) return -1;
    if ((p->tex_res > 0 && !p->tex) || (p->n_lights > 0 && !p->lights)) return -1;
    if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
    // Per-thread sparse (row, channel, value) lists, summed at the end.
    struct Entry {
        uint64_t row;
        int c;
        double v;
    };
    std::vector<std::vector<Entry>> parts(n_pix);
    const uint32_t spp = view->spp;
    parallel_for(n_pix, nthreads, [&](uint64_t k) {
        int64_t idx = pixels ? pixels[k] : (int64_t)k;
        uint32_t x = (uint32_t)(idx % view->w), y = (uint32_t)(idx / view->w);
        PathRecord rec;
        std::vector<Entry>& out = parts[k];
        for (uint32_t smp = 0; smp < spp; ++smp) {
            double L[3];
            trace_path(*s, *view, albedo, *p, x, y, smp, L, &rec, PathLogs{});
            const size_t m = rec.verts.size();
            for (int c = 0; c < 3; ++c) {
                double w = dimage[3 * k + c] / (double)spp;
                if (w == 0.0) continue;
                std::vector<double> a(m);
                for (size_t j = 0; j < m; ++j)
                    a[j] = albedo[3 * rec.verts[j].albedo_row + c] * rec.verts[j].tex[c];
                // Monomials: for each vertex k (1-based) the NEE term
                // (prod_{j<=k} a_j t_j) * nee_k, a_j the quad albedo and t_j its
                // texture factor; if the path escaped after its last vertex,
                // the term (prod_{j<=m} a_j t_j) * env.  Differentiate each
                // monomial by each of its albedo factors (d(a_j t_j)/da_j = t_j).
                for (size_t kk = 1; kk <= m; ++kk) {
                    double coef = rec.verts[kk - 1].nee[c];
                    if (kk == m && rec.escaped) coef += p->env[c];
                    if (coef == 0.0) continue;
                    for (size_t j = 0; j < kk; ++j) {
                        double prod = coef * rec.verts[j].tex[c];
                        for (size_t l = 0; l < kk; ++l)
                            if (l != j) prod *= a[l];
                        out.push_back(Entry{rec.verts[j].albedo_row, c, w * prod});
                    }
                }
            }
        }
    });
    for (auto& part : parts)
        for (const Entry& e : part) grad[3 * e.row + e.c] += e.v;
    return 0;
}

}  // extern "C"

// C ABI of the qrt library (include/qrt.h): argument checking, scene
// construction and upload, work-counter slots, launch configuration, CUDA
// graphs and the device error word.
#include "qrt.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bvh_build.h"
#include "lbvh.h"
#include "launch.h"
#include "radix_sort.h"
#include "wavefront.h"

using namespace qrt;

namespace {

// Last error message of the calling thread, in a fixed buffer so that
// reporting an error never allocates.
thread_local char g_err[512];

int fail(int code, const char* msg) {
    std::snprintf(g_err, sizeof(g_err), "%s", msg);
    return code;
}

int fail(int code, const std::string& msg) { return fail(code, msg.c_str()); }

int cuda_fail(cudaError_t e, const char* what) {
    std::snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? QRT_ERR_OOM : QRT_ERR_CUDA;
}

constexpr int kCounterSlots = 64;
constexpr size_t kSlotStride = 128;  // bytes between counters (own cache line)

}  // namespace

// CUDA events around each wavefront stage launch, accumulated per stage
// until read by qrt_stage_times (one stream at a time per scene).
struct StageTimer : StageHook {
    struct Rec {
        int stage;
        cudaEvent_t a, b;
    };
    std::mutex mu;
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> done;
    Rec open[kStages] = {};

    cudaEvent_t take() {
        cudaEvent_t e = nullptr;
        if (!pool.empty()) {
            e = pool.back();
            pool.pop_back();
        } else {
            cudaEventCreate(&e);
        }
        return e;
    }
    void begin(int stage, cudaStream_t s) override {
        std::lock_guard<std::mutex> g(mu);
        open[stage] = Rec{stage, take(), nullptr};
        cudaEventRecord(open[stage].a, s);
    }
    void end(int stage, cudaStream_t s) override {
        std::lock_guard<std::mutex> g(mu);
        Rec r = open[stage];
        r.b = take();
        cudaEventRecord(r.b, s);
        done.push_back(r);
    }
    void read(double* ms, uint32_t* n, bool reset) {
        std::lock_guard<std::mutex> g(mu);
        for (int k = 0; k < kStages; ++k) {
            ms[k] = 0.0;
            n[k] = 0;
        }
        for (const Rec& r : done) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.stage] += t;
            n[r.stage]++;
        }
        if (reset) {
            for (const Rec& r : done) {
                pool.push_back(r.a);
                pool.push_back(r.b);
            }
            done.clear();
        }
    }
    ~StageTimer() override {
        for (const Rec& r : done) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
};

// Scratch of one stream: a work counter for the single-kernel renderer and
// the wavefront workspace (grown on demand, outside stream capture).
struct StreamSlot {
    unsigned long long* counter = nullptr;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    WaveStreams ov;  // second stream for overlapping shadow and closest-hit launches
};

void destroy_streams(WaveStreams& w) {
    if (w.fork) cudaEventDestroy(w.fork);
    if (w.join) cudaEventDestroy(w.join);
    if (w.aux) cudaStreamDestroy(w.aux);
    w = WaveStreams{};
}

cudaError_t create_streams(WaveStreams& w) {
    cudaError_t e = cudaStreamCreateWithFlags(&w.aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.join, cudaEventDisableTiming);
    if (e != cudaSuccess) destroy_streams(w);
    return e;
}

struct qrt_scene_s {
    int device = -1;
    int sm_count = 0;
    DevScene S{};
    void* d_nodes = nullptr;
    void* d_quads = nullptr;
    void* d_prim = nullptr;
    void* d_inst = nullptr;
    void* d_inst64 = nullptr;
    uint32_t* d_err = nullptr;
    char* d_counters = nullptr;  // kCounterSlots counters, kSlotStride apart
    std::mutex mu;
    std::unordered_map<cudaStream_t, int> slot_of;
    std::vector<StreamSlot> slots;
    int next_slot = 0;
    qrt_scene_stats stats{};
    StageTimer timer;

    // Calls on one stream are ordered, so they may share scratch; different
    // streams get different slots (up to kCounterSlots, then reused).
    StreamSlot& slot_for(cudaStream_t s) {
        std::lock_guard<std::mutex> g(mu);
        if (slots.empty()) slots.resize(kCounterSlots);
        auto it = slot_of.find(s);
        int k;
        if (it != slot_of.end()) {
            k = it->second;
        } else {
            k = next_slot % kCounterSlots;
            next_slot++;
            slot_of[s] = k;
        }
        StreamSlot& sl = slots[k];
        sl.counter = reinterpret_cast<unsigned long long*>(d_counters + kSlotStride * k);
        return sl;
    }
};

struct qrt_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long* d_counter = nullptr;
    void* ws = nullptr;
    int device = -1;
};

namespace {

void free_scene(qrt_scene_s* s) {
    if (!s) return;
    cudaFree(s->d_nodes);
    cudaFree(s->d_quads);
    cudaFree(s->d_prim);
    cudaFree(s->d_inst);
    cudaFree(s->d_inst64);
    cudaFree(s->d_err);
    cudaFree(s->d_counters);
    for (StreamSlot& sl : s->slots) {
        cudaFree(sl.ws);
        destroy_streams(sl.ov);
    }
    delete s;
}

int check_device(const qrt_scene_s* s) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != s->device) {
        std::snprintf(g_err, sizeof(g_err), "scene belongs to device %d but device %d is current",
                      s->device, dev);
        return QRT_ERR_INVALID_ARG;
    }
    return QRT_OK;
}

Tune resolve_tuning(const qrt_tuning* t) {
    Tune r;
    if (!t) return r;
    if (t->block) r.block = (int)t->block;
    if (t->blocks_per_sm) r.blocks_per_sm = (int)t->blocks_per_sm;
    if (t->batch) r.batch = (int)t->batch;
    if (t->stack) r.stack = (int)t->stack;
    if (t->fetch) r.fetch = (int)t->fetch;
    if (t->occupancy) r.occupancy = (int)t->occupancy;
    if (t->mode) r.mode = (int)t->mode;
    if (t->chunk_log2) r.chunk_log2 = (int)t->chunk_log2;
    return r;
}

// Default wavefront chunk: the smallest 2^k >= the call's paths, k in
// [10, kFitChunkMax].  One chunk per call where it fits: every chunk pays
// its own run of draining launches, and a whole mid frame (2^22 paths) in
// one chunk renders 1.12x faster than in two (a Moana-scale frame of 2^25
// paths: 1.03x faster than in two).  2^25 paths of workspace is about 5.5 GB
// (adjoint included) per stream, 2 % of GB300's memory.
constexpr int kFitChunkMax = 25;

// Pixels a view renders: its crop rectangle, or the whole frame.
uint64_t region_pixels(const qrt_view& v) {
    if (v.crop_w == 0 && v.crop_h == 0) return (uint64_t)v.w * v.h;
    return (uint64_t)v.crop_w * v.crop_h;
}

void fit_chunk(Tune& t, const qrt_view* views, uint32_t n_views) {
    if (t.chunk_log2 != 0) return;
    uint64_t paths = 0;
    for (uint32_t v = 0; v < n_views; ++v) paths += region_pixels(views[v]) * views[v].spp;
    int k = 10;
    while (k < kFitChunkMax && (1ull << k) < paths) ++k;
    t.chunk_log2 = k;
}

int validate_tuning(const Tune& t) {
    if (t.block != 64 && t.block != 128 && t.block != 192 && t.block != 256)
        return fail(QRT_ERR_INVALID_ARG, "tuning.block must be 64, 128, 192 or 256");
    if (t.stack != 32 && t.stack != 64)
        return fail(QRT_ERR_INVALID_ARG, "tuning.stack must be 32 or 64");
    if (t.fetch != 16 && t.fetch != 32)
        return fail(QRT_ERR_INVALID_ARG, "tuning.fetch must be 16 or 32");
    if (t.batch < 1 || t.batch > 64) return fail(QRT_ERR_INVALID_ARG, "tuning.batch must be 1..64");
    if (t.blocks_per_sm < 0 || t.blocks_per_sm > 32)
        return fail(QRT_ERR_INVALID_ARG, "tuning.blocks_per_sm must be 0..32");
    if (t.occupancy != 16 && t.occupancy != 24 && t.occupancy != 32 && t.occupancy != 40 &&
        t.occupancy != 48)
        return fail(QRT_ERR_INVALID_ARG, "tuning.occupancy must be 0, 16, 24, 32, 40 or 48");
    if (t.mode < 1 || t.mode > 2) return fail(QRT_ERR_INVALID_ARG, "tuning.mode must be 0, 1 or 2");
    if (t.chunk_log2 != 0 && (t.chunk_log2 < 10 || t.chunk_log2 > 26))
        return fail(QRT_ERR_INVALID_ARG, "tuning.chunk_log2 must be 0 or 10..26");
    return QRT_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// 3x3 inverse by the adjugate, FP64.  Returns false for singular input.
bool inverse3(const double* m, double* r) {
    double c00 = m[4] * m[8] - m[5] * m[7];
    double c01 = m[5] * m[6] - m[3] * m[8];
    double c02 = m[3] * m[7] - m[4] * m[6];
    double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
    double scale = 0.0;
    for (int k = 0; k < 9; ++k) scale = std::max(scale, std::fabs(m[k]));
    if (!std::isfinite(det) || std::fabs(det) <= 1e-30 * scale * scale * scale || scale == 0.0)
        return false;
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
    return true;
}

const float kFInfHost = std::numeric_limits<float>::infinity();

BuildOpts resolve_build(const qrt_build_opts* o) {
    BuildOpts b;
    if (!o) return b;
    if (o->max_leaf) b.max_leaf = o->max_leaf;
    if (o->sah_bins) b.sah_bins = o->sah_bins;
    b.threads = o->threads;
    b.degenerate = o->degenerate;
    if (o->inst_boxes) b.inst_box_level = o->inst_boxes - 1;
    b.tlas_builder = o->tlas_builder;
    b.blas_builder = o->blas_builder;
    return b;
}

// The TLAS with the builder the options name (checked by the caller).
bool make_tlas(const std::vector<FBox>& boxes, const BuildOpts& bo, TlasResult& out, std::string& err) {
    if (bo.tlas_builder == 0) return build_tlas(boxes, bo, out, err);
    return build_tlas_lbvh(boxes, bo.tlas_builder == 1, out, err);
}

template <class T>
cudaError_t upload(void** dptr, const std::vector<T>& v) {
    size_t bytes = std::max<size_t>(v.size() * sizeof(T), 64);
    cudaError_t e = cudaMalloc(dptr, bytes);
    if (e != cudaSuccess) return e;
    if (!v.empty()) e = cudaMemcpy(*dptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

extern "C" {

const char* qrt_last_error(void) { return g_err; }

int qrt_version(void) { return QRT_VERSION; }

int qrt_scene_create(const qrt_mesh* meshes, uint32_t n_mesh, const float* xforms,
                     const uint32_t* mesh_ids, uint64_t n_inst, const qrt_build_opts* opts,
                     qrt_scene* out) {
    if (!out) return fail(QRT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!meshes || n_mesh == 0) return fail(QRT_ERR_INVALID_ARG, "no meshes");
    if (n_inst > 0 && (!xforms || !mesh_ids))
        return fail(QRT_ERR_INVALID_ARG, "xforms or mesh_ids is NULL");
    if (n_inst > (uint64_t)kMaxLocalIndex) return fail(QRT_ERR_INVALID_ARG, "too many instances");
    for (uint32_t m = 0; m < n_mesh; ++m) {
        if (!meshes[m].verts || !meshes[m].quads || meshes[m].n_quads == 0 || meshes[m].n_verts == 0)
            return fail(QRT_ERR_INVALID_ARG, "mesh " + std::to_string(m) + " is empty or NULL");
    }
    for (uint64_t i = 0; i < n_inst; ++i)
        if (mesh_ids[i] >= n_mesh)
            return fail(QRT_ERR_INVALID_ARG, "instance " + std::to_string(i) + " names mesh " +
                                                 std::to_string(mesh_ids[i]) + " out of range");
    if (opts && opts->inst_boxes > 6) return fail(QRT_ERR_INVALID_ARG, "build_opts.inst_boxes must be 0..6");
    if (opts && opts->tlas_builder > 2) return fail(QRT_ERR_INVALID_ARG, "build_opts.tlas_builder must be 0..2");
    if (opts && opts->blas_builder > 2) return fail(QRT_ERR_INVALID_ARG, "build_opts.blas_builder must be 0..2");
    if (opts && opts->blas_builder && opts->degenerate)
        return fail(QRT_ERR_INVALID_ARG, "build_opts.degenerate needs the host BLAS builder");
    const BuildOpts bo = resolve_build(opts);
    auto t0 = std::chrono::steady_clock::now();
    // wall time of each build phase (reported in qrt_scene_stats)
    double phase[6] = {0, 0, 0, 0, 0, 0};
    auto lap_t = t0;
    auto lap = [&](int k) {
        const auto now = std::chrono::steady_clock::now();
        phase[k] += std::chrono::duration<double>(now - lap_t).count();
        lap_t = now;
    };

    // 1. one BLAS per mesh, largest first, on a pool of host threads
    std::vector<BlasResult> blas(n_mesh);
    std::vector<std::string> errs(n_mesh);
    std::vector<uint32_t> order(n_mesh);
    for (uint32_t m = 0; m < n_mesh; ++m) order[m] = m;
    std::sort(order.begin(), order.end(),
              [&](uint32_t a, uint32_t b) { return meshes[a].n_quads > meshes[b].n_quads; });
    if (bo.blas_builder) {  // all meshes at once, linear BVHs
        std::vector<MeshView> mv(n_mesh);
        for (uint32_t m = 0; m < n_mesh; ++m)
            mv[m] = MeshView{meshes[m].verts, meshes[m].n_verts, meshes[m].quads, meshes[m].n_quads};
        std::string berr;
        if (!build_blases_lbvh(mv, std::max(1u, std::min(bo.max_leaf, 8u)), bo.blas_builder == 1, blas, berr))
            return fail(berr.compare(0, 5, "CUDA:") == 0 ? QRT_ERR_CUDA : QRT_ERR_INVALID_ARG, "BLAS: " + berr);
    } else {
        unsigned nt = bo.threads ? bo.threads : std::max(1u, std::thread::hardware_concurrency());
        nt = std::min<unsigned>(nt, n_mesh);
        std::atomic<uint32_t> next{0};
        auto work = [&]() {
            for (;;) {
                uint32_t k = next.fetch_add(1);
                if (k >= n_mesh) break;
                uint32_t m = order[k];
                build_blas(meshes[m].verts, meshes[m].n_verts, meshes[m].quads, meshes[m].n_quads,
                           bo, blas[m], errs[m]);
            }
        };
        std::vector<std::thread> th;
        for (unsigned k = 1; k < nt; ++k) th.emplace_back(work);
        work();
        for (auto& t : th) t.join();
    }
    for (uint32_t m = 0; m < n_mesh; ++m)
        if (!errs[m].empty()) return fail(QRT_ERR_INVALID_ARG, "mesh " + std::to_string(m) + ": " + errs[m]);
    lap(0);
    // Verify every BLAS before anything reaches the device: all child and
    // item indices in range, each quad referenced once, boxes conservative.
    {
        std::atomic<uint32_t> next{0};
        unsigned nt = bo.threads ? bo.threads : std::max(1u, std::thread::hardware_concurrency());
        nt = std::min<unsigned>(nt, n_mesh);
        auto work = [&]() {
            for (;;) {
                uint32_t m = next.fetch_add(1);
                if (m >= n_mesh) break;
                std::vector<FBox> items(blas[m].quads.size());
                for (size_t k = 0; k < items.size(); ++k) {
                    const float* v = blas[m].quads[k].v;
                    for (int a = 0; a < 3; ++a) {
                        items[k].lo[a] = std::min(std::min(v[a], v[3 + a]), std::min(v[6 + a], v[9 + a]));
                        items[k].hi[a] = std::max(std::max(v[a], v[3 + a]), std::max(v[6 + a], v[9 + a]));
                    }
                }
                uint32_t d = 0;
                if (!check_wide(blas[m].nodes, items, errs[m], &d)) errs[m] = "BLAS check: " + errs[m];
            }
        };
        std::vector<std::thread> th;
        for (unsigned k = 1; k < nt; ++k) th.emplace_back(work);
        work();
        for (auto& t : th) t.join();
    }
    for (uint32_t m = 0; m < n_mesh; ++m)
        if (!errs[m].empty()) return fail(QRT_ERR_INVALID_ARG, "mesh " + std::to_string(m) + ": " + errs[m]);

    lap(1);
    // 2. global layout: BLAS nodes mesh by mesh, then the TLAS
    std::vector<uint64_t> node_base(n_mesh), quad_base(n_mesh);
    uint64_t nn = 0, nq = 0;
    uint32_t max_blas_depth = 0;
    for (uint32_t m = 0; m < n_mesh; ++m) {
        node_base[m] = nn;
        quad_base[m] = nq;
        nn += blas[m].nodes.size();
        nq += blas[m].quads.size();
        max_blas_depth = std::max(max_blas_depth, blas[m].depth);
    }
    if (nq > 0xFFFFFFFFull || nn > 0xFFFFFFFFull)
        return fail(QRT_ERR_INVALID_ARG, "scene exceeds 2^32 quads or nodes");

    // 3. instances: FP64 inverse, world boxes
    std::vector<InstDev> inst(n_inst);
    std::vector<InstDev64> inst64(n_inst);
    std::vector<FBox> wbox(n_inst);
    std::vector<float> meshR(n_mesh);
    std::vector<std::vector<FBox>> mesh_cut(n_mesh);
    for (uint32_t m = 0; m < n_mesh; ++m) {
        float r = 0.f;
        for (int a = 0; a < 3; ++a)
            r = std::max(r, std::max(std::fabs(blas[m].box.lo[a]), std::fabs(blas[m].box.hi[a])));
        meshR[m] = r;
        mesh_cut[m] = level_boxes(blas[m].nodes, bo.inst_box_level);
    }
    // per instance: FP64 inverse, float records, world box (threads over
    // ranges of instances; the first bad instance is reported)
    std::atomic<uint64_t> bad_inst{~0ull};
    auto setup_instance = [&](uint64_t i) -> bool {
        const float* x = xforms + 12 * i;
        double A[9], Ai[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) A[3 * r + c] = x[4 * r + c];
        bool finite = true;
        for (int k = 0; k < 12; ++k) finite = finite && std::isfinite(x[k]);
        if (!finite || !inverse3(A, Ai)) return false;
        InstDev& I = inst[i];
        std::memset(&I, 0, sizeof(I));
        std::memset(&inst64[i], 0, sizeof(InstDev64));
        double na = 0.0, ni = 0.0;  // infinity norms (max row sum)
        for (int r = 0; r < 3; ++r) {
            na = std::max(na, std::fabs(A[3 * r]) + std::fabs(A[3 * r + 1]) + std::fabs(A[3 * r + 2]));
            ni = std::max(ni, std::fabs(Ai[3 * r]) + std::fabs(Ai[3 * r + 1]) + std::fabs(Ai[3 * r + 2]));
        }
        for (int k = 0; k < 9; ++k) {
            I.w[k] = (float)Ai[k];
            inst64[i].w[k] = Ai[k];
        }
        I.c[0] = x[3];
        I.c[1] = x[7];
        I.c[2] = x[11];
        const uint32_t m = mesh_ids[i];
        I.node_base = (uint32_t)node_base[m];
        I.quad_base = (uint32_t)quad_base[m];
        I.R = meshR[m];
        I.kappa = (float)(na * ni);
        // the transformed root box and the union of the transformed cut
        // boxes both contain the instance's geometry, so their intersection
        // does too
        FBox wb = transform_box(blas[m].box, x);
        if (!mesh_cut[m].empty()) {
            FBox u;
            for (int a = 0; a < 3; ++a) {
                u.lo[a] = kFInfHost;
                u.hi[a] = -kFInfHost;
            }
            for (const FBox& cb : mesh_cut[m]) {
                const FBox t = transform_box(cb, x);
                for (int a = 0; a < 3; ++a) {
                    u.lo[a] = std::min(u.lo[a], t.lo[a]);
                    u.hi[a] = std::max(u.hi[a], t.hi[a]);
                }
            }
            for (int a = 0; a < 3; ++a) {
                wb.lo[a] = std::max(wb.lo[a], u.lo[a]);
                wb.hi[a] = std::min(wb.hi[a], u.hi[a]);
            }
        }
        wbox[i] = wb;
        return true;
    };
    {
        unsigned nt = bo.threads ? bo.threads : std::max(1u, std::thread::hardware_concurrency());
        const uint64_t chunk = 4096;
        const uint64_t n_chunks = (n_inst + chunk - 1) / chunk;
        nt = (unsigned)std::min<uint64_t>(nt, std::max<uint64_t>(1, n_chunks));
        std::atomic<uint64_t> next{0};
        auto work = [&]() {
            for (;;) {
                const uint64_t c = next.fetch_add(1);
                if (c >= n_chunks) break;
                const uint64_t end = std::min(n_inst, (c + 1) * chunk);
                for (uint64_t i = c * chunk; i < end; ++i) {
                    if (!setup_instance(i)) {
                        uint64_t cur = bad_inst.load();
                        while (i < cur && !bad_inst.compare_exchange_weak(cur, i)) {
                        }
                    }
                }
            }
        };
        std::vector<std::thread> th;
        for (unsigned k = 1; k < nt; ++k) th.emplace_back(work);
        work();
        for (auto& t : th) t.join();
    }
    if (bad_inst.load() != ~0ull)
        return fail(QRT_ERR_INVALID_ARG, "instance " + std::to_string(bad_inst.load()) +
                                             " has a non-finite or singular transform");
    // Spot check of the instance bounds: for up to 256 evenly spaced
    // instances (at most 2^23 vertices in all), every vertex of every quad,
    // mapped to world space in FP64, lies inside the instance's TLAS box.
    {
        const uint64_t samples = std::min<uint64_t>(n_inst, 256);
        uint64_t budget = 1ull << 23;
        for (uint64_t k = 0; k < samples; ++k) {
            const uint64_t i = k * n_inst / samples;
            const uint32_t m = mesh_ids[i];
            const uint64_t nv = 4ull * blas[m].quads.size();
            if (nv > budget) continue;
            budget -= nv;
            const float* x = xforms + 12 * i;
            for (const QuadDev& q : blas[m].quads)
                for (int v = 0; v < 4; ++v)
                    for (int r = 0; r < 3; ++r) {
                        const double w = (double)x[4 * r] * q.v[3 * v] + (double)x[4 * r + 1] * q.v[3 * v + 1] +
                                         (double)x[4 * r + 2] * q.v[3 * v + 2] + (double)x[4 * r + 3];
                        if (!(w >= (double)wbox[i].lo[r] && w <= (double)wbox[i].hi[r]))
                            return fail(QRT_ERR_INVALID_ARG, "internal: instance " + std::to_string(i) +
                                                                 " lies outside its TLAS box");
                    }
        }
    }
    lap(2);
    TlasResult tlas;
    std::string terr;
    if (!make_tlas(wbox, bo, tlas, terr))
        return fail(terr.compare(0, 5, "CUDA:") == 0 ? QRT_ERR_CUDA : QRT_ERR_INVALID_ARG, "TLAS: " + terr);
    {
        uint32_t d = 0;
        if (!check_wide(tlas.nodes, wbox, terr, &d)) return fail(QRT_ERR_INVALID_ARG, "TLAS check: " + terr);
    }
    const uint64_t tlas_base = nn;
    if (nn + tlas.nodes.size() > 0xFFFFFFFFull) return fail(QRT_ERR_INVALID_ARG, "too many nodes");
    float R_top = 0.f;
    for (const FBox& b : wbox)
        for (int a = 0; a < 3; ++a) R_top = std::max(R_top, std::max(std::fabs(b.lo[a]), std::fabs(b.hi[a])));

    lap(3);
    // 4. concatenate: inner node references stay local to their structure
    std::vector<QNode> nodes;
    nodes.reserve(nn + tlas.nodes.size());
    std::vector<QuadDev> quads;
    quads.reserve(nq);
    std::vector<uint32_t> prim;
    prim.reserve(nq);
    for (uint32_t m = 0; m < n_mesh; ++m) {
        nodes.insert(nodes.end(), blas[m].nodes.begin(), blas[m].nodes.end());
        quads.insert(quads.end(), blas[m].quads.begin(), blas[m].quads.end());
        prim.insert(prim.end(), blas[m].prim.begin(), blas[m].prim.end());
        std::vector<QNode>().swap(blas[m].nodes);
        std::vector<QuadDev>().swap(blas[m].quads);
        std::vector<uint32_t>().swap(blas[m].prim);
    }
    nodes.insert(nodes.end(), tlas.nodes.begin(), tlas.nodes.end());
    const double build_s =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    lap(4);

    // 5. upload
    qrt_scene_s* s = new qrt_scene_s();
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "cudaGetDevice");
    }
    e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess) e = upload(&s->d_nodes, nodes);
    if (e == cudaSuccess) e = upload(&s->d_quads, quads);
    if (e == cudaSuccess) e = upload(&s->d_prim, prim);
    if (e == cudaSuccess) e = upload(&s->d_inst, inst);
    if (e == cudaSuccess) e = upload(&s->d_inst64, inst64);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_err, 2 * sizeof(uint32_t));
    if (e == cudaSuccess) {
        const uint32_t init[2] = {0u, 0xFFFFFFFFu};
        e = cudaMemcpy(s->d_err, init, sizeof(init), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_counters, kCounterSlots * kSlotStride);
    if (e == cudaSuccess) e = cudaMemset(s->d_counters, 0, kCounterSlots * kSlotStride);
    if (e != cudaSuccess) {
        free_scene(s);
        return cuda_fail(e, "scene upload");
    }
    s->S.nodes = static_cast<const QNode*>(s->d_nodes);
    s->S.quads = static_cast<const QuadDev*>(s->d_quads);
    s->S.prim = static_cast<const uint32_t*>(s->d_prim);
    s->S.inst = static_cast<const InstDev*>(s->d_inst);
    s->S.inst64 = static_cast<const InstDev64*>(s->d_inst64);
    s->S.tlas_base = (uint32_t)tlas_base;
    s->S.n_inst = (uint32_t)n_inst;
    s->S.R_top = R_top;
    s->S.err = s->d_err;
    s->stats.n_meshes = n_mesh;
    s->stats.n_instances = n_inst;
    s->stats.n_quads = nq;
    s->stats.blas_nodes = nn;
    s->stats.tlas_nodes = tlas.nodes.size();
    s->stats.device_bytes = nodes.size() * sizeof(QNode) + quads.size() * sizeof(QuadDev) +
                            prim.size() * 4 + inst.size() * (sizeof(InstDev) + sizeof(InstDev64));
    s->stats.max_blas_depth = max_blas_depth;
    s->stats.tlas_depth = tlas.depth;
    s->stats.build_seconds = build_s;
    lap(5);
    for (int k = 0; k < 6; ++k) s->stats.phase_seconds[k] = phase[k];
    *out = s;
    return QRT_OK;
}

int qrt_scene_destroy(qrt_scene scene) {
    if (!scene) return fail(QRT_ERR_INVALID_ARG, "scene is NULL");
    free_scene(scene);
    return QRT_OK;
}

int qrt_scene_stats_get(qrt_scene scene, qrt_scene_stats* out) {
    if (!scene || !out) return fail(QRT_ERR_INVALID_ARG, "NULL argument");
    *out = scene->stats;
    return QRT_OK;
}

static int trace_common(bool any, qrt_scene scene, const qrt_ray* d_rays, uint64_t n, void* out,
                        const qrt_tuning* tuning, qrt_stream stream) {
    if (!scene) return fail(QRT_ERR_INVALID_ARG, "scene is NULL");
    if (n == 0) return QRT_OK;
    if (!d_rays || !out) return fail(QRT_ERR_INVALID_ARG, "NULL device pointer");
    if (!aligned(d_rays, 16) || !aligned(out, any ? 4 : 16))
        return fail(QRT_ERR_ALIGN, "rays/hits must be 16-byte aligned (occlusion bits 4-byte)");
    Tune t = resolve_tuning(tuning);
    int rc = validate_tuning(t);
    if (rc) return rc;
    rc = check_device(scene);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_trace(any, scene->S, d_rays, n, any ? nullptr : out,
                                 any ? static_cast<uint32_t*>(out) : nullptr, 1u << 20,
                                 scene->slot_for(s).counter, nullptr, t, scene->sm_count, s);
    if (e != cudaSuccess) return cuda_fail(e, "trace launch");
    return QRT_OK;
}

int qrt_trace_closest(qrt_scene scene, const qrt_ray* d_rays, uint64_t n, qrt_hit* d_hits,
                      const qrt_tuning* tuning, qrt_stream stream) {
    return trace_common(false, scene, d_rays, n, d_hits, tuning, stream);
}

int qrt_trace_any(qrt_scene scene, const qrt_ray* d_rays, uint64_t n, uint32_t* d_occ_bits,
                  const qrt_tuning* tuning, qrt_stream stream) {
    return trace_common(true, scene, d_rays, n, d_occ_bits, tuning, stream);
}

}  // extern "C"

namespace {

// Builds the device view table for views[first, first+count).
int make_views(const qrt_view* views, uint32_t first, uint32_t count, const float* const* d_dimage,
               RenderArgs& A, uint64_t path_begin0) {
    uint64_t items = 0, paths = path_begin0;
    for (uint32_t k = 0; k < count; ++k) {
        const qrt_view& v = views[first + k];
        if (v.w == 0 || v.h == 0 || v.spp == 0) {
            std::snprintf(g_err, sizeof(g_err), "view %u has zero size or spp", first + k);
            return QRT_ERR_INVALID_ARG;
        }
        if (!v.out_rgb && !d_dimage) {
            std::snprintf(g_err, sizeof(g_err), "view %u has no out_rgb", first + k);
            return QRT_ERR_INVALID_ARG;
        }
        if (v.out_rgb && !aligned(v.out_rgb, 4)) return fail(QRT_ERR_ALIGN, "out_rgb must be 4-byte aligned");
        const bool crop = v.crop_w != 0 || v.crop_h != 0;
        if (crop && (v.crop_w == 0 || v.crop_h == 0 || (uint64_t)v.crop_x + v.crop_w > v.w ||
                     (uint64_t)v.crop_y + v.crop_h > v.h)) {
            std::snprintf(g_err, sizeof(g_err),
                          "view %u: crop %ux%u at (%u, %u) is empty or leaves the %ux%u frame",
                          first + k, v.crop_w, v.crop_h, v.crop_x, v.crop_y, v.w, v.h);
            return QRT_ERR_INVALID_ARG;
        }
        double eye[3] = {v.eye[0], v.eye[1], v.eye[2]};
        double f[3] = {v.look[0] - eye[0], v.look[1] - eye[1], v.look[2] - eye[2]};
        double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        if (!(fl > 0.0)) return fail(QRT_ERR_INVALID_ARG, "camera eye equals look");
        for (double& c : f) c /= fl;
        double up[3] = {v.up[0], v.up[1], v.up[2]};
        double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
        double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (!(rl > 0.0)) return fail(QRT_ERR_INVALID_ARG, "camera up is parallel to the view direction");
        for (double& c : r) c /= rl;
        double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
        if (!(v.vfov_deg > 0.f && v.vfov_deg < 180.f))
            return fail(QRT_ERR_INVALID_ARG, "vfov_deg must be in (0, 180)");
        const double th = std::tan(0.5 * (double)v.vfov_deg * 3.14159265358979323846 / 180.0);
        const double aspect = (double)v.w / (double)v.h;
        ViewDev& d = A.views[k];
        for (int c = 0; c < 3; ++c) {
            d.eye[c] = v.eye[c];
            d.f[c] = (float)f[c];
            d.r[c] = (float)r[c];
            d.u[c] = (float)u[c];
        }
        d.sx0 = (float)(-th * aspect);
        d.sxs = (float)(2.0 * th * aspect / v.w);
        d.sy0 = (float)th;
        d.sys = (float)(-2.0 * th / v.h);
        d.w = crop ? v.crop_w : v.w;
        d.h = crop ? v.crop_h : v.h;
        d.x0 = crop ? v.crop_x : 0;
        d.y0 = crop ? v.crop_y : 0;
        d.fw = v.w;
        d.spp = v.spp;
        d.sample_base = v.sample_base;
        d.pixel_base = v.pixel_base;
        d.item_begin = items;
        d.path_begin = paths;
        d.out = v.out_rgb;
        d.cost_out = nullptr;
        d.dimage = d_dimage ? d_dimage[first + k] : nullptr;
        if (d_dimage && !d.dimage) {
            std::snprintf(g_err, sizeof(g_err), "d_dimage[%u] is NULL", first + k);
            return QRT_ERR_INVALID_ARG;
        }
        items += (uint64_t)d.w * d.h;
        paths += (uint64_t)d.w * d.h * v.spp;
    }
    A.n_items = items;
    A.n_views = count;
    return QRT_OK;
}

int make_params(const qrt_params* p, ParamsDev& P) {
    if (!p) return fail(QRT_ERR_INVALID_ARG, "params is NULL");
    if (p->max_depth < 1 || p->max_depth > 256)
        return fail(QRT_ERR_INVALID_ARG, "max_depth must be 1..256");
    P.max_depth = p->max_depth;
    P.max_steps = p->max_steps ? p->max_steps : (1u << 20);
    P.seed = p->seed;
    for (int c = 0; c < 3; ++c) {
        P.env[c] = p->env[c];
        P.sun_E[c] = p->sun_E[c];
    }
    P.sun_on = (p->sun_E[0] != 0.f || p->sun_E[1] != 0.f || p->sun_E[2] != 0.f) ? 1u : 0u;
    const double sl = std::sqrt((double)p->sun_dir[0] * p->sun_dir[0] + (double)p->sun_dir[1] * p->sun_dir[1] +
                                (double)p->sun_dir[2] * p->sun_dir[2]);
    if (P.sun_on && !(sl > 0.0)) return fail(QRT_ERR_INVALID_ARG, "sun_dir is zero");
    for (int c = 0; c < 3; ++c) P.sun_l[c] = sl > 0.0 ? (float)(p->sun_dir[c] / sl) : 0.f;
    P.path_log = p->d_path_log;
    if (P.path_log && !aligned(P.path_log, 4)) return fail(QRT_ERR_ALIGN, "d_path_log must be 4-byte aligned");
    P.ray_log = p->d_ray_log;
    if (P.ray_log && !aligned(P.ray_log, 16)) return fail(QRT_ERR_ALIGN, "d_ray_log must be 16-byte aligned");
    P.tex = p->tex_res ? p->d_tex : nullptr;
    P.tex_res = p->d_tex ? p->tex_res : 0;
    if (P.tex_res > kMaxTexRes) return fail(QRT_ERR_INVALID_ARG, "tex_res exceeds QRT_MAX_TEX_RES");
    if (P.tex && !aligned(P.tex, 4)) return fail(QRT_ERR_ALIGN, "d_tex must be 4-byte aligned");
    if (p->n_lights > (uint32_t)kMaxLights) return fail(QRT_ERR_INVALID_ARG, "n_lights exceeds QRT_MAX_LIGHTS");
    if (p->n_lights && !p->lights) return fail(QRT_ERR_INVALID_ARG, "lights is NULL");
    P.n_lights = p->n_lights;
    for (uint32_t k = 0; k < p->n_lights; ++k)
        for (int c = 0; c < 12; ++c) {
            const float v = p->lights[12 * k + c];
            if (!std::isfinite(v)) return fail(QRT_ERR_INVALID_ARG, "light " + std::to_string(k) + " is not finite");
            P.lights[k][c] = v;
        }
    return QRT_OK;
}

// Ensures sl holds a wavefront workspace of at least `bytes`.  Allocation is
// refused while the stream is being captured.
int ensure_workspace(StreamSlot& sl, size_t bytes, cudaStream_t s) {
    if (sl.ws_bytes >= bytes) return QRT_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone)
        return fail(QRT_ERR_NOT_READY,
                    "wavefront workspace must be allocated before capture: render once on this "
                    "stream outside capture, or use qrt_render_graph_create");
    // the old workspace may still be in use by queued work on this stream
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    cudaFree(sl.ws);
    sl.ws = nullptr;
    sl.ws_bytes = 0;
    e = cudaMalloc(&sl.ws, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "wavefront workspace");
    sl.ws_bytes = bytes;
    return QRT_OK;
}

// Enqueues the wavefront render (or adjoint) of all views on stream s in
// the given workspace; W and R are the caller's storage for the launch
// parameter blocks (so this function allocates nothing).
int wave_enqueue(qrt_scene scene, const qrt_view* views, uint32_t n_views, const float* d_albedo,
                 const float* const* d_dimage, float* d_grad, const qrt_params* params,
                 const Tune& t, void* workspace, size_t ws_bytes, unsigned long long* stats,
                 cudaStream_t s, WaveArgs& W, RenderArgs& R, const WaveStreams* ov,
                 float* const* d_cost = nullptr) {
    static_assert(sizeof(WaveArgs) < 32000, "kernel parameter block too large");
    const bool adjoint = d_grad != nullptr;
    const uint64_t cap = 1ull << t.chunk_log2;
    if (wave_workspace_bytes(cap, adjoint) > ws_bytes)
        return fail(QRT_ERR_INVALID_ARG, "wavefront workspace too small for chunk_log2");
    // a chunk is cut at pixel boundaries, so it must hold all of a pixel's samples
    for (uint32_t v = 0; v < n_views; ++v)
        if ((uint64_t)views[v].spp > cap) {
            std::snprintf(g_err, sizeof(g_err),
                          "view %u: spp %u exceeds the %llu paths of a wavefront chunk "
                          "(tuning.chunk_log2 %d; qrt_render_spp_static allows at most 2^%d)",
                          v, views[v].spp, (unsigned long long)cap, t.chunk_log2, kStaticChunkLog2);
            return QRT_ERR_INVALID_ARG;
        }
    std::memset(&W, 0, sizeof(WaveArgs));
    std::memset(&R, 0, sizeof(RenderArgs));
    W.S = scene->S;
    W.albedo = d_albedo;
    W.grad = d_grad;
    W.stats = stats;
    W.capacity = cap;
    W.batch = (uint32_t)t.batch;
    W.cost_on = d_cost != nullptr;
    wave_carve(workspace, cap, adjoint, W.B);
    int rc = make_params(params, W.P);
    if (adjoint) {
        W.P.path_log = nullptr;
        W.P.ray_log = nullptr;
    }
    // the view table is shared with the single-kernel renderer's layout
    uint64_t paths = 0;
    for (uint32_t first = 0; rc == QRT_OK && first < n_views; first += kMaxViewsPerLaunch) {
        const uint32_t cnt = std::min<uint32_t>(kMaxViewsPerLaunch, n_views - first);
        rc = make_views(views, first, cnt, d_dimage, R, paths);
        if (rc) break;
        for (uint32_t k = 0; k < cnt; ++k) {
            W.views[k] = R.views[k];
            if (d_cost) W.views[k].cost_out = d_cost[first + k];
            paths += region_pixels(views[first + k]) * views[first + k].spp;
        }
        W.n_views = cnt;
        StageHook* hook = (params && (params->flags & QRT_FLAG_STAGE_TIMES)) ? &scene->timer : nullptr;
        // timed stages run in order: overlapping kernels would blur their times
        cudaError_t e = launch_wave(W, t, scene->sm_count, s, hook, hook ? nullptr : ov);
        if (e != cudaSuccess) rc = cuda_fail(e, "wavefront launch");
    }
    return rc;
}

// Enqueues the render (or adjoint) of all views on stream s.  counter serves
// the single-kernel renderer, workspace (bytes) the wavefront one.
int render_enqueue(qrt_scene scene, const qrt_view* views, uint32_t n_views, const float* d_albedo,
                   const float* const* d_dimage, float* d_grad, const qrt_params* params,
                   unsigned long long* counter, void* workspace, size_t ws_bytes,
                   unsigned long long* stats, cudaStream_t s, const WaveStreams* ov,
                   float* const* d_cost = nullptr) {
    Tune t = resolve_tuning(params ? &params->tuning : nullptr);
    fit_chunk(t, views, n_views);
    int rc = validate_tuning(t);
    if (rc) return rc;
    const bool adjoint = d_grad != nullptr;
    if (t.mode == 1) {
        static_assert(sizeof(RenderArgs) < 32000, "kernel parameter block too large");
        RenderArgs* A = new RenderArgs();
        std::memset(A, 0, sizeof(RenderArgs));
        A->S = scene->S;
        A->albedo = d_albedo;
        A->grad = d_grad;
        A->counter = counter;
        A->stats = stats;
        A->batch = (uint32_t)t.batch;
        rc = make_params(params, A->P);
        if (adjoint) {
            A->P.path_log = nullptr;
            A->P.ray_log = nullptr;
        }
        uint64_t paths = 0;
        for (uint32_t first = 0; rc == QRT_OK && first < n_views; first += kMaxViewsPerLaunch) {
            const uint32_t cnt = std::min<uint32_t>(kMaxViewsPerLaunch, n_views - first);
            rc = make_views(views, first, cnt, d_dimage, *A, paths);
            if (rc) break;
            for (uint32_t k = 0; k < cnt; ++k)
                paths += region_pixels(views[first + k]) * views[first + k].spp;
            cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
            if (e == cudaSuccess) e = launch_render(*A, t, scene->sm_count, s);
            if (e != cudaSuccess) rc = cuda_fail(e, "render launch");
        }
        delete A;
        return rc;
    }
    WaveArgs* W = new WaveArgs();
    RenderArgs* R = new RenderArgs();
    rc = wave_enqueue(scene, views, n_views, d_albedo, d_dimage, d_grad, params, t, workspace,
                      ws_bytes, stats, s, *W, *R, ov, d_cost);
    delete R;
    delete W;
    return rc;
}

// Scratch for a plain (non-graph) call on stream s.
int stream_scratch(qrt_scene scene, const qrt_params* params, const qrt_view* views,
                   uint32_t n_views, bool adjoint, cudaStream_t s, unsigned long long** counter,
                   void** ws, size_t* ws_bytes, const WaveStreams** ov) {
    StreamSlot& sl = scene->slot_for(s);
    *counter = sl.counter;
    *ov = nullptr;
    Tune t = resolve_tuning(params ? &params->tuning : nullptr);
    fit_chunk(t, views, n_views);
    int rc = validate_tuning(t);
    if (rc) return rc;
    if (t.mode == 2) {
        // one workspace per stream, sized for the adjoint so both fit
        rc = ensure_workspace(sl, wave_workspace_bytes(1ull << t.chunk_log2, true), s);
        if (rc) return rc;
        // the second stream is made outside capture; a capture started
        // before the first render on this stream runs the stages in order
        if (!sl.ov.aux) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
                cudaError_t e = create_streams(sl.ov);
                if (e != cudaSuccess) return cuda_fail(e, "overlap stream");
            }
        }
        if (sl.ov.aux) *ov = &sl.ov;
    }
    (void)adjoint;
    *ws = sl.ws;
    *ws_bytes = sl.ws_bytes;
    return QRT_OK;
}

int render_args_check(qrt_scene scene, const qrt_view* views, uint32_t n_views, const float* d_albedo) {
    if (!scene) return fail(QRT_ERR_INVALID_ARG, "scene is NULL");
    if (n_views > 0 && !views) return fail(QRT_ERR_INVALID_ARG, "views is NULL");
    if (n_views > 0 && !d_albedo) return fail(QRT_ERR_INVALID_ARG, "d_albedo is NULL");
    if (d_albedo && !aligned(d_albedo, 4)) return fail(QRT_ERR_ALIGN, "d_albedo must be 4-byte aligned");
    return check_device(scene);
}

}  // namespace

extern "C" {

int qrt_render_spp(qrt_scene scene, const qrt_view* views, uint32_t n_views, const float* d_albedo,
                   const qrt_params* params, qrt_stream stream) {
    int rc = render_args_check(scene, views, n_views, d_albedo);
    if (rc) return rc;
    if (n_views == 0) return QRT_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* ctr;
    void* ws;
    size_t wsb;
    const WaveStreams* ov = nullptr;
    rc = stream_scratch(scene, params, views, n_views, false, s, &ctr, &ws, &wsb, &ov);
    if (rc) return rc;
    return render_enqueue(scene, views, n_views, d_albedo, nullptr, nullptr, params, ctr, ws, wsb,
                          nullptr, s, ov);
}

// qrt_render_spp without any allocation: the wavefront renderer with its
// workspace in a fixed device array of the library (see qrt.h).
int qrt_render_spp_static(qrt_scene scene, const qrt_view* views, uint32_t n_views,
                          const float* d_albedo, const qrt_params* params, qrt_stream stream) {
    int rc = render_args_check(scene, views, n_views, d_albedo);
    if (rc) return rc;
    if (!params) return fail(QRT_ERR_INVALID_ARG, "params is NULL");
    if (n_views == 0) return QRT_OK;
    qrt_tuning tt = params->tuning;
    if (tt.mode == 1)
        return fail(QRT_ERR_INVALID_ARG,
                    "qrt_render_spp_static runs the wavefront renderer only (tuning.mode 0 or 2)");
    if (tt.chunk_log2 == 0) tt.chunk_log2 = kStaticChunkLog2;
    if (tt.chunk_log2 > (uint32_t)kStaticChunkLog2)
        return fail(QRT_ERR_INVALID_ARG,
                    "tuning.chunk_log2 exceeds the static workspace (at most 17: 131072 paths "
                    "per chunk)");
    Tune t = resolve_tuning(&tt);
    rc = validate_tuning(t);
    if (rc) return rc;
    void* ws = nullptr;
    cudaError_t e = static_workspace(&ws);
    if (e != cudaSuccess) return cuda_fail(e, "static workspace address");
    WaveArgs W;  // parameter blocks on the stack: nothing is allocated
    RenderArgs R;
    return wave_enqueue(scene, views, n_views, d_albedo, nullptr, nullptr, params, t, ws,
                        kStaticWorkspaceBytes, nullptr, reinterpret_cast<cudaStream_t>(stream), W, R,
                        nullptr);
}

// Same as qrt_render_spp with traversal counters added into d_stats (device
// uint64[5]: rays, inner nodes, quads tested, instances entered, FP64
// re-tests).  Used to compute the algorithmic bytes of a render.
int qrt_render_spp_stats(qrt_scene scene, const qrt_view* views, uint32_t n_views,
                         const float* d_albedo, const qrt_params* params,
                         unsigned long long* d_stats, qrt_stream stream) {
    int rc = render_args_check(scene, views, n_views, d_albedo);
    if (rc) return rc;
    if (!d_stats || !aligned(d_stats, 8)) return fail(QRT_ERR_INVALID_ARG, "d_stats NULL or unaligned");
    if (n_views == 0) return QRT_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* ctr;
    void* ws;
    size_t wsb;
    const WaveStreams* ov = nullptr;
    rc = stream_scratch(scene, params, views, n_views, false, s, &ctr, &ws, &wsb, &ov);
    if (rc) return rc;
    return render_enqueue(scene, views, n_views, d_albedo, nullptr, nullptr, params, ctr, ws, wsb,
                          d_stats, s, ov);
}

int qrt_render_cost(qrt_scene scene, const qrt_view* views, uint32_t n_views, const float* d_albedo,
                    const qrt_params* params, float* const* d_cost, unsigned long long* d_stats,
                    qrt_stream stream) {
    int rc = render_args_check(scene, views, n_views, d_albedo);
    if (rc) return rc;
    if (!d_stats || !aligned(d_stats, 8)) return fail(QRT_ERR_INVALID_ARG, "d_stats NULL or unaligned");
    if (n_views == 0) return QRT_OK;
    if (!d_cost) return fail(QRT_ERR_INVALID_ARG, "d_cost is NULL");
    for (uint32_t v = 0; v < n_views; ++v)
        if (!d_cost[v] || !aligned(d_cost[v], 4)) {
            std::snprintf(g_err, sizeof(g_err), "d_cost[%u] is NULL or unaligned", v);
            return QRT_ERR_INVALID_ARG;
        }
    if (params && params->tuning.mode == 1)
        return fail(QRT_ERR_INVALID_ARG, "cost maps come from the wavefront renderer (tuning.mode 0 or 2)");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* ctr;
    void* ws;
    size_t wsb;
    const WaveStreams* ov = nullptr;
    rc = stream_scratch(scene, params, views, n_views, false, s, &ctr, &ws, &wsb, &ov);
    if (rc) return rc;
    return render_enqueue(scene, views, n_views, d_albedo, nullptr, nullptr, params, ctr, ws, wsb,
                          d_stats, s, ov, d_cost);
}

int qrt_trace_stats(qrt_scene scene, int any, const qrt_ray* d_rays, uint64_t n, void* d_out,
                    const qrt_tuning* tuning, unsigned long long* d_stats, qrt_stream stream) {
    if (!scene) return fail(QRT_ERR_INVALID_ARG, "scene is NULL");
    if (n == 0) return QRT_OK;
    if (!d_rays || !d_out || !d_stats) return fail(QRT_ERR_INVALID_ARG, "NULL device pointer");
    if (!aligned(d_rays, 16) || !aligned(d_out, any ? 4 : 16) || !aligned(d_stats, 8))
        return fail(QRT_ERR_ALIGN, "misaligned device pointer");
    Tune t = resolve_tuning(tuning);
    int rc = validate_tuning(t);
    if (rc) return rc;
    rc = check_device(scene);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_trace(any != 0, scene->S, d_rays, n, any ? nullptr : d_out,
                                 any ? static_cast<uint32_t*>(d_out) : nullptr, 1u << 20,
                                 scene->slot_for(s).counter, d_stats, t, scene->sm_count, s);
    if (e != cudaSuccess) return cuda_fail(e, "trace launch");
    return QRT_OK;
}

int qrt_render_adjoint(qrt_scene scene, const qrt_view* views, uint32_t n_views,
                       const float* d_albedo, const float* const* d_dimage, float* d_grad_albedo,
                       const qrt_params* params, qrt_stream stream) {
    int rc = render_args_check(scene, views, n_views, d_albedo);
    if (rc) return rc;
    if (n_views == 0) return QRT_OK;
    if (!d_dimage) return fail(QRT_ERR_INVALID_ARG, "d_dimage is NULL");
    if (!d_grad_albedo || !aligned(d_grad_albedo, 4))
        return fail(QRT_ERR_INVALID_ARG, "d_grad_albedo is NULL or unaligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* ctr;
    void* ws;
    size_t wsb;
    const WaveStreams* ov = nullptr;
    rc = stream_scratch(scene, params, views, n_views, true, s, &ctr, &ws, &wsb, &ov);
    if (rc) return rc;
    return render_enqueue(scene, views, n_views, d_albedo, d_dimage, d_grad_albedo, params, ctr, ws,
                          wsb, nullptr, s, ov);
}

int qrt_accumulate(float* d_sum, const float* d_frame, float* d_mean, uint64_t n, uint32_t frames,
                   qrt_stream stream) {
    if (n == 0) return QRT_OK;
    if (!d_sum || !d_frame) return fail(QRT_ERR_INVALID_ARG, "NULL image pointer");
    if (frames == 0) return fail(QRT_ERR_INVALID_ARG, "frames must be at least 1");
    if (!aligned(d_sum, 4) || !aligned(d_frame, 4) || (d_mean && !aligned(d_mean, 4)))
        return fail(QRT_ERR_ALIGN, "image pointers must be 4-byte aligned");
    cudaError_t e = launch_accumulate(d_sum, d_frame, d_mean, n, frames,
                                      reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "accumulate launch");
    return QRT_OK;
}

int qrt_l2_loss(const float* d_img, const float* d_target, uint64_t n, double* d_loss,
                float* d_dimage, qrt_stream stream) {
    if (!d_loss) return fail(QRT_ERR_INVALID_ARG, "d_loss is NULL");
    if (n > 0 && (!d_img || !d_target)) return fail(QRT_ERR_INVALID_ARG, "NULL image pointer");
    if (!aligned(d_loss, 8)) return fail(QRT_ERR_ALIGN, "d_loss must be 8-byte aligned");
    cudaError_t e = launch_l2_loss(d_img, d_target, n, d_loss, d_dimage,
                                   reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "loss launch");
    return QRT_OK;
}

int qrt_read_bandwidth(const void* d_buf, uint64_t bytes, uint32_t reps, uint32_t* d_sink,
                       qrt_stream stream) {
    if (bytes == 0 || reps == 0) return QRT_OK;
    if (!d_buf || !d_sink) return fail(QRT_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned(d_buf, 16) || bytes % 16 != 0)
        return fail(QRT_ERR_ALIGN, "d_buf must be 16-byte aligned and bytes a multiple of 16");
    if (!aligned(d_sink, 4)) return fail(QRT_ERR_ALIGN, "d_sink must be 4-byte aligned");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = launch_read_sweep(d_buf, bytes, reps, d_sink, sms, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "read sweep launch");
    return QRT_OK;
}

int qrt_render_graph_create(qrt_scene scene, const qrt_view* views, uint32_t n_views,
                            const float* d_albedo, const qrt_params* params, qrt_graph* out) {
    if (!out) return fail(QRT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int rc = render_args_check(scene, views, n_views, d_albedo);
    if (rc) return rc;
    if (n_views == 0) return fail(QRT_ERR_INVALID_ARG, "no views");
    Tune tg = resolve_tuning(params ? &params->tuning : nullptr);
    fit_chunk(tg, views, n_views);
    rc = validate_tuning(tg);
    if (rc) return rc;
    qrt_graph_s* g = new qrt_graph_s();
    g->device = scene->device;
    const size_t wsb = tg.mode == 2 ? wave_workspace_bytes(1ull << tg.chunk_log2, false) : 0;
    cudaError_t e = cudaMalloc((void**)&g->d_counter, kSlotStride);
    if (e == cudaSuccess && wsb) e = cudaMalloc(&g->ws, wsb);
    if (e != cudaSuccess) {
        cudaFree(g->d_counter);
        cudaFree(g->ws);
        delete g;
        return cuda_fail(e, "graph scratch");
    }
    cudaStream_t cs = nullptr;
    WaveStreams ov;  // joins the capture through its fork event, so the graph keeps the overlap
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess && tg.mode == 2) e = create_streams(ov);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        destroy_streams(ov);
        if (cs) cudaStreamDestroy(cs);
        cudaFree(g->d_counter);
        cudaFree(g->ws);
        delete g;
        return cuda_fail(e, "graph capture");
    }
    rc = render_enqueue(scene, views, n_views, d_albedo, nullptr, nullptr, params, g->d_counter,
                        g->ws, wsb, nullptr, cs, ov.aux ? &ov : nullptr);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    destroy_streams(ov);
    if (rc == QRT_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "graph capture");
    if (rc == QRT_OK) {
        g->graph = graph;
        e = cudaGraphInstantiate(&g->exec, graph, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "graph instantiate");
    } else if (graph) {
        cudaGraphDestroy(graph);
    }
    if (rc != QRT_OK) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        cudaFree(g->d_counter);
        cudaFree(g->ws);
        delete g;
        return rc;
    }
    *out = g;
    return QRT_OK;
}

int qrt_graph_launch(qrt_graph graph, qrt_stream stream) {
    if (!graph) return fail(QRT_ERR_INVALID_ARG, "graph is NULL");
    cudaError_t e = cudaGraphLaunch(graph->exec, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    return QRT_OK;
}

int qrt_graph_destroy(qrt_graph graph) {
    if (!graph) return fail(QRT_ERR_INVALID_ARG, "graph is NULL");
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    cudaFree(graph->d_counter);
    cudaFree(graph->ws);
    delete graph;
    return QRT_OK;
}

int qrt_stage_times(qrt_scene scene, qrt_stream stream, double* ms, uint32_t* launches, int reset) {
    if (!scene || !ms || !launches) return fail(QRT_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    scene->timer.read(ms, launches, reset != 0);
    return QRT_OK;
}

int qrt_check(qrt_scene scene, qrt_stream stream) {
    if (!scene) return fail(QRT_ERR_INVALID_ARG, "scene is NULL");
    int rc = check_device(scene);
    if (rc) return rc;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    uint32_t w[2];
    e = cudaMemcpy(w, scene->d_err, sizeof(w), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "error word read");
    if (w[0] == 0) return QRT_OK;
    const uint32_t init[2] = {0u, 0xFFFFFFFFu};
    e = cudaMemcpy(scene->d_err, init, sizeof(init), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "error word reset");
    if (w[0] & kErrStackOverflow)
        return fail(QRT_ERR_STACK_OVERFLOW,
                    "traversal stack overflow (first affected item " + std::to_string(w[1]) + ")");
    return fail(QRT_ERR_STEP_LIMIT,
                "traversal step limit exceeded (first affected item " + std::to_string(w[1]) + ")");
}

int qrt_tlas_build_check(const float* boxes, uint64_t n, const qrt_build_opts* opts,
                         uint64_t* n_nodes, uint32_t* depth) {
    if (!boxes && n) return fail(QRT_ERR_INVALID_ARG, "boxes is NULL");
    if (opts && opts->tlas_builder > 2) return fail(QRT_ERR_INVALID_ARG, "build_opts.tlas_builder must be 0..2");
    std::vector<FBox> items(n);
    for (uint64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            items[i].lo[a] = boxes[6 * i + a];
            items[i].hi[a] = boxes[6 * i + 3 + a];
        }
    TlasResult t;
    std::string err;
    if (!make_tlas(items, resolve_build(opts), t, err)) {
        const bool cuda = err.compare(0, 5, "CUDA:") == 0;
        return fail(cuda ? QRT_ERR_CUDA : QRT_ERR_INVALID_ARG, err);
    }
    uint32_t d = 0;
    if (!t.nodes.empty() && !check_wide(t.nodes, items, err, &d)) return fail(QRT_ERR_INVALID_ARG, err);
    if (n_nodes) *n_nodes = t.nodes.size();
    if (depth) *depth = d;
    return QRT_OK;
}

// Invariants of one built BLAS: every original quad in exactly one slot,
// and the four-wide tree checked against the quads' exact boxes.
static bool check_blas(const BlasResult& r, uint32_t n_quads, std::string& err, uint32_t* depth) {
    std::vector<FBox> items(r.quads.size());
    for (size_t s = 0; s < r.quads.size(); ++s) {
        FBox b;
        for (int a = 0; a < 3; ++a) {
            b.lo[a] = std::min(std::min(r.quads[s].v[a], r.quads[s].v[3 + a]),
                               std::min(r.quads[s].v[6 + a], r.quads[s].v[9 + a]));
            b.hi[a] = std::max(std::max(r.quads[s].v[a], r.quads[s].v[3 + a]),
                               std::max(r.quads[s].v[6 + a], r.quads[s].v[9 + a]));
        }
        items[s] = b;
    }
    std::vector<uint8_t> seen(n_quads, 0);
    if (r.prim.size() != n_quads) {
        err = "slot permutation broken";
        return false;
    }
    for (uint32_t p : r.prim)
        if (p >= n_quads || seen[p]++) {
            err = "slot permutation broken";
            return false;
        }
    return check_wide(r.nodes, items, err, depth);
}

int qrt_blases_build_check(const qrt_mesh* meshes, uint32_t n_mesh, const qrt_build_opts* opts,
                           uint64_t* n_nodes, uint32_t* max_depth) {
    if (!meshes || n_mesh == 0) return fail(QRT_ERR_INVALID_ARG, "meshes is NULL or empty");
    const BuildOpts bo = resolve_build(opts);
    if (bo.blas_builder > 2) return fail(QRT_ERR_INVALID_ARG, "build_opts.blas_builder must be 0..2");
    std::vector<BlasResult> out(n_mesh);
    std::string err;
    if (bo.blas_builder) {
        std::vector<MeshView> mv(n_mesh);
        for (uint32_t m = 0; m < n_mesh; ++m) {
            if (!meshes[m].verts || !meshes[m].quads) return fail(QRT_ERR_INVALID_ARG, "mesh arrays are NULL");
            mv[m] = MeshView{meshes[m].verts, meshes[m].n_verts, meshes[m].quads, meshes[m].n_quads};
        }
        if (!build_blases_lbvh(mv, std::max(1u, std::min(bo.max_leaf, 8u)), bo.blas_builder == 1, out, err))
            return fail(err.compare(0, 5, "CUDA:") == 0 ? QRT_ERR_CUDA : QRT_ERR_INVALID_ARG, err);
    } else {
        for (uint32_t m = 0; m < n_mesh; ++m)
            if (!meshes[m].verts || !meshes[m].quads ||
                !build_blas(meshes[m].verts, meshes[m].n_verts, meshes[m].quads, meshes[m].n_quads, bo,
                            out[m], err))
                return fail(QRT_ERR_INVALID_ARG, "mesh " + std::to_string(m) + ": " + err);
    }
    uint64_t total = 0;
    uint32_t dmax = 0;
    for (uint32_t m = 0; m < n_mesh; ++m) {
        uint32_t d = 0;
        if (!check_blas(out[m], meshes[m].n_quads, err, &d))
            return fail(QRT_ERR_INVALID_ARG, "mesh " + std::to_string(m) + ": " + err);
        total += out[m].nodes.size();
        dmax = std::max(dmax, d);
    }
    if (n_nodes) *n_nodes = total;
    if (max_depth) *max_depth = dmax;
    return QRT_OK;
}

int qrt_blas_build_check(const qrt_mesh* mesh, const qrt_build_opts* opts, uint64_t* n_nodes,
                         uint32_t* depth) {
    if (!mesh || !mesh->verts || !mesh->quads)
        return fail(QRT_ERR_INVALID_ARG, "mesh or its arrays are NULL");
    BlasResult r;
    std::string err;
    const BuildOpts bo = resolve_build(opts);
    if (bo.blas_builder > 2) return fail(QRT_ERR_INVALID_ARG, "build_opts.blas_builder must be 0..2");
    if (bo.blas_builder) {
        std::vector<BlasResult> out;
        const std::vector<MeshView> mv{MeshView{mesh->verts, mesh->n_verts, mesh->quads, mesh->n_quads}};
        if (!build_blases_lbvh(mv, std::max(1u, std::min(bo.max_leaf, 8u)), bo.blas_builder == 1, out, err))
            return fail(err.compare(0, 5, "CUDA:") == 0 ? QRT_ERR_CUDA : QRT_ERR_INVALID_ARG, err);
        r = std::move(out[0]);
    } else if (!build_blas(mesh->verts, mesh->n_verts, mesh->quads, mesh->n_quads, bo, r, err)) {
        return fail(QRT_ERR_INVALID_ARG, err);
    }
    std::vector<FBox> items(r.quads.size());
    for (size_t s = 0; s < r.quads.size(); ++s) {
        FBox b;
        for (int a = 0; a < 3; ++a) {
            b.lo[a] = std::min(std::min(r.quads[s].v[a], r.quads[s].v[3 + a]),
                               std::min(r.quads[s].v[6 + a], r.quads[s].v[9 + a]));
            b.hi[a] = std::max(std::max(r.quads[s].v[a], r.quads[s].v[3 + a]),
                               std::max(r.quads[s].v[6 + a], r.quads[s].v[9 + a]));
        }
        items[s] = b;
    }
    // every original quad appears once in slot order
    std::vector<uint8_t> seen(mesh->n_quads, 0);
    for (uint32_t p : r.prim) {
        if (p >= mesh->n_quads || seen[p]++) return fail(QRT_ERR_INVALID_ARG, "slot permutation broken");
    }
    uint32_t d = 0;
    if (!check_wide(r.nodes, items, err, &d)) return fail(QRT_ERR_INVALID_ARG, err);
    if (n_nodes) *n_nodes = r.nodes.size();
    if (depth) *depth = d;
    return QRT_OK;
}

int qrt_test_sort_pairs(const uint64_t* keys, const uint32_t* vals, uint64_t n, uint32_t end_bit,
                        uint64_t* keys_out, uint32_t* vals_out) {
    if (n && (!keys || !vals || !keys_out || !vals_out)) return fail(QRT_ERR_INVALID_ARG, "NULL array");
    if (n > 0xFFFFFFFFull - 2048) return fail(QRT_ERR_INVALID_ARG, "n above 2^32 - 2049");
    if (end_bit > 64) return fail(QRT_ERR_INVALID_ARG, "end_bit above 64");
    if (n == 0) return QRT_OK;
    const size_t sizes[5] = {(size_t)n * 8, (size_t)n * 4, (size_t)n * 8, (size_t)n * 4,
                             sort_pairs_scratch_bytes((uint32_t)n)};
    void* bufs[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 5 && e == cudaSuccess; ++b) e = cudaMalloc(&bufs[b], sizes[b]);
    if (e == cudaSuccess) e = cudaMemcpy(bufs[0], keys, sizes[0], cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bufs[1], vals, sizes[1], cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = sort_pairs(static_cast<uint64_t*>(bufs[0]), static_cast<uint32_t*>(bufs[1]),
                       static_cast<uint64_t*>(bufs[2]), static_cast<uint32_t*>(bufs[3]), (uint32_t)n,
                       (int)end_bit, bufs[4], 0);
    if (e == cudaSuccess) e = cudaMemcpy(keys_out, bufs[2], sizes[0], cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(vals_out, bufs[3], sizes[1], cudaMemcpyDeviceToHost);
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (e != cudaSuccess) return fail(QRT_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    return QRT_OK;
}

}  // extern "C"

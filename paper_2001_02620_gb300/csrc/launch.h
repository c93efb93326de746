// Host-side launch interface between the C ABI (capi.cpp) and the CUDA
// translation units (trace.cu, render.cu).  Plain C++ types only.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <stdint.h>

#include "qrt_layout.h"

namespace qrt {

// Resident blocks per SM of one kernel at a given block size (no dynamic
// shared memory), queried once per device and block size and then reused:
// the query costs more host time than launching a trace kernel on a short
// queue, and the persistent kernels size their grid from it on every launch.
// Each kernel variant owns one (a static in its launcher).
struct ResidentBlocks {
    std::atomic<int> cached[16][5];  // [device][block / 64], 0 = not queried yet

    template <class Kernel>
    int get(Kernel kernel, int block) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16 || block % 64 != 0 ||
            block / 64 > 4)
            return query(kernel, block);
        std::atomic<int>& c = cached[dev][block / 64];
        int n = c.load(std::memory_order_relaxed);
        if (n == 0) {
            n = query(kernel, block);
            c.store(n, std::memory_order_relaxed);
        }
        return n;
    }

    template <class Kernel>
    static int query(Kernel kernel, int block) {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, 0);
        return n < 1 ? 1 : n;
    }
};

// Register budget per thread that lets `warps` warps reside on one SM
// (65,536 registers per SM, allocated in multiples of 8 per thread).
constexpr int occupancy_regs(int warps) { return (65536 / (32 * warps)) & ~7; }

// Resolved launch configuration.
struct Tune {
    int block = 256;
    int blocks_per_sm = 0;  // 0 = occupancy maximum
    int batch = 1;          // single kernel: 32-pixel groups a warp claims; trace kernels: rays a lane claims
    int stack = 64;         // 32 or 64
    int fetch = 32;         // node fetch bytes per load: 16 or 32
    int occupancy = 40;     // trace kernels: target resident warps per SM (16, 24, 32, 40 or 48)
    int mode = 2;           // 1 = single persistent kernel, 2 = wavefront
    int chunk_log2 = 0;     // wavefront paths per chunk = 2^chunk_log2; 0 = fit the call
};

// A view with its camera basis precomputed on the host (FP64 -> FP32).
// w x h is the rendered region (the whole frame, or a crop of it at (x0, y0));
// the camera and the random streams are those of the whole frame, whose
// width is fw: region pixel k is frame pixel (x0 + k % w, y0 + k / w) with
// global index pixel_base + y * fw + x.
struct ViewDev {
    float eye[3];
    float f[3], r[3], u[3];
    float sx0, sxs, sy0, sys;  // sx = sx0 + px*sxs, sy = sy0 + py*sys
    uint32_t w, h, spp, sample_base;
    uint32_t x0, y0, fw;
    uint64_t pixel_base;
    uint64_t item_begin;  // first work item (pixel) of this view in the launch
    uint64_t path_begin;  // first path index of this view (for the path log)
    float* out;           // float [h*w*3]
    float* cost_out;      // cost map float [h*w] (mean inner nodes visited per sample) or null
    const float* dimage;  // adjoint input, float [h*w*3]
};

constexpr int kMaxViewsPerLaunch = 64;
constexpr int kMaxLights = 32;
constexpr uint32_t kMaxTexRes = 16;

struct ParamsDev {
    uint32_t max_depth;
    uint32_t max_steps;
    uint64_t seed;
    float env[3];
    float sun_l[3];  // unit vector toward the sun
    float sun_E[3];
    uint32_t sun_on;
    uint32_t* path_log;
    float* ray_log;     // diagnostics: kRayLogFloats per path and depth (see qrt_params)
    const float* tex;   // per-face textures, tex_res^2 RGB texels per quad (or null)
    uint32_t tex_res;
    uint32_t n_lights;  // key lights: corner, edge1, edge2, radiance
    float lights[kMaxLights][12];
};

// Floats per path and depth in the ray log: closest-hit ray (8), spawn
// point (3) and one unused, key-light shadow direction and distance (4).
constexpr int kRayLogFloats = 16;
// Words per path in the path log: (inst, prim) per depth, sun shadow bits,
// key-light shadow bits.
__host__ __device__ constexpr uint64_t path_log_words(uint32_t max_depth) { return 2ull * max_depth + 2; }
// Random stream (fourth Philox counter word) of the key-light sample drawn
// at a path's vertex of depth i: kLightStream + i.
constexpr uint32_t kLightStream = 0x40000000u;

struct RenderArgs {
    DevScene S;
    const float* albedo;
    float* grad;
    ParamsDev P;
    unsigned long long* counter;
    unsigned long long* stats;  // optional: [rays, nodes, quads, instances, fp64 re-tests, vertices]
    uint64_t n_items;
    uint32_t n_views;
    uint32_t batch;
    ViewDev views[kMaxViewsPerLaunch];
};

// Persistent ray-query launch; cursor is a device counter the launch resets.
cudaError_t launch_trace(bool any, const DevScene& S, const void* rays, uint64_t n, void* hits,
                         uint32_t* occ_bits, uint32_t max_steps, unsigned long long* cursor,
                         unsigned long long* stats, const Tune& t, int sm_count, cudaStream_t s);

constexpr int kStatsWords = 6;

// Persistent render (grad == nullptr) or adjoint (grad != nullptr) launch;
// A.counter must be zero when the kernel starts.
cudaError_t launch_render(const RenderArgs& A, const Tune& t, int sm_count, cudaStream_t s);

cudaError_t launch_read_sweep(const void* buf, uint64_t bytes, uint32_t reps, uint32_t* sink,
                              int sm_count, cudaStream_t s);
cudaError_t launch_accumulate(float* sum, const float* frame, float* mean, uint64_t n,
                              uint32_t frames, cudaStream_t s);
cudaError_t launch_l2_loss(const float* img, const float* target, uint64_t n, double* loss,
                           float* dimage, cudaStream_t s);

// Maximum resident blocks per SM for the render kernel variant.
int render_occupancy(const Tune& t, bool adjoint);

}  // namespace qrt

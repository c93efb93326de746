// Wavefront renderer interface (wavefront.cu): per-path state in a
// workspace of `capacity` paths, carved by wave_carve().
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"
#include "qrt_layout.h"

namespace qrt {

// Counter block per depth: queue lengths and the trace kernels' fetch cursors.
constexpr int kCtrStride = 8;
constexpr int kCtrClosest = 0;      // closest-ray queue length of this depth
constexpr int kCtrShadow = 1;       // shadow-ray queue length of this depth
constexpr int kCtrFetchClosest = 2;
constexpr int kCtrFetchShadow = 3;

// Depths whose sun shadow-ray visibility the primal pass of the adjoint
// records (one bit each), so that the replay need not trace those shadow
// rays (key-light shadow rays are traced again).
constexpr int kVisDepths = 32;
// Shadow-queue entries of key-light shadow rays carry this bit.
constexpr uint32_t kLightRay = 0x80000000u;

struct WaveBufs {
    float4* ray_o;   // origin.xyz, tmin (0: path rays span (0, inf))
    float4* ray_d;   // direction.xyz, tmax (inf)
    float4* beta;    // throughput
    float4* L;       // radiance (primal) / sun terms so far (replay); w: bits
                     // of the path's unoccluded shadow rays, depths 1..32
    float4* pend;    // sun term waiting for its shadow ray
    float4* sray_o;  // shadow-ray origin
    float4* lray_d;  // key-light shadow ray: direction, distance
    float4* lpend;   // key-light term waiting for its shadow ray
    uint4* hit;      // t bits, instance, quad, slot
    float2* hit_uv;  // quad-space (u, v) of the hit (per-face textures)
    uint2* meta;     // (pixel item, sample)
    uint32_t* q[2];  // closest-ray queues, ping-pong by depth parity
    uint32_t* qs;    // shadow-ray queue
    uint32_t* cost;  // cost maps: inner BVH nodes visited by each path's rays
    float4* Ltot;    // adjoint: radiance of the first pass
    uint32_t* ctr;   // kCtrStride words per depth 0..max_depth+1
};

// Host-side hook around each stage launch (stage timers); may be null.
enum Stage { kStageGen = 0, kStageTrace = 1, kStageShade = 2, kStageShadow = 3, kStageAccum = 4,
             kStages = 5 };
// A second stream and two events that let the shadow rays of depth i run
// beside the closest-hit rays of depth i + 1 (both read what shade(i)
// wrote and write disjoint buffers), so each persistent launch's draining
// tail is filled by the other.  aux == nullptr runs the stages in order on
// one stream.  Results do not depend on it.
struct WaveStreams {
    cudaStream_t aux = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

struct StageHook {
    virtual void begin(int stage, cudaStream_t s) = 0;
    virtual void end(int stage, cudaStream_t s) = 0;
    virtual ~StageHook() {}
};

struct WaveArgs {
    DevScene S;
    const float* albedo;
    float* grad;
    ParamsDev P;
    WaveBufs B;
    unsigned long long* stats;
    uint64_t P0;        // first path of the current chunk
    uint64_t capacity;  // paths per chunk
    uint32_t n_views;
    uint32_t batch;     // rays a lane claims per fetch
    uint32_t cost_on;   // record per-path traversal cost (counting launches only)
    ViewDev views[kMaxViewsPerLaunch];
};

// Bytes wave_carve() takes for `capacity` paths (each piece 256-B aligned).
constexpr size_t wave_workspace_bytes(uint64_t capacity, bool adjoint) {
    return 9 * (((16 * capacity) + 255) & ~uint64_t(255)) + 2 * (((8 * capacity) + 255) & ~uint64_t(255)) +
           4 * (((4 * capacity) + 255) & ~uint64_t(255)) +
           ((sizeof(uint32_t) * kCtrStride * 258 + 255) & ~uint64_t(255)) +
           (adjoint ? (((16 * capacity) + 255) & ~uint64_t(255)) : 0);
}

// Fixed device scratch for renders that must not allocate: a primal
// workspace of 2^kStaticChunkLog2 paths in a file-scope __device__ array.
constexpr int kStaticChunkLog2 = 17;
constexpr size_t kStaticWorkspaceBytes = wave_workspace_bytes(1ull << kStaticChunkLog2, false);

// Device address of that array on the current device (looked up once per
// device with cudaGetSymbolAddress; allocates nothing).
cudaError_t static_workspace(void** ptr);
void wave_carve(void* base, uint64_t capacity, bool adjoint, WaveBufs& B);
cudaError_t launch_wave(WaveArgs& A, const Tune& t, int sm_count, cudaStream_t s, StageHook* hook,
                        const WaveStreams* ov);

}  // namespace qrt

// Device data layout of a qrt scene in HBM, shared by the host builder
// (bvh_build.cpp) and the CUDA kernels.
//
//   nodes   QNode[ sum of BLAS nodes | TLAS nodes ]   64 B each, 64-B aligned
//   quads   QuadDev[ all meshes, leaf order ]          48 B each (4 x float3)
//   prim    uint32[ same slots ]: original quad index within its mesh
//   inst    InstDev[ n_inst ]                          64 B each
//   inst64  InstDev64[ n_inst ]: FP64 transform for the exact re-test, 80 B
//
// All indices are 32-bit offsets from 64-bit bases.  Stack references are
// local to the current level (TLAS or one BLAS), so every object may hold up
// to 2^27 nodes and 2^27 quads.
#pragma once
#include <stdint.h>

namespace qrt {

// Four-wide node with conservatively quantised child boxes.
// Child i spans [o + qlo*2^e, o + qhi*2^e] per axis, rounded outward so that
// the dequantised box always contains the exact child box.
struct alignas(64) QNode {
    float ox, oy, oz;      // quantisation origin
    int8_t ex, ey, ez;     // per-axis scale exponents
    uint8_t nchild;        // number of valid children
    uint8_t qlo[3][4];     // [axis][child]
    uint8_t qhi[3][4];     // [axis][child]
    uint32_t child[4];     // internal: local node index; leaf: first local quad slot / instance
    uint8_t meta[4];       // 0 = empty, kMetaInner = inner node, 1..16 = leaf item count
    uint32_t pad;
};
static_assert(sizeof(QNode) == 64, "QNode must be 64 bytes");

constexpr uint8_t kMetaInner = 0xFF;
constexpr uint32_t kMaxLeaf = 16;

// Stack/child reference: bit 31 = leaf; a leaf keeps (count-1) in bits 27..30
// and its first item in bits 0..26.  An inner reference is a node index.
constexpr uint32_t kRefLeaf = 0x80000000u;
constexpr uint32_t kRefIndexMask = 0x07FFFFFFu;
constexpr uint32_t kMaxLocalIndex = kRefIndexMask;

struct alignas(16) QuadDev {
    float v[12];  // v0, v1, v2, v3 as packed float3
};
static_assert(sizeof(QuadDev) == 48, "QuadDev must be 48 bytes");

// Instance record, 64 bytes.  A ray entering the instance is re-centred on
// the world ray with error-free FP32 transformations (the point o + t_e d and
// its offset from c are formed exactly as float pairs), so the FP32 object-
// space ray's error scales with the object's size and the transform's
// condition number kappa, not with the object's distance.
struct alignas(64) InstDev {
    float c[3];          // object origin in world space (translation of object->world)
    float R;             // max |coordinate| of the object's bounding box
    float w[9];          // world->object linear part, row-major (FP32 of the FP64 inverse)
    uint32_t node_base;  // global index of this object's BLAS root
    uint32_t quad_base;  // global slot of its first quad == its first albedo row
    float kappa;         // infinity-norm condition number of the linear part
};
static_assert(sizeof(InstDev) == 64, "InstDev must be 64 bytes");

// FP64 world->object linear part, read only by the exact quad re-test.
struct alignas(16) InstDev64 {
    double w[9];
    double pad;
};
static_assert(sizeof(InstDev64) == 80, "InstDev64 must be 80 bytes");

// Everything a kernel needs, passed by value.
struct DevScene {
    const QNode* nodes;
    const QuadDev* quads;
    const uint32_t* prim;
    const InstDev* inst;
    const InstDev64* inst64;
    uint32_t tlas_base;  // global node index of the TLAS root
    uint32_t n_inst;
    float R_top;         // max |coordinate| of the world box
    uint32_t pad;
    uint32_t* err;       // device error word [0] = bits, [1] = first bad index
};

// Device error bits.
constexpr uint32_t kErrStackOverflow = 1u;
constexpr uint32_t kErrStepLimit = 2u;

// Traversal stack entries per ray allocated by the ray-query and wavefront
// trace kernels; tuning.stack caps how many a ray may use (32 or 64).
constexpr int kMaxStack = 64;

}  // namespace qrt

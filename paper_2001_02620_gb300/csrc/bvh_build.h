// Host BVH builder: binned-SAH binary trees collapsed to four-wide nodes with
// conservatively quantised child boxes (qrt_layout.h).  One BLAS per object,
// one TLAS over instance world boxes (Section 5.2: objects instanced, quads as
// the primitive).  Off the hot path: runs once in qrt_scene_create.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "qrt_layout.h"

namespace qrt {

struct BuildOpts {
    uint32_t max_leaf = 2;  // quads per BLAS leaf (2 measured fastest of 1..8)
    uint32_t sah_bins = 16;
    uint32_t threads = 0;
    uint32_t degenerate = 0;
    uint32_t inst_box_level = 5;  // BLAS level whose node boxes bound an instance (0 = root box)
    uint32_t tlas_builder = 0;    // 0 binned SAH (host), 1 linear BVH (device), 2 linear BVH (host)
    uint32_t blas_builder = 0;    // the same choice for the BLASes
};

struct FBox {
    float lo[3], hi[3];
};

struct BlasResult {
    std::vector<QNode> nodes;     // local node indices, root = 0
    std::vector<QuadDev> quads;   // leaf order
    std::vector<uint32_t> prim;   // original quad index of each slot
    FBox box;                     // exact box of all vertices referenced by quads
    uint32_t depth = 0;
};

struct TlasResult {
    std::vector<QNode> nodes;  // local node indices, root = 0; leaves hold instance ids
    uint32_t depth = 0;
};

bool build_blas(const float* verts, uint32_t n_verts, const uint32_t* quads, uint32_t n_quads,
                const BuildOpts& opts, BlasResult& out, std::string& err);

bool build_tlas(const std::vector<FBox>& inst_boxes, const BuildOpts& opts, TlasResult& out,
                std::string& err);

// Invariants of a four-wide tree whose leaves reference items [0, n_items)
// (slots for a BLAS, instance ids for a TLAS): every item exactly once, and
// every dequantised child box contains the exact box of everything below it.
bool check_wide(const std::vector<QNode>& nodes, const std::vector<FBox>& item_boxes,
                std::string& err, uint32_t* depth);

// World box of an object box under an object->world float 3x4 transform:
// centre and half extent mapped in FP64 (the exact box of the eight
// transformed corners), widened by a bound on that arithmetic's rounding and
// rounded outward to float.
FBox transform_box(const FBox& b, const float* xform);

// Dequantised boxes of the BLAS nodes `level` levels below the root (level 1
// = the root's children) together with the leaves above that level; every
// quad of the BLAS lies in one of them.  level 0 returns nothing (use the
// root box).
std::vector<FBox> level_boxes(const std::vector<QNode>& nodes, uint32_t level);

// Dequantised bound used by both the builder and the checker.
float dequant(uint8_t q, int8_t e, float origin);

}  // namespace qrt

// Linear BVH builds of the TLAS and of the BLASes (builders the paper does
// not have: its BVHs come from Embree on the CPU).  Items (instance boxes, or
// quads keyed by mesh) are ordered along a Morton curve of their centres, the
// binary hierarchy over that order is formed node by node in parallel
// (Karras, "Maximizing Parallelism in the Construction of BVHs, Octrees, and
// k-d Trees", HPG 2012), node boxes are merged bottom-up, and the binary tree
// is collapsed top-down to four-wide nodes with conservatively quantised
// child boxes (qrt_layout.h), the same format the host's binned-SAH builder
// writes.  Off the hot path: they run in qrt_scene_create when the caller
// asks for them.
#pragma once
#include <string>
#include <vector>

#include "bvh_build.h"

namespace qrt {

// Builds the TLAS over inst_boxes (one leaf per instance).  on_device = true
// runs every step on the current CUDA device (the nodes are copied back for
// the host's invariant check and the common upload); false runs the same
// per-node functions in host loops (a test aid that needs no GPU).  Returns
// false with err set on bad input or a CUDA error.
bool build_tlas_lbvh(const std::vector<FBox>& inst_boxes, bool on_device, TlasResult& out,
                     std::string& err);

// One mesh's arrays as given to qrt_scene_create (host memory).
struct MeshView {
    const float* verts;
    uint32_t n_verts;
    const uint32_t* quads;
    uint32_t n_quads;
};

// Builds every mesh's BLAS in one pass: all quads sorted by (mesh, Morton
// code of the quad centre on the mesh's own grid of cubic cells), one radix
// tree over them whose mesh-sized subtrees are the BLASes, subtrees of at
// most max_leaf quads taken as leaves, collapsed to four-wide quantised
// nodes with each mesh's nodes numbered from its own root.  The results have
// the host builder's form (nodes, quads in slot order, original quad index
// per slot, box, depth).  on_device as for the TLAS; at most 8192 meshes.
bool build_blases_lbvh(const std::vector<MeshView>& meshes, uint32_t max_leaf, bool on_device,
                       std::vector<BlasResult>& out, std::string& err);

}  // namespace qrt

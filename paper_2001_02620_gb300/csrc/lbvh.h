// Linear BVH build of the TLAS (a builder the paper does not have: its BVHs
// come from Embree on the CPU).  Instance boxes are ordered along a 63-bit
// Morton curve of their centres, the binary hierarchy over that order is
// formed node by node in parallel (Karras, "Maximizing Parallelism in the
// Construction of BVHs, Octrees, and k-d Trees", HPG 2012), node boxes are
// merged bottom-up, and the binary tree is collapsed top-down to four-wide
// nodes with conservatively quantised child boxes (qrt_layout.h), the same
// format the host's binned-SAH builder writes.  Off the hot path: it runs in
// qrt_scene_create when the caller asks for it.
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

}  // namespace qrt

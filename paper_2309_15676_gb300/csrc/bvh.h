// Host BVH builder interface.
#pragma once

#include <stdint.h>

#include <vector>

namespace mer {

// Inner node as built on the host: child boxes and child references. A child
// reference >= 0 is a local inner-node index; < 0 is a leaf ~((first << 3) | (count-1))
// over the leaf-ordered triangle range [first, first+count).
struct HostNode {
    float lo[2][3], hi[2][3];
    int child[2];
};

// Builds a binned-SAH BVH over n_tris triangles (vertex positions pos[nv][3], indices
// tris[n][3]). Returns the root's local index (-1 if no triangles); order[k] is the
// original triangle id of leaf-ordered triangle k.
int build_bvh(const float* pos, const int32_t* tris, int n_tris, std::vector<HostNode>& nodes,
              std::vector<int>& order);

}  // namespace mer

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

// Four-wide inner node: up to four child boxes and references (same encoding as HostNode;
// unused slots hold kEmptyChild and an empty box).
constexpr int kEmptyChild = 0x7fffffff;
struct HostNode4 {
    float lo[4][3], hi[4][3];
    int child[4];
};

// Collapses a binary BVH (root `root`) into a four-wide one, root at index 0: each wide node
// starts from a binary node's two children and repeatedly replaces the inner child of largest
// surface area by its own two children until it holds four (or only leaves are left).
void collapse_bvh4(const std::vector<HostNode>& bin, int root, std::vector<HostNode4>& out);

// Inner-node levels on the deepest root-to-leaf path of a four-wide tree (root = level 1; 0 for an
// empty tree). A nearest-first traversal keeps at most three deferred children per level on its
// stack, so it needs 3 x levels stack entries.
int bvh4_levels(const std::vector<HostNode4>& nodes);

// Builds a binned-SAH BVH over n_tris triangles (vertex positions pos[nv][3], indices
// tris[n][3]). Returns the root's local index (-1 if no triangles); order[k] is the
// original triangle id of leaf-ordered triangle k.
int build_bvh(const float* pos, const int32_t* tris, int n_tris, std::vector<HostNode>& nodes,
              std::vector<int>& order);

}  // namespace mer

// Host-side BVH construction: binned SAH over triangle bounds (16 bins per axis,
// leaves of at most 4 triangles), then collapsed into the four-wide nodes the traversal
// kernels read (see Node in mer_internal.cuh).
#include "bvh.h"

#include <algorithm>
#include <cfloat>
#include <cmath>

namespace mer {

namespace {

struct Box {
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX};
    float hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    void grow(const float* p) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], p[k]);
            hi[k] = std::max(hi[k], p[k]);
        }
    }
    void grow(const Box& b) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], b.lo[k]);
            hi[k] = std::max(hi[k], b.hi[k]);
        }
    }
    float area() const {
        if (lo[0] > hi[0]) return 0.0f;
        const float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0f * (dx * dy + dy * dz + dz * dx);
    }
};

constexpr int kBins = 16;
constexpr int kLeaf = 4;

struct Builder {
    std::vector<Box> tb;              // triangle boxes
    std::vector<float> cen;           // centroids [n][3]
    std::vector<int> idx;             // permutation being partitioned
    std::vector<HostNode> nodes;

    Box range_box(int b, int e) const {
        Box r;
        for (int i = b; i < e; ++i) r.grow(tb[idx[i]]);
        return r;
    }

    // split [b, e) and return the midpoint; falls back to an index median
    int split(int b, int e) {
        Box cb;
        for (int i = b; i < e; ++i) cb.grow(&cen[3 * idx[i]]);
        int best_axis = -1, best_bin = -1;
        float best_cost = FLT_MAX;
        for (int ax = 0; ax < 3; ++ax) {
            const float ext = cb.hi[ax] - cb.lo[ax];
            if (!(ext > 0.0f)) continue;
            Box bb[kBins];
            int bc[kBins] = {0};
            const float sc = kBins / ext;
            for (int i = b; i < e; ++i) {
                int k = (int)((cen[3 * idx[i] + ax] - cb.lo[ax]) * sc);
                k = std::min(std::max(k, 0), kBins - 1);
                bb[k].grow(tb[idx[i]]);
                bc[k]++;
            }
            float la[kBins], ra[kBins];
            int lc[kBins], rc[kBins];
            Box acc;
            int n = 0;
            for (int k = 0; k < kBins; ++k) {
                acc.grow(bb[k]);
                n += bc[k];
                la[k] = acc.area();
                lc[k] = n;
            }
            acc = Box();
            n = 0;
            for (int k = kBins - 1; k >= 0; --k) {
                acc.grow(bb[k]);
                n += bc[k];
                ra[k] = acc.area();
                rc[k] = n;
            }
            for (int k = 0; k < kBins - 1; ++k) {
                if (lc[k] == 0 || rc[k + 1] == 0) continue;
                const float cost = la[k] * lc[k] + ra[k + 1] * rc[k + 1];
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = ax;
                    best_bin = k;
                }
            }
        }
        int mid;
        if (best_axis >= 0) {
            const float ext = cb.hi[best_axis] - cb.lo[best_axis];
            const float sc = kBins / ext;
            auto it = std::partition(idx.begin() + b, idx.begin() + e, [&](int t) {
                int k = (int)((cen[3 * t + best_axis] - cb.lo[best_axis]) * sc);
                k = std::min(std::max(k, 0), kBins - 1);
                return k <= best_bin;
            });
            mid = (int)(it - idx.begin());
        } else {
            mid = (b + e) / 2;
        }
        if (mid <= b || mid >= e) mid = (b + e) / 2;
        return mid;
    }

    // child reference for range [b, e): a leaf if small, otherwise a new inner node
    int child(int b, int e, int depth) {
        if (e - b <= kLeaf) return ~((b << 3) | (e - b - 1));
        return inner(b, e, depth);
    }

    int inner(int b, int e, int depth) {
        const int me = (int)nodes.size();
        nodes.emplace_back();
        int mid = (e - b <= kLeaf) ? (b + (e - b + 1) / 2) : split(b, e);
        if (e - b == 1) mid = e;  // single triangle: both children reference it
        const Box L = range_box(b, mid), R = (e - b == 1) ? range_box(b, e) : range_box(mid, e);
        const int lref = (e - b == 1) ? ~((b << 3) | 0) : child(b, mid, depth + 1);
        const int rref = (e - b == 1) ? ~((b << 3) | 0) : child(mid, e, depth + 1);
        HostNode& n = nodes[me];
        for (int k = 0; k < 3; ++k) {
            n.lo[0][k] = L.lo[k];
            n.hi[0][k] = L.hi[k];
            n.lo[1][k] = R.lo[k];
            n.hi[1][k] = R.hi[k];
        }
        n.child[0] = lref;
        n.child[1] = rref;
        return me;
    }
};

}  // namespace

int build_bvh(const float* pos, const int32_t* tris, int n_tris, std::vector<HostNode>& nodes,
              std::vector<int>& order) {
    nodes.clear();
    order.clear();
    if (n_tris <= 0) return -1;
    Builder B;
    B.tb.resize(n_tris);
    B.cen.resize(3 * (size_t)n_tris);
    B.idx.resize(n_tris);
    for (int i = 0; i < n_tris; ++i) {
        for (int v = 0; v < 3; ++v) B.tb[i].grow(pos + 3 * (size_t)tris[3 * (size_t)i + v]);
        for (int k = 0; k < 3; ++k) B.cen[3 * (size_t)i + k] = 0.5f * (B.tb[i].lo[k] + B.tb[i].hi[k]);
        B.idx[i] = i;
    }
    B.nodes.reserve(2 * (size_t)n_tris / kLeaf + 2);
    const int root = B.inner(0, n_tris, 0);
    nodes.swap(B.nodes);
    order.swap(B.idx);
    return root;
}

namespace {

struct Slot {
    float lo[3], hi[3];
    int ref;
    float area() const {
        const float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0f * (dx * dy + dy * dz + dz * dx);
    }
};

Slot slot_of(const HostNode& n, int k) {
    Slot s;
    for (int a = 0; a < 3; ++a) {
        s.lo[a] = n.lo[k][a];
        s.hi[a] = n.hi[k][a];
    }
    s.ref = n.child[k];
    return s;
}

int emit4(const std::vector<HostNode>& bin, int n2, std::vector<HostNode4>& out) {
    const int me = (int)out.size();
    out.emplace_back();
    Slot slots[4];
    int ns = 2;
    slots[0] = slot_of(bin[n2], 0);
    slots[1] = slot_of(bin[n2], 1);
    while (ns < 4) {
        int best = -1;
        float best_area = -1.0f;
        for (int k = 0; k < ns; ++k)
            if (slots[k].ref >= 0 && slots[k].area() > best_area) {
                best = k;
                best_area = slots[k].area();
            }
        if (best < 0) break;
        const HostNode& c = bin[slots[best].ref];
        slots[best] = slot_of(c, 0);
        slots[ns++] = slot_of(c, 1);
    }
    int refs[4];
    for (int k = 0; k < ns; ++k) refs[k] = slots[k].ref >= 0 ? emit4(bin, slots[k].ref, out) : slots[k].ref;
    HostNode4& w = out[me];
    for (int k = 0; k < 4; ++k) {
        for (int a = 0; a < 3; ++a) {
            w.lo[k][a] = k < ns ? slots[k].lo[a] : 0.0f;
            w.hi[k][a] = k < ns ? slots[k].hi[a] : 0.0f;
        }
        w.child[k] = k < ns ? refs[k] : kEmptyChild;
    }
    return me;
}

}  // namespace

int bvh4_levels(const std::vector<HostNode4>& nodes) {
    if (nodes.empty()) return 0;
    // inner levels along the deepest root-to-leaf path (iterative: node, level)
    std::vector<std::pair<int, int>> todo{{0, 1}};
    int best = 0;
    while (!todo.empty()) {
        const auto [n, lv] = todo.back();
        todo.pop_back();
        best = std::max(best, lv);
        for (int k = 0; k < 4; ++k) {
            const int c = nodes[n].child[k];
            if (c >= 0 && c != kEmptyChild) todo.push_back({c, lv + 1});
        }
    }
    return best;
}

void collapse_bvh4(const std::vector<HostNode>& bin, int root, std::vector<HostNode4>& out) {
    out.clear();
    if (root < 0) return;
    out.reserve(bin.size() / 2 + 1);
    emit4(bin, root, out);
}

}  // namespace mer

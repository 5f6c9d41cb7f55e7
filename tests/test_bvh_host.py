"""The host BVH builder (binned SAH, collapsed to four-wide nodes) checked on the CPU with a small
C++ program linked against it: the leaf order is a permutation of the triangles, every child box
of the binary and of the four-wide tree contains its subtree's triangles, the four-wide leaves
cover every triangle exactly once (a one-triangle scene's root holds it twice), the reported number of
inner levels (which bounds the traversal stack) equals the depth found by recursion, and a stack
traversal of the four-wide tree finds the same
closest hit as brute force for random rays. Inputs: a small spiral and a small displaced sphere
(the synthetic scenes), and degenerate sets (one triangle, many identical triangles, a flat grid
whose boxes have zero thickness, long thin triangles). On the synthetic meshes the tree's SAH cost
is also compared with that of an object-median tree built by the checker."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2309_15676_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2309_15676_gb300", "csrc")

PROG = r'''
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>
#include "bvh.h"
using namespace mer;
static int nv, nt;
static std::vector<float> P;
static std::vector<int> T;
static bool inside(const float* lo, const float* hi, int tri) {
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a) {
            const float x = P[3 * T[3 * tri + k] + a];
            if (x < lo[a] || x > hi[a]) return false;
        }
    return true;
}
static bool hit_tri(int tri, const double o[3], const double d[3], double& t) {
    double v[3][3];
    for (int k = 0; k < 3; ++k) for (int a = 0; a < 3; ++a) v[k][a] = P[3 * T[3 * tri + k] + a];
    double e1[3], e2[3], pv[3], tv[3], qv[3];
    for (int a = 0; a < 3; ++a) { e1[a] = v[1][a] - v[0][a]; e2[a] = v[2][a] - v[0][a]; tv[a] = o[a] - v[0][a]; }
    pv[0] = d[1] * e2[2] - d[2] * e2[1]; pv[1] = d[2] * e2[0] - d[0] * e2[2]; pv[2] = d[0] * e2[1] - d[1] * e2[0];
    const double det = e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2];
    if (det == 0.0) return false;
    const double u = (tv[0] * pv[0] + tv[1] * pv[1] + tv[2] * pv[2]) / det;
    if (u < 0 || u > 1) return false;
    qv[0] = tv[1] * e1[2] - tv[2] * e1[1]; qv[1] = tv[2] * e1[0] - tv[0] * e1[2]; qv[2] = tv[0] * e1[1] - tv[1] * e1[0];
    const double w = (d[0] * qv[0] + d[1] * qv[1] + d[2] * qv[2]) / det;
    if (w < 0 || u + w > 1) return false;
    t = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) / det;
    return t > 0;
}
static bool box_hit(const float* lo, const float* hi, const double o[3], const double d[3], double tmax) {
    double t0 = 0, t1 = tmax;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0) { if (o[a] < lo[a] || o[a] > hi[a]) return false; continue; }
        double ta = (lo[a] - o[a]) / d[a], tb = (hi[a] - o[a]) / d[a];
        if (ta > tb) std::swap(ta, tb);
        t0 = std::max(t0, ta); t1 = std::min(t1, tb);
    }
    return t0 <= t1 * (1 + 1e-9) + 1e-12;
}
int main() {
    if (scanf("%d %d", &nv, &nt) != 2) return 2;
    P.resize(3 * nv); T.resize(3 * nt);
    for (auto& x : P) if (scanf("%f", &x) != 1) return 2;
    for (auto& x : T) if (scanf("%d", &x) != 1) return 2;
    std::vector<HostNode> bin; std::vector<int> order;
    const int root = build_bvh(P.data(), T.data(), nt, bin, order);
    // order: a permutation
    std::vector<int> seen(nt, 0);
    if ((int)order.size() != nt) { printf("FAIL order size\n"); return 1; }
    for (int x : order) { if (x < 0 || x >= nt || seen[x]++) { printf("FAIL order perm\n"); return 1; } }
    // binary: child boxes contain their subtrees
    std::vector<std::pair<int,int>> range(bin.size(), {1 << 30, -1});
    std::function<void(int, int&, int&)> walk;
    int bad = 0;
    std::function<void(int, const float*, const float*)> check_bin = [&](int ref, const float* lo, const float* hi) {
        if (ref < 0) {
            const int x = ~ref, first = x >> 3, cnt = (x & 7) + 1;
            for (int k = first; k < first + cnt; ++k) if (!inside(lo, hi, order[k])) ++bad;
            return;
        }
        for (int c = 0; c < 2; ++c) {
            const HostNode& n = bin[ref];
            for (int a = 0; a < 3; ++a) if (n.lo[c][a] < lo[a] || n.hi[c][a] > hi[a]) ++bad;
            check_bin(n.child[c], n.lo[c], n.hi[c]);
        }
    };
    const float big_lo[3] = {-1e30f, -1e30f, -1e30f}, big_hi[3] = {1e30f, 1e30f, 1e30f};
    if (root >= 0) check_bin(root, big_lo, big_hi);
    if (bad) { printf("FAIL binary boxes %d\n", bad); return 1; }
    // four-wide: boxes contain subtrees, leaves cover every leaf-ordered triangle once
    std::vector<HostNode4> w;
    collapse_bvh4(bin, root, w);
    std::vector<int> cover(nt, 0), visits(w.size(), 0);
    std::function<void(int)> check4 = [&](int i) {
        if (visits[i]++) { ++bad; return; }
        for (int c = 0; c < 4; ++c) {
            const int ref = w[i].child[c];
            if (ref == kEmptyChild) continue;
            if (ref < 0) {
                const int x = ~ref, first = x >> 3, cnt = (x & 7) + 1;
                for (int k = first; k < first + cnt; ++k) {
                    if (k < 0 || k >= nt) { ++bad; continue; }
                    ++cover[k];
                    if (!inside(w[i].lo[c], w[i].hi[c], order[k])) ++bad;
                }
            } else {
                if (ref >= (int)w.size()) { ++bad; continue; }
                for (int c2 = 0; c2 < 4; ++c2) {
                    if (w[ref].child[c2] == kEmptyChild) continue;
                    for (int a = 0; a < 3; ++a)
                        if (w[ref].lo[c2][a] < w[i].lo[c][a] || w[ref].hi[c2][a] > w[i].hi[c][a]) ++bad;
                }
                check4(ref);
            }
        }
    };
    if (!w.empty()) check4(0);
    // inner levels of the deepest path (the traversal stack bound) by recursion
    std::function<int(int)> levels = [&](int i) -> int {
        int m = 0;
        for (int c = 0; c < 4; ++c) if (w[i].child[c] >= 0 && w[i].child[c] != kEmptyChild) m = std::max(m, levels(w[i].child[c]));
        return 1 + m;
    };
    if (bvh4_levels(w) != (w.empty() ? 0 : levels(0))) { printf("FAIL levels\n"); return 1; }
    // exactly once (a one-triangle scene's root references its triangle from both children)
    for (int k = 0; k < nt; ++k) if (nt == 1 ? cover[k] < 1 : cover[k] != 1) ++bad;
    if (bad) { printf("FAIL four-wide %d\n", bad); return 1; }
    // closest hit: stack traversal of the four-wide tree == brute force
    float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
    for (int i = 0; i < nv; ++i) for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], P[3 * i + a]); hi[a] = std::max(hi[a], P[3 * i + a]); }
    std::mt19937 rng(7); std::uniform_real_distribution<double> U(0, 1);
    int hits = 0;
    for (int r = 0; r < 2000; ++r) {
        double o[3], tg[3], d[3];
        for (int a = 0; a < 3; ++a) { const double ext = hi[a] - lo[a] + 1e-3; o[a] = lo[a] - 0.5 * ext + 2 * ext * U(rng); tg[a] = lo[a] + ext * U(rng); d[a] = tg[a] - o[a]; }
        const double len = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]); for (double& x : d) x /= len;
        double tb = INFINITY; int pb = -1;
        for (int k = 0; k < nt; ++k) { double t; if (hit_tri(k, o, d, t) && (t < tb || (t == tb && k < pb))) { tb = t; pb = k; } }
        double tt = INFINITY; int pt = -1;
        std::vector<int> st; if (!w.empty()) st.push_back(0);
        while (!st.empty()) {
            const int i = st.back(); st.pop_back();
            for (int c = 0; c < 4; ++c) {
                const int ref = w[i].child[c];
                if (ref == kEmptyChild || !box_hit(w[i].lo[c], w[i].hi[c], o, d, tt)) continue;
                if (ref >= 0) { st.push_back(ref); continue; }
                const int x = ~ref, first = x >> 3, cnt = (x & 7) + 1;
                for (int k = first; k < first + cnt; ++k) { double t; const int id = order[k];
                    if (hit_tri(id, o, d, t) && (t < tt || (t == tt && id < pt))) { tt = t; pt = id; } }
            }
        }
        if (pt != pb) { printf("FAIL ray %d: %d vs %d\n", r, pt, pb); return 1; }
        hits += pb >= 0;
    }
    // SAH cost of the binary tree (node areas relative to the root: one unit per inner node
    // reached, one per triangle tested) against an object-median tree built here (longest
    // centroid axis, leaves of at most 4)
    auto tri_box = [&](int t, float* lo, float* hi) {
        for (int a = 0; a < 3; ++a) { lo[a] = 1e30f; hi[a] = -1e30f; }
        for (int k = 0; k < 3; ++k) for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], P[3 * T[3 * t + k] + a]); hi[a] = std::max(hi[a], P[3 * T[3 * t + k] + a]); }
    };
    auto area = [](const float* lo, const float* hi) {
        const double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    };
    double root_area = 0.0;
    {
        float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
        for (int t = 0; t < nt; ++t) { float a[3], b[3]; tri_box(t, a, b);
            for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], a[k]); hi[k] = std::max(hi[k], b[k]); } }
        root_area = std::max(area(lo, hi), 1e-30);
    }
    std::function<double(int, const float*, const float*)> lib_cost = [&](int ref, const float* lo, const float* hi) -> double {
        const double a = area(lo, hi) / root_area;
        if (ref < 0) return a * ((~ref & 7) + 1);
        const HostNode& n = bin[ref];
        return a + lib_cost(n.child[0], n.lo[0], n.hi[0]) + lib_cost(n.child[1], n.lo[1], n.hi[1]);
    };
    std::vector<int> ids(nt);
    for (int t = 0; t < nt; ++t) ids[t] = t;
    std::function<double(int, int)> med_cost = [&](int b, int e) -> double {
        float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f}, clo[3] = {1e30f, 1e30f, 1e30f}, chi[3] = {-1e30f, -1e30f, -1e30f};
        for (int i = b; i < e; ++i) { float x[3], y[3]; tri_box(ids[i], x, y);
            for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], x[k]); hi[k] = std::max(hi[k], y[k]);
                const float c = 0.5f * (x[k] + y[k]); clo[k] = std::min(clo[k], c); chi[k] = std::max(chi[k], c); } }
        const double a = area(lo, hi) / root_area;
        if (e - b <= 4) return a * (e - b);
        int ax = 0;
        for (int k = 1; k < 3; ++k) if (chi[k] - clo[k] > chi[ax] - clo[ax]) ax = k;
        const int m = (b + e) / 2;
        std::nth_element(ids.begin() + b, ids.begin() + m, ids.begin() + e, [&](int u, int v) {
            float ul[3], uh[3], vl[3], vh[3]; tri_box(u, ul, uh); tri_box(v, vl, vh);
            return ul[ax] + uh[ax] < vl[ax] + vh[ax]; });
        return a + med_cost(b, m) + med_cost(m, e);
    };
    const double c_lib = root >= 0 ? 1.0 + lib_cost(bin[root].child[0], bin[root].lo[0], bin[root].hi[0]) +
                                         lib_cost(bin[root].child[1], bin[root].lo[1], bin[root].hi[1]) : 0.0;
    const double c_med = nt > 0 ? med_cost(0, nt) : 0.0;
    printf("ok %zu %zu %d %.6g %.6g\n", bin.size(), w.size(), hits, c_lib, c_med);
    return 0;
}
'''


def _cases():
    rng = np.random.default_rng(3)
    sp = synth.workload_spiral(16, 16, 32, 8, 16, max_depth=3).scene
    ds = synth.workload_sphere(64, 64, 64, 40, max_depth=3).scene if hasattr(synth, "workload_sphere") else None
    out = [("spiral", sp["positions"], sp["tris"])]
    if ds is not None:
        out.append(("dsphere", ds["positions"], ds["tris"]))
    one = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    out.append(("one", one, np.array([[0, 1, 2]], np.int32)))
    same = np.tile(one, (37, 1))
    out.append(("identical", same, np.arange(3 * 37, dtype=np.int32).reshape(37, 3)))
    g = 12   # flat grid: every box has zero thickness in z
    xs, ys = np.meshgrid(np.arange(g + 1, dtype=np.float32), np.arange(g + 1, dtype=np.float32))
    grid = np.stack([xs.ravel(), ys.ravel(), np.zeros(xs.size, np.float32)], 1)
    tris = []
    for y in range(g):
        for x in range(g):
            a = y * (g + 1) + x
            tris += [[a, a + 1, a + g + 1], [a + 1, a + g + 2, a + g + 1]]
    out.append(("flat", grid, np.asarray(tris, np.int32)))
    thin = rng.uniform(-1, 1, (60, 3)).astype(np.float32)
    thin[1::3] = thin[0::3] + np.array([50.0, 0.0, 0.0], np.float32)   # long slivers
    thin[2::3] = thin[0::3] + np.array([50.0, 1e-3, 0.0], np.float32)
    out.append(("thin", thin, np.arange(60, dtype=np.int32).reshape(20, 3)))
    return out


@pytest.fixture(scope="module")
def checker():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "bvhcheck.cpp")
    exe = os.path.join(d, "bvhcheck")
    open(src, "w").write(PROG.replace("#include <random>", "#include <random>\n#include <functional>\n#include <algorithm>"))
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, src, os.path.join(CSRC, "bvh.cpp"), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    yield exe
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("case", [c[0] for c in _cases()])
def test_bvh_invariants_and_closest_hits(checker, case):
    name, pos, tris = [c for c in _cases() if c[0] == case][0]
    pos = np.asarray(pos, np.float32)
    tris = np.asarray(tris, np.int32)
    inp = f"{pos.shape[0]} {tris.shape[0]}\n" + " ".join(repr(float(x)) for x in pos.ravel()) + "\n" + \
        " ".join(str(int(x)) for x in tris.ravel()) + "\n"
    r = subprocess.run([checker], input=inp, capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), (case, r.stdout, r.stderr)
    if case in ("spiral", "dsphere"):
        # the binned-SAH tree costs well under an object-median tree of the same leaf size (0.41x and
        # 0.21x on these meshes); a builder that lost its SAH split would not
        c_lib, c_med = (float(x) for x in r.stdout.split()[4:6])
        assert 0.0 < c_lib <= 0.7 * c_med, (case, c_lib, c_med)

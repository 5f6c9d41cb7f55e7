// Wavefront pass machinery shared by the tracer kernels and their host launcher.
#pragma once

#include "mer_internal.cuh"

namespace mer {

enum PassMode : int { MODE_PRIMAL = 0, MODE_ADJ_FWD = 1, MODE_REPLAY = 2 };

// counter block layout (u32); words [0, CNT_ERR) are zeroed at the start of every pass
constexpr int CNT_Q = 0;       // [k]: entries of the path queue consumed at depth k
constexpr int CNT_S = 32;      // [k]: shadow entries produced at depth k
constexpr int CNT_R = 64;      // records produced by the pass
constexpr int CNT_FETCH = 65;  // [k]: work units taken by the trace launch of depth k (k <= 17)
constexpr int CNT_ERR = 95;    // first error code seen by a kernel (bounds, waits), kept across passes
constexpr int CNT_WORDS = 96;

// path-queue fields (float), per branch b: base index b * QF_PER_BRANCH
constexpr int QF_O = 0, QF_D = 3, QF_BETA = 6, QF_PDFB = 9, QF_PDFENV = 10, QF_PER_BRANCH = 11;
// path-queue words (u32): path id, flags (bit0/1 branch alive, bit2 coincident, bits 8..15 problem)
constexpr int QU_PATH = 0, QU_FLAGS = 1, QU_WORDS = 2;
// hit fields (float), per branch: t, b1, b2; prim (int) separately
constexpr int HF_T = 0, HF_B1 = 1, HF_B2 = 2, HF_PER_BRANCH = 3;
// shadow entry fields (float): origin, direction, tmax, then per slot: contrib rgb, g_nee[5]
constexpr int SF_O = 0, SF_D = 3, SF_TMAX = 6, SF_SLOT = 7, SF_PER_SLOT = 8;
// shadow entry words: path id, meta (problem | slot mask << 8), record index per slot
constexpr int SU_PATH = 0, SU_META = 1, SU_REC = 2;
// gradient record, 32 B (two 16-byte accesses): footprint word (problem << 24 | (y0+1) << 12 |
// (x0+1)), bilinear fractions, and the derivative g[5] w.r.t. the fetched channels
struct __align__(16) Record {
    uint32_t pos;
    float fx, fy;
    float g[5];
};

constexpr uint32_t FLAG_A = 1u, FLAG_B = 2u, FLAG_COINC = 4u;

struct PassArgs {
    // problems taking part: table form (entry e covers paths [path_off[e], path_off[e+1])) or,
    // if inl_prob >= 0, the single problem inl_prob with paths [0, n_paths)
    const ProblemDev* probs;
    ProbState* pstate;
    const int32_t* entry_prob;
    const int64_t* path_off;
    int32_t n_entries;
    int32_t inl_prob;
    int64_t n_paths;
    uint32_t stream;
    int32_t fd_kind;          // 1: FD pair samples (spp_fd; problems at iteration 0 have none)
    int32_t iter_override;    // >= 0: Philox iteration word for every problem
    int32_t spp_override;     // > 0: samples per pixel of the estimate (adjoint weight 1/spp)
    int32_t sample_base;      // first sample index of this chunk of paths
    // single-problem overrides: textures per branch and adjoint images per branch
    const float* tex_over[2];
    const float* dimg_over[2];
    // wavefront buffers
    float* qf[2];
    uint32_t* qu[2];
    int64_t qcap;
    float* hitf;
    int32_t* hitp;
    float* shf;
    uint32_t* shu;
    int64_t shcap;
    uint32_t* cnt;
    float* lacc;              // [NB*3][qcap] radiance accumulated by this pass
    const float* ltot;        // [NB*3][qcap] radiance of the ADJ_FWD pass (REPLAY)
    Record* rec;
    int64_t rcap;
    // hit store of a PRB pair of passes: the ADJ_FWD pass (PRIMAL kernels) writes, for branch b,
    // depth k (1-based) and path g, the closest hit hs[(b * hs_depth + k - 1) * hs_cap + g] =
    // {t, b1, b2, prim bits} (its shade kernel, as it reads the hit) and the visibility of the NEE
    // shadow ray hvis[same index] (0 / 1, the shadow test); its REPLAY pass reads them and launches
    // no traversal. nullptr: the replay re-traces.
    float4* hs;
    uint8_t* hvis;
    int32_t hs_depth;
    int64_t hs_cap;
    int32_t smem_nodes;       // top BVH nodes of problem smem_prob staged in shared memory
    int32_t smem_prob;
    int32_t refill;           // traversal: idle lanes of a warp that trigger fetching new rays
    unsigned long long* stats; // counting run: [2*class] node tests, [2*class+1] primitive tests
};

__device__ __forceinline__ int find_entry(const int64_t* off, int n, int64_t g) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace mer

// Gradient scatter (step a10), image loss and adjoint images (step a7), Philox fill.
#include "kernels.cuh"
#include "wavefront.cuh"

namespace mer {

KernelTimer* g_timer = nullptr;

constexpr unsigned FULLM = 0xffffffffu;

// Fire-and-forget reduction: no value comes back, so the issuing warp never waits on the L2
// (the vector atomicAdd overloads return the old value and compile to waiting atomics)
__device__ __forceinline__ void red_add(float* p, float a) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(a) : "memory");
}

// L2 policy that keeps lines resident ahead of streamed data: the gradient textures are cleared
// with it right before their scatter, and the scatter's reductions carry it, so that the
// read-modify-writes find their lines in L2 while the records stream through (evict-first)
__device__ __forceinline__ uint64_t evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// No "memory" clobber: nothing in the scatter reads the gradient texture, and without it the
// compiler may hoist the shared-memory loads of the next rows above the reduction
__device__ __forceinline__ void red_add_keep(float* p, float a, uint64_t pol) {
    asm volatile("red.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(a), "l"(pol));
}


// per-problem fields the scatter needs, cached in shared memory: the layout and the gradient
// texture this launch adds to (NULL: the problem has none and its records are skipped)
struct SProb {
    int C, W, H, pad;
    float* tgt;
    float* pad2;
};

// gradient texture `which` of a problem: 0 F, 1 dF, 2 F_var, 3 dF_var
__device__ __forceinline__ float* grad_target(const ProblemDev& P, int which) {
    return which == 0 ? P.F : which == 1 ? P.dF : which == 2 ? P.Fv : P.dFv;
}

template <int CC>
__device__ __forceinline__ void fill_row(float (&v)[10], const float (&g)[MAXC], float wa, float wb) {
#pragma unroll
    for (int c = 0; c < CC; ++c) {
        v[c] = wa * g[c];
        v[CC + c] = wb * g[c];   // ignored beyond the run length when the taps merged
    }
}

// ---- staging: per-warp bulk-copy (TMA) ring of records and per-record reduction rows ----

constexpr int SC_THREADS = 256;
constexpr int SC_WARPS = SC_THREADS / 32;
constexpr int SC_STAGES = 2;                        // chunks in flight per warp
constexpr int SC_CHUNK = 32;                        // records per chunk (one per lane in phase 1)
constexpr int SC_ROWS = 2 * SC_CHUNK;               // bilinear rows of a chunk
constexpr uint32_t SC_WAIT_POLLS = 1u << 20;        // bound on the polls of one stage barrier
constexpr uint64_t SC_WAIT_NS = 200000000ull;       // and on its wall time (0.2 s)
constexpr uint32_t SC_SUSPEND_NS = 1000;            // suspend hint of one poll

// Per-warp staging. The chunk's non-empty bilinear rows are compacted: row q keeps its ten values
// (zero beyond its length) at vals[10 q ...] and the address of its first float at addr[q], so that
// a reduction step of three rows reads thirty contiguous values (one shared-memory wavefront) and
// three row addresses. When footprints merge, vals first holds each lane's two raw rows at
// vals[20 lane ...].
struct __align__(16) WarpArea {
    Record ring[SC_STAGES][SC_CHUNK];   // records, filled by bulk copies
    float vals[SC_ROWS * 10];           // row values, compacted
    float* addr[SC_ROWS];               // row start addresses, compacted
};
constexpr size_t SC_HEAD = 256;         // stage barriers, then the warp areas, then the problem table

size_t scatter_smem(int n_probs) { return SC_HEAD + sizeof(WarpArea) * SC_WARPS + sizeof(SProb) * (size_t)n_probs; }

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

// one elected lane: arm the stage barrier with the byte count, then start the bulk copy that
// completes it (source and destination 16-byte aligned, size a multiple of 16). The records are
// read once: the copy marks their lines evict-first so that they do not push the gradient
// texture out of L2.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(SC_SUSPEND_NS)
        : "memory");
    return done != 0;
}

// polls the barrier phase with the given parity; false once limit_ns have passed (or after
// SC_WAIT_POLLS polls) without the phase completing. The clock is read only after a first
// unsuccessful poll.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = SC_WAIT_NS) {
    const uint32_t a = smem_addr(bar);
    if (mbar_try(a, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t k = 0; k < SC_WAIT_POLLS; ++k) {
        if (mbar_try(a, parity)) return true;
        if ((k & 15u) == 15u && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// Self-test of the bounded wait: one thread arms a fresh barrier for one arrival that nothing
// makes, waits with the given limit and records the outcome (MER_OK or MER_ERR_TIMEOUT) and
// the time the wait took.
__global__ void k_wait_selftest(uint64_t limit_ns, int32_t* status, uint64_t* waited_ns) {
    __shared__ __align__(8) uint64_t bar;
    mbar_init(&bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const uint64_t t0 = global_ns();
    const bool ok = mbar_wait(&bar, 0u, limit_ns);
    *waited_ns = global_ns() - t0;
    *status = ok ? MER_OK : MER_ERR_TIMEOUT;
}

int run_wait_selftest(uint64_t limit_ns, int32_t* status, uint64_t* waited_ns, cudaStream_t st) {
    k_wait_selftest<<<1, 1, 0, st>>>(limit_ns, status, waited_ns);
    return 1;
}

// Records of a chunk that share a footprint origin are merged only when some origin is held by at
// least this many lanes: at 1024^2 over a 2048^2 texture a chunk's groups are pairs at most in 99%
// of chunks, and merging pairs costs more instructions than the 3% of reductions it saves; an image
// much finer than its texture (many lanes per texel) merges.
constexpr int SC_MERGE_MIN = 3;

// Writes compacted row q (values v[0..10), zero beyond the row's length, to be added at p)
__device__ __forceinline__ void put_row(WarpArea& WA, int q, float* p, const float (&v)[10]) {
    float2* d = reinterpret_cast<float2*>(WA.vals + 10 * q);
#pragma unroll
    for (int j = 0; j < 5; ++j) d[j] = make_float2(v[2 * j], v[2 * j + 1]);
    WA.addr[q] = p;
}

// Phase 1, one record per lane: the bilinear footprint (clamp-to-edge) of the record's texel
// window becomes two rows of up to 2C contiguous floats (taps xa, xb of texel rows ya, yb;
// taps that clamp onto the same texel are merged first) holding w_k g[c]; the values beyond a
// row's length are zero (a single-texel row's second tap has weight zero). Lanes whose record is
// absent or all-zero sit out. When some footprint origin is held by SC_MERGE_MIN lanes or more,
// each group's first lane adds its peers' rows (in lane order) and alone keeps them. The non-empty
// rows are compacted (ballot + prefix count: every lane's first row, then every lane's second row)
// into the warp's area; returns their number, the same on every lane.
__device__ __forceinline__ int stage_record(bool valid, float4 a, float4 b, const SProb* sp, float* grad_over,
                                            WarpArea& WA, int lane) {
    const uint32_t pos = __float_as_uint(a.x);
    const float g[MAXC] = {a.w, b.x, b.y, b.z, b.w};
    valid = valid && (g[0] != 0.0f || g[1] != 0.0f || g[2] != 0.0f || g[3] != 0.0f || g[4] != 0.0f);
    const unsigned vmask = __ballot_sync(FULLM, valid);
    bool r0 = false, r1 = false;
    int off0 = 0, off1 = 0;
    float* base = nullptr;
    unsigned peers = 0;
    int maxg = 0;
    float v0[10], v1[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) v0[k] = v1[k] = 0.0f;
    if (valid) {
        const SProb P = sp[pos >> 24];
        const int C = P.C, W = P.W, H = P.H;
        const int x0 = (int)(pos & 0xfff) - 1, y0 = (int)((pos >> 12) & 0xfff) - 1;
        const float fx = a.y, fy = a.z;
        const int xa = max(x0, 0), xb = min(x0 + 1, W - 1), ya = max(y0, 0), yb = min(y0 + 1, H - 1);
        float w00 = (1.0f - fx) * (1.0f - fy), w10 = fx * (1.0f - fy), w01 = (1.0f - fx) * fy, w11 = fx * fy;
        const bool one_x = xa == xb, one_y = ya == yb;
        if (one_x) { w00 += w10; w10 = 0.0f; w01 += w11; w11 = 0.0f; }
        if (one_y) { w00 += w01; w10 += w11; w01 = 0.0f; w11 = 0.0f; }
        if (C == 5) { fill_row<5>(v0, g, w00, w10); fill_row<5>(v1, g, w01, w11); }
        else { fill_row<3>(v0, g, w00, w10); fill_row<3>(v1, g, w01, w11); }
        // texture extents are below 4096 per side and C <= 5: offsets fit in 32 bits
        off0 = (ya * W + xa) * C;
        off1 = (yb * W + xa) * C;
        base = grad_over ? grad_over : P.tgt;
        r0 = base != nullptr;
        r1 = r0 && !one_y;
        // same pos => same problem and layout
        peers = __match_any_sync(vmask, pos);
        maxg = (int)__reduce_max_sync(vmask, (unsigned)__popc(peers));
    }
    maxg = __shfl_sync(FULLM, maxg, vmask ? __ffs(vmask) - 1 : 0);
    if (maxg >= SC_MERGE_MIN) {   // warp-uniform
        float4* d = reinterpret_cast<float4*>(WA.vals + 20 * lane);
        if (valid) {
            d[0] = make_float4(v0[0], v0[1], v0[2], v0[3]);
            d[1] = make_float4(v0[4], v0[5], v0[6], v0[7]);
            d[2] = make_float4(v0[8], v0[9], v1[0], v1[1]);
            d[3] = make_float4(v1[2], v1[3], v1[4], v1[5]);
            d[4] = make_float4(v1[6], v1[7], v1[8], v1[9]);
        }
        __syncwarp();
        const bool lead = valid && lane == __ffs(peers) - 1;
        unsigned others = lead ? (peers & ~(1u << lane)) : 0u;
        for (int i = 1; i < maxg; ++i) {
            if (others) {
                const float4* o = reinterpret_cast<const float4*>(WA.vals + 20 * (__ffs(others) - 1));
                const float4 x0 = o[0], x1 = o[1], x2 = o[2], x3 = o[3], x4 = o[4];
                v0[0] += x0.x; v0[1] += x0.y; v0[2] += x0.z; v0[3] += x0.w;
                v0[4] += x1.x; v0[5] += x1.y; v0[6] += x1.z; v0[7] += x1.w;
                v0[8] += x2.x; v0[9] += x2.y; v1[0] += x2.z; v1[1] += x2.w;
                v1[2] += x3.x; v1[3] += x3.y; v1[4] += x3.z; v1[5] += x3.w;
                v1[6] += x4.x; v1[7] += x4.y; v1[8] += x4.z; v1[9] += x4.w;
                others &= others - 1;
            }
        }
        __syncwarp();   // every raw row is read before the compacted rows overwrite the area
        if (valid && !lead) r0 = r1 = false;
    }
    const unsigned m0 = __ballot_sync(FULLM, r0), m1 = __ballot_sync(FULLM, r1);
    const unsigned below = (1u << lane) - 1u;
    const int n0 = __popc(m0);
    if (r0) put_row(WA, __popc(m0 & below), base + off0, v0);
    if (r1) put_row(WA, n0 + __popc(m1 & below), base + off1, v1);
    return n0 + __popc(m1);
}

// Phase 2, ten lanes per row and three rows per step over the compacted rows: step t reads the
// contiguous values vals[30 t + lane] and the three row addresses, and each reduction instruction
// adds up to three runs of 2C floats, which the load/store unit packs into one request per 32-byte
// sector. Zero values (a row's padding, or an exactly zero product) add nothing and are skipped.
__device__ __forceinline__ void reduce_rows(const WarpArea& WA, int lane, int nrows, uint64_t pol) {
    const int slot = lane / 10, e = lane - 10 * slot;
    if (slot >= 3) return;
    for (int q = slot, f = lane; q < nrows; q += 3, f += 30) {
        const float v = WA.vals[f];
        float* p = WA.addr[q];
        if (v != 0.0f) red_add_keep(p + e, v, pol);
    }
}

// Persistent over chunks of 32 records: warp w of the grid takes chunks w, w + total_warps, ...
// Lane 0 keeps SC_STAGES bulk copies (1 KB each) in flight into the warp's shared-memory ring;
// every lane reads its record once the stage's barrier completes, the ring slot is refilled with
// the chunk SC_STAGES ahead, and the chunk is staged (phase 1) and reduced (phase 2) while the
// copies are in flight. A barrier that does not complete within its bound stops the warp,
// records MER_ERR_TIMEOUT in the error word and waits (bounded) for its copies still in flight.
__global__ void __launch_bounds__(SC_THREADS) k_scatter(uint32_t* __restrict__ cnt, const Record* __restrict__ rec,
                                                        int64_t rcap, const ProblemDev* __restrict__ probs,
                                                        int n_probs, float* grad_over, int which) {
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm);
    WarpArea* areas = reinterpret_cast<WarpArea*>(sm + SC_HEAD);
    SProb* sp = reinterpret_cast<SProb*>(sm + SC_HEAD + sizeof(WarpArea) * SC_WARPS);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    WarpArea& WA = areas[wib];
    uint64_t* bar = bars + wib * SC_STAGES;
    const uint64_t keep = evict_last_policy();
    for (int t = threadIdx.x; t < n_probs; t += blockDim.x) {
        const ProblemDev& P = probs[t];
        sp[t] = SProb{P.tex_c, P.tex_w, P.tex_h, 0, grad_target(P, which), nullptr};
    }
    if (lane == 0)
        for (int s = 0; s < SC_STAGES; ++s) mbar_init(&bar[s]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();

    const int64_t n = min((int64_t)cnt[CNT_R], rcap);
    const int64_t nchunks = (n + SC_CHUNK - 1) / SC_CHUNK;
    const int64_t gw = (int64_t)blockIdx.x * SC_WARPS + wib, tw = (int64_t)gridDim.x * SC_WARPS;
    const int64_t my = nchunks > gw ? (nchunks - gw + tw - 1) / tw : 0;   // chunks of this warp
    auto issue = [&](int64_t k) {
        const int64_t first = (gw + k * tw) * SC_CHUNK;
        const uint32_t cnt_k = (uint32_t)min((int64_t)SC_CHUNK, n - first);
        bulk_load(WA.ring[k % SC_STAGES], rec + first, cnt_k * (uint32_t)sizeof(Record), &bar[k % SC_STAGES]);
    };
    if (lane == 0)
        for (int64_t k = 0; k < min(my, (int64_t)SC_STAGES); ++k) issue(k);
    for (int64_t k = 0; k < my; ++k) {
        const int s = (int)(k % SC_STAGES);
        const bool ok = mbar_wait(&bar[s], (uint32_t)(k / SC_STAGES) & 1u);
        if (!__all_sync(FULLM, ok)) {
            if (lane == 0) {
                atomicCAS(&cnt[CNT_ERR], 0u, (uint32_t)MER_ERR_TIMEOUT);
                // drain the copies still in flight into this warp's ring before the block can
                // leave (ten times the normal limit); the host refuses the context from now on
                for (int64_t q = k; q < min(my, k + SC_STAGES); ++q)
                    mbar_wait(&bar[q % SC_STAGES], (uint32_t)(q / SC_STAGES) & 1u, 10 * SC_WAIT_NS);
            }
            __syncwarp();
            return;
        }
        const bool valid = (gw + k * tw) * SC_CHUNK + lane < n;
        float4 a = make_float4(0, 0, 0, 0), b = a;
        if (valid) {
            // lanes 4-7 of each group of eight read the two halves in the other order, so that the
            // eight 16-byte reads of one shared-memory wavefront fall on distinct banks
            const float4* r = reinterpret_cast<const float4*>(&WA.ring[s][lane]);
            const int h = (lane >> 2) & 1;
            const float4 x = r[h], y = r[h ^ 1];
            a = h ? y : x;
            b = h ? x : y;
        }
        __syncwarp();
        if (lane == 0 && k + SC_STAGES < my) {
            // the generic-proxy reads of this slot are ordered before the async-proxy refill
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(k + SC_STAGES);
        }
        const int nrows = stage_record(valid, a, b, sp, grad_over, WA, lane);
        __syncwarp();
        reduce_rows(WA, lane, nrows, keep);
        __syncwarp();   // the rows are read before the next chunk overwrites them
    }
}

// float4 stores over each problem's gradient texture `which` (16-byte aligned allocations;
// scalar tail; problems without one are skipped), marked evict-last in L2 for the scatter that
// follows
__global__ void k_zero_grads(const ProblemDev* __restrict__ probs, int n_probs, int which) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t keep = evict_last_policy();
    for (int q = 0; q < n_probs; ++q) {
        float* g = grad_target(probs[q], which);
        if (!g) continue;
        const int64_t n = probs[q].n_par, n4 = n >> 2;
        float4* g4 = reinterpret_cast<float4*>(g);
        for (int64_t i = t0; i < n4; i += stride)
            asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %1, %1, %1}, %2;" ::"l"(g4 + i), "f"(0.0f),
                         "l"(keep)
                         : "memory");
        for (int64_t i = 4 * n4 + t0; i < n; i += stride) g[i] = 0.0f;
    }
}

int run_zero_grads(const ProblemDev* probs, int n_probs, int which, int grid, cudaStream_t st) {
    MER_TIMED(KC_ZERO, st, k_zero_grads<<<grid, 256, 0, st>>>(probs, n_probs, which));
    return 1;
}

int run_scatter(uint32_t* cnt, const Record* rec, int64_t rcap, const ProblemDev* probs, int n_probs,
                float* grad_over, int which, int grid, cudaStream_t st) {
    // resident blocks only (the loop is persistent): occupancy x multiprocessors, at most `grid`;
    // the shared-memory size depends on the number of problems, so the occupancy is kept per count
    static int resident[MER_MAX_PROBLEMS + 1] = {0};
    static bool attr = false;
    const size_t smem = scatter_smem(n_probs);
    if (!attr) {
        cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scatter_smem(MER_MAX_PROBLEMS));
        attr = true;
    }
    if (!resident[n_probs]) {
        int occ = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_scatter, SC_THREADS, smem) != cudaSuccess || occ < 1)
            occ = 1;
        resident[n_probs] = occ * sms;
    }
    grid = grid < resident[n_probs] ? grid : resident[n_probs];
    MER_TIMED(KC_SCATTER, st,
              k_scatter<<<grid, SC_THREADS, smem, st>>>(cnt, rec, rcap, probs, n_probs, grad_over, which));
    return 1;
}

// Image loss (step a7) and its adjoint image, per problem: L2, L = 1/(3N) sum (I - T)^2 with
// dL/dI = 2 (I - T) / (3N), or MRSE, each term divided by (T^2 + 0.01), for the proportional
// image (parts & L2_PROP; the loss accumulated per problem in FP64) and the two images of the FD pair
// (parts & L2_FD). Pixels of all problems are enumerated through the prefix pix_pref.
__global__ void __launch_bounds__(256) k_l2(const ProblemDev* __restrict__ probs, const int64_t* __restrict__ pix_pref,
                                            int n_probs, int64_t total_pix, int parts, double* loss_acc) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nw = (total_pix + 31) & ~(int64_t)31;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nw; p += stride) {
        const bool valid = p < total_pix;
        int q = -1;
        double l = 0.0;
        if (valid) {
            q = find_entry(pix_pref, n_probs, p);
            const ProblemDev& P = probs[q];
            const int64_t lp = p - pix_pref[q];
            const float sc = 2.0f / (3.0f * (float)P.n_pix);
            const bool rel = P.loss_kind == MER_LOSS_MRSE;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int64_t k = lp * 3 + c;
                const float t = P.target[k];
                const float w = rel ? 1.0f / (t * t + 0.01f) : 1.0f;
                if (parts & L2_PROP) {
                    const float r = P.img[k] - t;
                    P.dimg[k] = sc * r * w;
                    l += (double)r * (double)r * (double)w;
                }
                if ((parts & L2_FD) && P.imgA) {
                    P.dimgA[k] = sc * (P.imgA[k] - t) * w;
                    P.dimgB[k] = sc * (P.imgB[k] - t) * w;
                }
            }
        }
        if (!(parts & L2_PROP)) continue;    // (uniform) the FD images carry no loss
        // warp reduce when the whole warp belongs to one problem, else per lane
        const int q0 = __shfl_sync(FULLM, q, 0);
        const bool same = __all_sync(FULLM, q == q0);
        if (same) {
            for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(FULLM, l, o);
            if ((threadIdx.x & 31) == 0 && q0 >= 0) atomicAdd(loss_acc + q0, l / (3.0 * (double)probs[q0].n_pix));
        } else if (valid) {
            atomicAdd(loss_acc + q, l / (3.0 * (double)probs[q].n_pix));
        }
    }
}

int run_l2(const ProblemDev* probs, const int64_t* pix_pref, int n_probs, int64_t total_pix, int parts,
           double* loss_acc, int grid, cudaStream_t st) {
    MER_TIMED(KC_L2, st, k_l2<<<grid, 256, 0, st>>>(probs, pix_pref, n_probs, total_pix, parts, loss_acc));
    return 1;
}

__global__ void k_philox(uint32_t k0, uint32_t k1, const uint4* __restrict__ ctr, int64_t n, uint4* out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = philox4x32_10(ctr[i], k0, k1);
}

int run_philox(uint32_t k0, uint32_t k1, const uint32_t* ctr, int64_t n, uint32_t* out, cudaStream_t st) {
    if (n <= 0) return 0;
    const int64_t blocks = (n + 255) / 256;
    k_philox<<<(unsigned)(blocks < 65535 ? blocks : 65535), 256, 0, st>>>(k0, k1, reinterpret_cast<const uint4*>(ctr), n,
                                                                        reinterpret_cast<uint4*>(out));
    return 1;
}

}  // namespace mer

namespace mer {

__global__ void k_fill(float* p, int64_t n, float v) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = v;
}

int run_fill(float* p, int64_t n, float v, cudaStream_t st) {
    if (n <= 0) return 0;
    const int64_t blocks = (n + 255) / 256;
    k_fill<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(p, n, v);
    return 1;
}

}  // namespace mer

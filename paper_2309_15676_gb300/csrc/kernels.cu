// Gradient scatter (step a10), image loss and adjoint images (step a7), Philox fill.
#include "kernels.cuh"
#include "wavefront.cuh"

namespace mer {

KernelTimer* g_timer = nullptr;

constexpr unsigned FULLM = 0xffffffffu;

// sum of v over the lanes of `peers` (lanes listed in vmask all call this); every lane gets
// the sum over its own peer group, in a fixed lane order
__device__ __forceinline__ float peer_sum(unsigned vmask, unsigned peers, float v, int maxg) {
    const unsigned lane = threadIdx.x & 31u;
    unsigned others = peers & ~(1u << lane);
    float acc = v;
    for (int i = 1; i < maxg; ++i) {
        const int src = others ? (__ffs(others) - 1) : (int)lane;
        const float x = __shfl_sync(vmask, v, src);
        if (others) {
            acc += x;
            others &= others - 1;
        }
    }
    return acc;
}

// Adds v[0..len) to the contiguous floats base[f0 ..) with the widest aligned vector
// reductions available (float4 where 16-byte aligned, float2 where 8-byte aligned, else
// scalar); base itself must be 16-byte aligned. Unrolled so that v stays in registers.
__device__ __forceinline__ void red_run(float* base, int64_t f0, const float (&v)[13], int len) {
    int s = 0;
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        if (k == s && k < len) {
            const int64_t f = f0 + k;
            const int rem = len - k;
            if ((f & 3) == 0 && rem >= 4) {
                atomicAdd(reinterpret_cast<float4*>(base + f), make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]));
                s += 4;
            } else if ((f & 1) == 0 && rem >= 2) {
                atomicAdd(reinterpret_cast<float2*>(base + f), make_float2(v[k], v[k + 1]));
                s += 2;
            } else {
                atomicAdd(base + f, v[k]);
                s += 1;
            }
        }
    }
}

template <int CC>
__device__ __forceinline__ void fill_rows(float (&v)[2][13], const float (&g)[MAXC], float w00, float w10, float w01,
                                          float w11) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const float wa = r ? w01 : w00, wb = r ? w11 : w10;
#pragma unroll
        for (int k = 0; k < 13; ++k) v[r][k] = 0.0f;
#pragma unroll
        for (int c = 0; c < CC; ++c) {
            v[r][c] = wa * g[c];
            v[r][CC + c] = wb * g[c];   // ignored beyond the run length when the taps merged
        }
    }
}

// per-problem fields the scatter needs, cached in shared memory
struct SProb {
    int C, W, H, pad;
    float* F;
    float* dF;
};

// One record: adds w_k g[c] to the four bilinear taps (clamp-to-edge) of the problem's HWC
// gradient texture. The two taps of a row are adjacent texels, i.e. one run of up to 2C
// contiguous floats, issued as aligned vector reductions (taps that clamp onto the same texel
// are merged first). Lanes holding the same footprint origin are merged with __match_any_sync
// and a segmented shuffle sum; only the group's first lane issues the reductions. Lanes whose
// record is absent or all-zero sit out; every shuffle runs over exactly the participating lanes.
__device__ __forceinline__ void scatter_one(bool valid, float4 a, float4 b, const SProb* sp, float* grad_over,
                                            int which) {
    const uint32_t pos = __float_as_uint(a.x);
    float g[MAXC] = {a.w, b.x, b.y, b.z, b.w};
    valid = valid && (g[0] != 0.0f || g[1] != 0.0f || g[2] != 0.0f || g[3] != 0.0f || g[4] != 0.0f);
    const unsigned vmask = __ballot_sync(FULLM, valid);
    if (!valid) return;
    const SProb P = sp[pos >> 24];
    const int C = P.C, W = P.W, H = P.H;
    const int x0 = (int)(pos & 0xfff) - 1, y0 = (int)((pos >> 12) & 0xfff) - 1;
    const float fx = a.y, fy = a.z;
    const int xa = max(x0, 0), xb = min(x0 + 1, W - 1), ya = max(y0, 0), yb = min(y0 + 1, H - 1);
    float w00 = (1.0f - fx) * (1.0f - fy), w10 = fx * (1.0f - fy), w01 = (1.0f - fx) * fy, w11 = fx * fy;
    const bool one_x = xa == xb, one_y = ya == yb;
    if (one_x) { w00 += w10; w10 = 0.0f; w01 += w11; w11 = 0.0f; }
    if (one_y) { w00 += w01; w10 += w11; w01 = 0.0f; w11 = 0.0f; }
    // row r holds [tap xa channels..., tap xb channels...] (compile-time indices per C)
    float v[2][13];
    if (C == 5) fill_rows<5>(v, g, w00, w10, w01, w11);
    else fill_rows<3>(v, g, w00, w10, w01, w11);
    const unsigned peers = __match_any_sync(vmask, pos);
    const int maxg = (int)__reduce_max_sync(vmask, (unsigned)__popc(peers));
    bool issue = true;
    if (maxg > 1) {
        // same pos => same problem and layout; every participating lane runs every shuffle
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int k = 0; k < 10; ++k) v[r][k] = peer_sum(vmask, peers, v[r][k], maxg);
        issue = (int)(threadIdx.x & 31u) == __ffs(peers) - 1;
    }
    if (issue) {
        float* base = grad_over ? grad_over : (which ? P.dF : P.F);
        const int len = (one_x ? 1 : 2) * C;
        red_run(base, ((int64_t)ya * W + xa) * C, v[0], len);
        if (!one_y) red_run(base, ((int64_t)yb * W + xa) * C, v[1], len);
    }
}

// Persistent grid-stride over records, one per lane (two 16-byte streaming loads each); the
// next record is loaded while the current one is scattered.
__global__ void __launch_bounds__(256) k_scatter(const uint32_t* __restrict__ cnt, const Record* __restrict__ rec,
                                                 int64_t rcap, const ProblemDev* __restrict__ probs, int n_probs,
                                                 float* grad_over, int which) {
    __shared__ SProb sp[MER_MAX_PROBLEMS];
    for (int t = threadIdx.x; t < n_probs; t += blockDim.x) {
        const ProblemDev& P = probs[t];
        sp[t] = SProb{P.tex_c, P.tex_w, P.tex_h, 0, P.F, P.dF};
    }
    __syncthreads();
    const int64_t n = min((int64_t)cnt[CNT_R], rcap);
    const int64_t nw = (n + 31) & ~(int64_t)31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float4* R = reinterpret_cast<const float4*>(rec);
    const int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float4 a = make_float4(0, 0, 0, 0), b = a;
    if (start < n) { a = __ldcs(R + 2 * start); b = __ldcs(R + 2 * start + 1); }
    for (int64_t i = start; i < nw; i += stride) {
        const int64_t j = i + stride;
        float4 na = make_float4(0, 0, 0, 0), nb = na;
        if (j < n) { na = __ldcs(R + 2 * j); nb = __ldcs(R + 2 * j + 1); }
        scatter_one(i < n, a, b, sp, grad_over, which);
        a = na;
        b = nb;
    }
}

int run_scatter(const uint32_t* cnt, const Record* rec, int64_t rcap, const ProblemDev* probs, int n_probs,
                float* grad_over, int which, int grid, cudaStream_t st) {
    // resident blocks only (the loop is persistent): occupancy x multiprocessors, at most `grid`
    static int resident = 0;
    if (!resident) {
        int occ = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_scatter, 256, 0) != cudaSuccess || occ < 1) occ = 1;
        resident = occ * sms;
    }
    grid = grid < resident ? grid : resident;
    MER_TIMED(KC_SCATTER, st, k_scatter<<<grid, 256, 0, st>>>(cnt, rec, rcap, probs, n_probs, grad_over, which));
    return 1;
}

// L2 loss L = 1/(3N) sum (I - T)^2 and its adjoint image dL/dI = 2 (I - T) / (3N), for the
// proportional image (loss accumulated per problem in FP64) and, with_fd, the two images of the
// FD pair. Pixels of all problems are enumerated through the prefix pix_pref.
__global__ void __launch_bounds__(256) k_l2(const ProblemDev* __restrict__ probs, const int64_t* __restrict__ pix_pref,
                                            int n_probs, int64_t total_pix, int with_fd, double* loss_acc) {
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
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int64_t k = lp * 3 + c;
                const float t = P.target[k];
                const float r = P.img[k] - t;
                P.dimg[k] = sc * r;
                l += (double)r * (double)r;
                if (with_fd && P.imgA) {
                    P.dimgA[k] = sc * (P.imgA[k] - t);
                    P.dimgB[k] = sc * (P.imgB[k] - t);
                }
            }
        }
        // warp reduce when the whole warp belongs to one problem, else per lane
        const int q0 = __shfl_sync(FULLM, q, 0);
        const bool same = __all_sync(FULLM, q == q0);
        if (same) {
            for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(FULLM, l, o);
            if ((threadIdx.x & 31) == 0 && q0 >= 0) atomicAdd(loss_acc + q0, l);
        } else if (valid) {
            atomicAdd(loss_acc + q, l);
        }
    }
}

int run_l2(const ProblemDev* probs, const int64_t* pix_pref, int n_probs, int64_t total_pix, int with_fd,
           double* loss_acc, int grid, cudaStream_t st) {
    MER_TIMED(KC_L2, st, k_l2<<<grid, 256, 0, st>>>(probs, pix_pref, n_probs, total_pix, with_fd, loss_acc));
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

// Fused per-parameter update (step a11): one HBM pass over every parameter of every
// problem. META mode (Sec. 4, Sec. 5 and the appendix pseudocode):
//   m2f <- m2f + cF (F^2 - m2f)                                  Var[<F_i>]  (Eq. varest, start-up corrected)
//   if FD available: m2d <- m2d + cD ((dF/||dpi||)^2 - m2d)      Var[<dF_i>]_D (Sec. 4.2)
//                    vard = m2d ||dpi||^2                         (Eq. vardiff)
//   mean += dF ; var += vard                                      (Eq. recurrent_meta, varmeta: carried terms)
//   a = m2f / (m2f + var + eps_alpha) ; a = min(a, 1/(2 - a_prev))  (Eqs. alpha, alpha_clip_2)
//   mean = a mean + (1-a) F ; var = a^2 var + (1-a)^2 m2f
//   pi' = clamp(pi - lr mean / (sqrt(var) + eps))                 (update rule of Sec. 5)
// ADAM mode (Sec. 5, Eqs. adam_moment, adam_ema_startup, adam_step) keeps m in `mean` and v
// in `m2f`. Both modes write pi' into the other parameter slot, optionally clear F and dF, and
// reduce ||pi' - pi||^2 per problem deterministically (per-block partials, fixed-order sum).
// META segments with MER_META_* variant flags take a scalar path (meta_elem_var) through the
// same blocks; the method as stated keeps the float4 path.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "kernels.cuh"
#include "update.cuh"

namespace mer {

constexpr int UPD_THREADS = 256;
constexpr int UPD_VEC_PER_THREAD = 4;                       // float4 per thread per block
constexpr int64_t UPD_CHUNK = (int64_t)UPD_THREADS * UPD_VEC_PER_THREAD * 4;   // params per block

int64_t update_blocks_for(int64_t n) { return (n + UPD_CHUNK - 1) / UPD_CHUNK; }

const char* hyper_problem(const mer_hyper& h) {
    auto decay = [](float b) { return b >= 0.0f && b < 1.0f; };
    auto nonneg = [](float x) { return x >= 0.0f && x < INFINITY; };
    if (h.mode != MER_MODE_META && h.mode != MER_MODE_ADAM) return "unknown optimiser mode";
    if (h.flags & ~127) return "unknown MER_META_* flag bits";
    if (!decay(h.beta_f) || !decay(h.beta_d) || !decay(h.beta1) || !decay(h.beta2))
        return "EMA decays must lie in [0, 1)";
    if (!nonneg(h.lr) || !nonneg(h.eps) || !nonneg(h.eps_alpha) || !nonneg(h.precond_lambda))
        return "lr, eps, eps_alpha and precond_lambda must be finite and >= 0";
    return nullptr;
}

using Coef = UpdCoef;

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

// one element of META mode; returns the applied step
__device__ __forceinline__ float meta_elem(const mer_hyper& h, const Coef& k, float p, float F, float dF, float& m2f,
                                           float& m2d, float& mean, float& var, float& ap, float lo, float hi,
                                           float& pnew) {
    m2f = m2f + k.cF * (F * F - m2f);
    float vard = 0.0f, dfu = 0.0f;
    if (k.stepD) {
        const float x = dF * k.inv_norm;
        m2d = m2d + k.cD * (x * x - m2d);
        vard = m2d * k.norm2;
        dfu = dF;
    }
    mean = mean + dfu;
    var = var + vard;
    float a = m2f / (m2f + var + h.eps_alpha);
    a = fminf(a, 1.0f / (2.0f - ap));
    ap = a;
    const float b = 1.0f - a;
    mean = a * mean + b * F;
    var = a * a * var + b * b * m2f;
    const float step = -h.lr * mean / (sqrtf(var) + h.eps);
    pnew = clampf(p + step, lo, hi);
    return pnew - p;
}

__device__ __forceinline__ float adam_elem(const mer_hyper& h, const Coef& k, float p, float F, float& v, float& m,
                                           float lo, float hi, float& pnew) {
    m = h.beta1 * m + (1.0f - h.beta1) * F;
    v = h.beta2 * v + (1.0f - h.beta2) * F * F;
    const float step = -h.lr * (m * k.c1) / (sqrtf(v * k.c2) + h.eps);
    pnew = clampf(p + step, lo, hi);
    return pnew - p;
}

// one element of META mode with variant flags (see the header); pprev = pi_{i-1} (PER_ELEMENT);
// every state array is read and written through the segment at index e; returns the applied step
__device__ __forceinline__ float meta_elem_var(const UpdSeg& S, const Coef& k, int64_t e, float p, float pprev,
                                               float lo, float hi, float& pnew) {
    const mer_hyper& h = S.hyper;
    const int fl = h.flags;
    const float F = S.F[e];
    const float xF = (fl & MER_META_UNCORRELATED) ? S.Fv[e] : F;
    float m2f = S.m2f[e] + k.cF * (xF * xF - S.m2f[e]);
    S.m2f[e] = m2f;
    float varf = m2f;
    if (fl & MER_META_CENTRED) {
        const float mu = S.mu_f[e] + k.cF * (xF - S.mu_f[e]);
        S.mu_f[e] = mu;
        varf = fmaxf(m2f - mu * mu, 0.0f);
    }
    float mean = S.mean[e], var = S.var[e];
    if (k.stepD) {
        const float dF = S.dF[e];
        const float xD = (fl & MER_META_UNCORRELATED) ? S.dFv[e] : dF;
        float d2, x;
        bool live = true;
        if (fl & MER_META_PER_ELEMENT) {
            const float d = p - pprev;
            d2 = d * d;
            live = d2 > 0.0f;
            x = live ? xD / fabsf(d) : 0.0f;
        } else {
            d2 = k.norm2;
            x = xD * k.inv_norm;
        }
        float m2d = S.m2d[e];
        if (live) {
            m2d = m2d + k.cD * (x * x - m2d);
            S.m2d[e] = m2d;
        }
        float vdd = m2d;
        if (fl & MER_META_CENTRED) {
            float mu = S.mu_d[e];
            if (live) {
                mu = mu + k.cD * (x - mu);
                S.mu_d[e] = mu;
            }
            vdd = fmaxf(m2d - mu * mu, 0.0f);
        }
        mean = mean + dF;
        var = var + vdd * d2;
    }
    float a = varf / (varf + var + h.eps_alpha);
    if (!(fl & MER_META_NO_CLIP)) a = fminf(a, 1.0f / (2.0f - S.ap[e]));
    S.ap[e] = a;
    const float b = 1.0f - a;
    mean = a * mean + b * F;
    var = a * a * var + b * b * varf;
    S.mean[e] = mean;
    S.var[e] = var;
    float step;
    if (fl & MER_META_NAIVE_ADAM) {
        const float m = h.beta1 * S.am[e] + (1.0f - h.beta1) * mean;
        const float v = h.beta2 * S.av[e] + (1.0f - h.beta2) * mean * mean;
        S.am[e] = m;
        S.av[e] = v;
        step = -h.lr * (m * k.c1) / (sqrtf(v * k.c2) + h.eps);
    } else {
        step = -h.lr * mean / (sqrtf(var) + h.eps);
    }
    pnew = clampf(p + step, lo, hi);
    return pnew - p;
}

#define F4(ptr, i) (reinterpret_cast<float4*>(ptr)[i])
#define CF4(ptr, i) (reinterpret_cast<const float4*>(ptr)[i])

// one float4 group of every state array
struct Grp {
    float4 p, F, dF, m2f, m2d, mean, var, ap;
};

__device__ __forceinline__ void load_grp(Grp& g, const UpdSeg& S, const float* pin, bool meta, int64_t v) {
    g.p = CF4(pin, v);
    g.F = CF4(S.F, v);
    g.m2f = CF4(S.m2f, v);
    g.mean = CF4(S.mean, v);
    if (meta) {
        g.dF = CF4(S.dF, v);
        g.m2d = CF4(S.m2d, v);
        g.var = CF4(S.var, v);
        g.ap = CF4(S.ap, v);
    } else {
        g.dF = g.m2d = g.var = g.ap = make_float4(0, 0, 0, 0);
    }
}

// updates one group in registers, stores it, returns the sum of squared applied steps
__device__ __forceinline__ float proc_grp(Grp& g, const UpdSeg& S, const Coef& k, float* pout, bool meta, int64_t v) {
    float pv[4] = {g.p.x, g.p.y, g.p.z, g.p.w}, Fv[4] = {g.F.x, g.F.y, g.F.z, g.F.w};
    float dFv[4] = {g.dF.x, g.dF.y, g.dF.z, g.dF.w}, m2fv[4] = {g.m2f.x, g.m2f.y, g.m2f.z, g.m2f.w};
    float m2dv[4] = {g.m2d.x, g.m2d.y, g.m2d.z, g.m2d.w}, meanv[4] = {g.mean.x, g.mean.y, g.mean.z, g.mean.w};
    float varv[4] = {g.var.x, g.var.y, g.var.z, g.var.w}, apv[4] = {g.ap.x, g.ap.y, g.ap.z, g.ap.w};
    float out[4];
    float acc = 0.0f;
    const int C = S.C;
    // channel of the group's first element (32-bit modulo while the index fits in 32 bits)
    const int c0 = (v * 4 < ((int64_t)1 << 32)) ? (int)((uint32_t)(v * 4) % (uint32_t)C) : (int)((v * 4) % C);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        int c = c0 + l;
        while (c >= C) c -= C;   // C = 1 wraps up to three times
        float st;
        if (meta)
            st = meta_elem(S.hyper, k, pv[l], Fv[l], dFv[l], m2fv[l], m2dv[l], meanv[l], varv[l], apv[l], S.lo[c],
                           S.hi[c], out[l]);
        else
            st = adam_elem(S.hyper, k, pv[l], Fv[l], m2fv[l], meanv[l], S.lo[c], S.hi[c], out[l]);
        acc += st * st;
    }
    F4(pout, v) = make_float4(out[0], out[1], out[2], out[3]);
    F4(S.m2f, v) = make_float4(m2fv[0], m2fv[1], m2fv[2], m2fv[3]);
    F4(S.mean, v) = make_float4(meanv[0], meanv[1], meanv[2], meanv[3]);
    if (meta) {
        if (k.stepD) F4(S.m2d, v) = make_float4(m2dv[0], m2dv[1], m2dv[2], m2dv[3]);
        F4(S.var, v) = make_float4(varv[0], varv[1], varv[2], varv[3]);
        F4(S.ap, v) = make_float4(apv[0], apv[1], apv[2], apv[3]);
    }
    if (S.zero_grads) {
        F4(S.F, v) = make_float4(0, 0, 0, 0);
        if (meta) F4(S.dF, v) = make_float4(0, 0, 0, 0);
    }
    return acc;
}

// processes one block's chunk of one segment; returns this thread's sum of squared steps
// (one float4 group of all state arrays per step keeps registers low and occupancy high)
__device__ __forceinline__ float update_block(const UpdSeg& S, const Coef& k, int cur, int64_t local_block) {
    const float* pin = cur ? S.pB : S.pA;
    float* pout = cur ? S.pA : S.pB;
    const bool meta = S.hyper.mode == MER_MODE_META;
    float acc = 0.0f;
    if (meta && S.hyper.flags) {
        // variants: one element per thread and step over the block's chunk (pout still holds
        // pi_{i-1} when its element is read)
        const int64_t e0 = local_block * UPD_CHUNK;
        for (int it = 0; it < UPD_VEC_PER_THREAD * 4; ++it) {
            const int64_t e = e0 + (int64_t)it * UPD_THREADS + threadIdx.x;
            if (e >= S.n) break;
            const int c = (int)((uint64_t)e % (uint64_t)S.C);
            float pnew;
            const float st = meta_elem_var(S, k, e, pin[e], pout[e], S.lo[c], S.hi[c], pnew);
            pout[e] = pnew;
            if (S.zero_grads) {
                S.F[e] = 0.0f;
                S.dF[e] = 0.0f;
            }
            acc += st * st;
        }
        return acc;
    }
    const int64_t n4 = S.n >> 2;          // float4 count (the tail below handles n % 4)
    const int64_t v0 = local_block * (UPD_CHUNK >> 2);
#pragma unroll
    for (int it = 0; it < UPD_VEC_PER_THREAD; ++it) {
        const int64_t v = v0 + (int64_t)it * UPD_THREADS + threadIdx.x;
        if (v >= n4) break;
        Grp g;
        load_grp(g, S, pin, meta, v);
        acc += proc_grp(g, S, k, pout, meta, v);
    }
    // scalar tail (n not a multiple of 4): first block, first threads
    if (local_block == 0 && threadIdx.x < (int)(S.n & 3)) {
        const int64_t e = (n4 << 2) + threadIdx.x;
        const int c = (int)(e % S.C);
        float m2f = S.m2f[e], mean = S.mean[e], pnew, st;
        if (meta) {
            float m2d = S.m2d[e], var = S.var[e], ap = S.ap[e];
            st = meta_elem(S.hyper, k, pin[e], S.F[e], S.dF[e], m2f, m2d, mean, var, ap, S.lo[c], S.hi[c], pnew);
            if (k.stepD) S.m2d[e] = m2d;
            S.var[e] = var;
            S.ap[e] = ap;
        } else {
            st = adam_elem(S.hyper, k, pin[e], S.F[e], m2f, mean, S.lo[c], S.hi[c], pnew);
        }
        pout[e] = pnew;
        S.m2f[e] = m2f;
        S.mean[e] = mean;
        if (S.zero_grads) {
            S.F[e] = 0.0f;
            if (meta) S.dF[e] = 0.0f;
        }
        acc += st * st;
    }
    return acc;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[UPD_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < UPD_THREADS / 32; ++i) s += red[i];
    return s;
}

// context form: segment table on the device, per-problem scalars in ProbState
__global__ void __launch_bounds__(UPD_THREADS) k_update_ctx(const UpdSeg* segs, const int64_t* blk_off, int n_segs,
                                                            ProbState* ps, double* partials) {
    __shared__ Coef sk;
    __shared__ int s_seg, s_cur;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_segs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (blk_off[mid] <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        s_seg = lo;
        const UpdSeg& S = segs[lo];
        sk = ps[S.prob].coef;
        s_cur = ps[S.prob].cur;
    }
    __syncthreads();
    const UpdSeg& S = segs[s_seg];
    const float acc = update_block(S, sk, s_cur, (int64_t)blockIdx.x - blk_off[s_seg]);
    const double tot = block_sum((double)acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// per segment: fixed-order sum of its partials, then advance the problem's scalars
__global__ void __launch_bounds__(UPD_THREADS) k_update_finalize_ctx(const UpdSeg* segs, const int64_t* blk_off,
                                                                     ProbState* ps, const double* partials) {
    const int sgi = blockIdx.x;
    const UpdSeg& S = segs[sgi];
    double v = 0.0;
    for (int64_t i = blk_off[sgi] + threadIdx.x; i < blk_off[sgi + 1]; i += UPD_THREADS) v += partials[i];
    const double tot = block_sum(v);
    if (threadIdx.x == 0) {
        ProbState& st = ps[S.prob];
        if (S.hyper.mode == MER_MODE_META) {
            const bool stepD = st.iteration >= 1 && st.dpi_norm2 > 0.0;
            st.count_f += 1;
            st.count_d += stepD ? 1 : 0;
        } else {
            st.count_f += 1;
        }
        st.iteration += 1;
        st.cur ^= 1;
        st.dpi_norm2 = tot;
        st.coef = update_coef(S.hyper, st.iteration, st.count_f, st.count_d, tot);
    }
}

// standalone form: one segment passed by value, scalars from the caller
__global__ void __launch_bounds__(UPD_THREADS) k_update_raw(UpdSeg S, Coef k, double* partials) {
    const float acc = update_block(S, k, 0, blockIdx.x);
    const double tot = block_sum((double)acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(UPD_THREADS) k_update_finalize_raw(const double* partials, int64_t nb,
                                                                     double* out) {
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < nb; i += UPD_THREADS) v += partials[i];
    const double tot = block_sum(v);
    if (threadIdx.x == 0) *out = tot;
}

cudaError_t launch_update_ctx(const UpdSeg* segs_dev, const int64_t* blk_off_dev, int n_segs, int64_t total_blocks,
                              ProbState* ps, double* partials, cudaStream_t st) {
    if (total_blocks <= 0) return cudaSuccess;
    MER_TIMED(KC_UPDATE, st,
              k_update_ctx<<<(unsigned)total_blocks, UPD_THREADS, 0, st>>>(segs_dev, blk_off_dev, n_segs, ps, partials));
    MER_TIMED(KC_UPDATE_FIN, st, k_update_finalize_ctx<<<n_segs, UPD_THREADS, 0, st>>>(segs_dev, blk_off_dev, ps, partials));
    return cudaGetLastError();
}

cudaError_t launch_update_raw(const UpdSeg& S, int iteration, int count_f, int count_d, double n2, double* partials,
                              int64_t nblocks, double* out, cudaStream_t st) {
    if (g_timer) g_timer->add_units(KC_UPDATE, S.n);
    if (nblocks > 0)
        MER_TIMED(KC_UPDATE, st,
                  k_update_raw<<<(unsigned)nblocks, UPD_THREADS, 0, st>>>(
                      S, update_coef(S.hyper, iteration, count_f, count_d, n2), partials));
    MER_TIMED(KC_UPDATE_FIN, st, k_update_finalize_raw<<<1, UPD_THREADS, 0, st>>>(partials, nblocks, out));
    return cudaGetLastError();
}

__global__ void __launch_bounds__(UPD_THREADS) k_force_step(const float* __restrict__ pnew,
                                                            const float* __restrict__ pold, int64_t n, ProbState* ps,
                                                            mer_hyper h) {
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += UPD_THREADS) {
        const double d = (double)pnew[i] - (double)pold[i];
        v += d * d;
    }
    const double tot = block_sum(v);
    if (threadIdx.x == 0) {
        ps->dpi_norm2 = tot;
        ps->coef = update_coef(h, ps->iteration, ps->count_f, ps->count_d, tot);
    }
}

cudaError_t launch_force_step(const float* pnew, const float* pold, int64_t n, ProbState* ps, const mer_hyper& h,
                              cudaStream_t st) {
    k_force_step<<<1, UPD_THREADS, 0, st>>>(pnew, pold, n, ps, h);
    return cudaGetLastError();
}

const char* raw_update_seg(const mer_hyper* hyper, int64_t n, int32_t C, const float* lo, const float* hi,
                           const mer_update_arrays* arrays, int32_t zero_grads, const double* out, UpdSeg* S) {
    if (!hyper || !arrays || n < 0 || C < 1 || C > 8 || !lo || !hi || !out)
        return "bad arguments to the standalone update";
    if (const char* why = hyper_problem(*hyper)) return why;
    const mer_update_arrays& A = *arrays;
    const bool meta = hyper->mode == MER_MODE_META;
    const int fl = meta ? hyper->flags : 0;
    if (n > 0 && (!A.pi || !A.pi_next || !A.F || !A.m2f || !A.mean ||
                  (meta && (!A.dF || !A.m2d || !A.var || !A.alpha_prev))))
        return "missing arrays in the standalone update";
    if (n > 0 && (((fl & MER_META_CENTRED) && (!A.mu_f || !A.mu_d)) ||
                  ((fl & MER_META_NAIVE_ADAM) && (!A.adam_m || !A.adam_v)) ||
                  ((fl & MER_META_UNCORRELATED) && (!A.F_var || !A.dF_var))))
        return "the update's flags need variant arrays that are missing (mer_meta_step_raw_ex takes them)";
    const void* ptrs[] = {A.pi, A.pi_next, A.F, A.dF, A.m2f, A.m2d, A.mean, A.var, A.alpha_prev,
                          A.mu_f, A.mu_d, A.adam_m, A.adam_v, A.F_var, A.dF_var};
    for (const void* q : ptrs)
        if (q && ((uintptr_t)q & 15u)) return "arrays must be 16-byte aligned";
    if (A.pi == A.pi_next && n > 0) return "pi_next may not alias pi";
    memset(S, 0, sizeof *S);
    S->pA = const_cast<float*>(A.pi);
    S->pB = A.pi_next;
    S->F = A.F; S->dF = A.dF; S->m2f = A.m2f; S->m2d = A.m2d; S->mean = A.mean; S->var = A.var; S->ap = A.alpha_prev;
    if (fl & MER_META_CENTRED) { S->mu_f = A.mu_f; S->mu_d = A.mu_d; }
    if (fl & MER_META_NAIVE_ADAM) { S->am = A.adam_m; S->av = A.adam_v; }
    if (fl & MER_META_UNCORRELATED) { S->Fv = A.F_var; S->dFv = A.dF_var; }
    S->n = n;
    S->C = C;
    S->zero_grads = zero_grads;
    for (int k = 0; k < C; ++k) {
        S->lo[k] = lo[k];
        S->hi[k] = hi[k];
    }
    S->hyper = *hyper;
    return nullptr;
}

// ---------------------------------------------------------------------------------------
// Allocation-free form of the standalone update. Its only scratch is the per-block partial
// sums of ||pi' - pi||^2; here they live in a fixed file-scope device array instead of a
// buffer the library allocates. Every GPU that loads the library holds this array (512 KiB)
// until the process exits.
// ---------------------------------------------------------------------------------------
constexpr int64_t NOALLOC_MAX_BLOCKS = 65536;   // -> at most 65536 * UPD_CHUNK parameters
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS];

constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mu;
static double* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {nullptr};

int64_t noalloc_max_params() { return NOALLOC_MAX_BLOCKS * UPD_CHUNK; }

}  // namespace mer

extern "C" mer_status mer_meta_step_raw_noalloc(const mer_hyper* hyper, int64_t n, int32_t C, const float* lo,
                                                const float* hi, const float* pi, float* pi_next, float* F,
                                                float* dF, float* m2f, float* m2d, float* mean, float* var,
                                                float* alpha_prev, int32_t iteration, int32_t count_f,
                                                int32_t count_d, double dpi_norm2, int32_t zero_grads,
                                                double* dpi_norm2_out, void* cuda_stream) {
    using namespace mer;
    mer_update_arrays A;
    memset(&A, 0, sizeof A);
    A.pi = pi; A.pi_next = pi_next; A.F = F; A.dF = dF; A.m2f = m2f; A.m2d = m2d; A.mean = mean; A.var = var;
    A.alpha_prev = alpha_prev;
    UpdSeg S;
    if (const char* why = raw_update_seg(hyper, n, C, lo, hi, &A, zero_grads, dpi_norm2_out, &S))
        return mer_internal_fail(MER_ERR_INVALID_ARG, why);
    const int64_t nb = update_blocks_for(n);
    if (nb > NOALLOC_MAX_BLOCKS)
        return mer_internal_fail(MER_ERR_INVALID_ARG,
                                 "mer_meta_step_raw_noalloc: n exceeds the fixed scratch (at most 268435456 parameters)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return mer_internal_fail(MER_ERR_CUDA, "mer_meta_step_raw_noalloc: no usable current device");
    double* scratch = nullptr;
    {
        // once per device, with that device current: the array's device address
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            double* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_partials);
            if (e != cudaSuccess || !p)
                return mer_internal_fail(MER_ERR_CUDA, "mer_meta_step_raw_noalloc: cudaGetSymbolAddress failed");
            g_noalloc_addr[dev] = p;
        }
        scratch = g_noalloc_addr[dev];
    }
    // every block writes its own partial before the finalize kernel reads it, so nothing in the
    // shared array has to start at zero
    const cudaError_t e = launch_update_raw(S, iteration, count_f, count_d, dpi_norm2, scratch, nb, dpi_norm2_out,
                                            (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return mer_internal_fail(MER_ERR_CUDA, cudaGetErrorString(e));
    return MER_OK;
}

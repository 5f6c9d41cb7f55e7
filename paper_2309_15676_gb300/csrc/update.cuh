// Fused update: segment description and launchers.
#pragma once

#include "mer_internal.cuh"

namespace mer {

// one problem's parameter-shaped arrays (device), n elements, channel = index % C
struct UpdSeg {
    float* pA;           // parameter slot 0
    float* pB;           // parameter slot 1 (pi' goes to the slot that is not current)
    float* F;
    float* dF;
    float* m2f;          // META: Var[<F>] Moment2;  ADAM: v
    float* m2d;          // META: Var[<dF>]_D Moment2
    float* mean;         // META: <F>_M;            ADAM: m
    float* var;          // META: Var[<F>_M]
    float* ap;           // META: alpha_{i-1}
    // variant state (MER_META_* flags; NULL when the flag is off)
    float* mu_f;         // CENTRED: EMA of the Var[<F>] samples
    float* mu_d;         // CENTRED: EMA of the Var[<dF>]_D samples
    float* am;           // NAIVE_ADAM: Adam's m over <F>_M
    float* av;           // NAIVE_ADAM: Adam's v over <F>_M
    const float* Fv;     // UNCORRELATED: independent samples for Var[<F>]
    const float* dFv;    // UNCORRELATED: independent samples for Var[<dF>]_D
    int64_t n;
    int32_t C;
    int32_t prob;        // problem index (context form)
    int32_t zero_grads;
    float lo[8], hi[8];
    mer_hyper hyper;
};

// beta^n for an integer n >= 0 by binary exponentiation (about 2 log2 n double multiplies, a few
// ulp): every exponent of the update's start-up and bias corrections is a step count, and the
// general pow is slow in the one FP64 thread that computes the coefficients each iteration
__host__ __device__ inline double ipow(double beta, long long n) {
    double r = 1.0, b = beta;
    while (n > 0) {
        if (n & 1) r *= b;
        b *= b;
        n >>= 1;
    }
    return r;
}

// prod_{j<=k} max(beta, j/(j+1)) in closed form: beta^min(k+1, K) * (k >= K ? K/(k+1) : 1),
// K the first j with j/(j+1) > beta (MER_META_GROWING_BETA)
__host__ __device__ inline double growing_prod(double beta, int k) {
    long long K = (long long)floor(beta / (1.0 - beta));
    if (K < 0) K = 0;
    while (K > 0 && (double)(K - 1) / (double)K > beta) --K;
    while ((double)K / (double)(K + 1) <= beta) ++K;
    const long long reps = (long long)k + 1 < K ? (long long)k + 1 : K;
    double p = ipow(beta, reps);
    if ((long long)k >= K) p *= (double)K / (double)(k + 1);
    return p;
}

// The update's scalars for iteration `iteration` with Moment2 counts count_f, count_d before the
// step and ||dpi_i||^2 = n2 (double precision, once per problem; the per-element kernel reads them)
__host__ __device__ inline UpdCoef update_coef(const mer_hyper& h, int iteration, int count_f, int count_d,
                                               double n2) {
    UpdCoef k;
    k.pad = 0;
    const long long t = (long long)iteration + 1;
    k.c1 = (float)(1.0 / (1.0 - ipow((double)h.beta1, t)));   // Adam (and NAIVE_ADAM) bias corrections
    k.c2 = (float)(1.0 / (1.0 - ipow((double)h.beta2, t)));
    if (h.mode == MER_MODE_META) {
        const double bf = (double)h.beta_f, bd = (double)h.beta_d;
        if (h.flags & MER_META_GROWING_BETA) {
            const double b = fmax(bf, (double)count_f / (double)(count_f + 1));
            k.cF = (float)((1.0 - b) / (1.0 - growing_prod(bf, count_f)));
        } else {
            k.cF = (float)((1.0 - bf) / (1.0 - ipow(bf, (long long)count_f + 1)));
        }
        k.stepD = (iteration >= 1 && n2 > 0.0) ? 1 : 0;
        k.cD = k.stepD ? (float)((1.0 - bd) / (1.0 - ipow(bd, (long long)count_d + 1))) : 0.0f;
        k.norm2 = (float)n2;
        k.inv_norm = k.stepD ? (float)(1.0 / sqrt(n2)) : 0.0f;
    } else {
        k.cF = k.cD = k.norm2 = k.inv_norm = 0.0f;
        k.stepD = 0;
    }
    return k;
}

int64_t update_blocks_for(int64_t n);
// records a context-free error message (thread-local) and returns code
int mer_internal_fail(int code, const char* msg);
// why a hyper-parameter set cannot run (a mode other than META / ADAM, unknown flag bits, a decay
// outside [0, 1) whose start-up correction would divide by zero, a negative or non-finite rate,
// epsilon or preconditioning weight), or nullptr
const char* hyper_problem(const mer_hyper& h);
cudaError_t launch_update_ctx(const UpdSeg* segs_dev, const int64_t* blk_off_dev, int n_segs, int64_t total_blocks,
                              ProbState* ps, double* partials, cudaStream_t st);
// ||pnew - pold||^2 over n parameters (one block, fixed order) into ps->dpi_norm2, and the next
// update's coefficients for it
cudaError_t launch_force_step(const float* pnew, const float* pold, int64_t n, ProbState* ps, const mer_hyper& h,
                              cudaStream_t st);
cudaError_t launch_update_raw(const UpdSeg& S, int iteration, int count_f, int count_d, double n2, double* partials,
                              int64_t nblocks, double* out, cudaStream_t st);   // coefficients computed on the host
// The argument checks of the standalone update (mer_meta_step_raw, _ex and _noalloc share them):
// fills *S from the arrays and returns nullptr, or returns why the call cannot run (every such
// case is MER_ERR_INVALID_ARG).
const char* raw_update_seg(const mer_hyper* hyper, int64_t n, int32_t C, const float* lo, const float* hi,
                           const mer_update_arrays* arrays, int32_t zero_grads, const double* out, UpdSeg* S);

}  // namespace mer

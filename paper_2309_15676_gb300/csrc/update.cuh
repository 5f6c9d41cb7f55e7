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

int64_t update_blocks_for(int64_t n);
// records a context-free error message (thread-local) and returns code
int mer_internal_fail(int code, const char* msg);
cudaError_t launch_update_ctx(const UpdSeg* segs_dev, const int64_t* blk_off_dev, int n_segs, int64_t total_blocks,
                              ProbState* ps, double* partials, cudaStream_t st);
cudaError_t launch_update_raw(const UpdSeg& S, int iteration, int count_f, int count_d, double n2, double* partials,
                              int64_t nblocks, double* out, cudaStream_t st);

}  // namespace mer

// Launchers of the scatter, loss and Philox kernels, and of the wavefront passes.
#pragma once

#include "mer_internal.cuh"

namespace mer {

// launch classes for the optional per-kernel event timing
enum KernelClass {
    KC_TRACE1_PRIMAL, KC_TRACE1_REPLAY, KC_SHADE1_PRIMAL, KC_SHADE1_REPLAY,
    KC_TRACE2_PRIMAL, KC_TRACE2_REPLAY, KC_SHADE2_PRIMAL, KC_SHADE2_REPLAY,
    KC_RESOLVE, KC_L2, KC_ZERO, KC_SCATTER, KC_PRECOND, KC_UPDATE, KC_UPDATE_FIN, KC_COUNT
};

// records CUDA events around launches when installed (diagnostic mode, one thread)
struct KernelTimer {
    virtual void before(int cls, cudaStream_t st) = 0;
    virtual void after(int cls, cudaStream_t st) = 0;
    virtual void add_units(int cls, int64_t n) = 0;
    virtual ~KernelTimer() {}
};
extern KernelTimer* g_timer;

#define MER_TIMED(cls, st, ...)                       \
    do {                                              \
        if (g_timer) g_timer->before((cls), (st));    \
        __VA_ARGS__;                                  \
        if (g_timer) g_timer->after((cls), (st));     \
    } while (0)

struct PassArgs;
struct Record;
struct LaunchShape {
    int block;        // threads per block of the wavefront kernels (<= 256)
    int per_sm;       // cap on resident blocks per SM of the persistent grids (0 = occupancy)
    int smem_nodes;   // BVH nodes staged in shared memory
    int sms;          // multiprocessors of the device
    int refill;       // traversal: idle lanes of a warp that trigger fetching new rays (1..32)
};

int run_pass(const PassArgs& A, int nb, int mode, int max_depth, const LaunchShape& L, cudaStream_t st);
int run_resolve(const PassArgs& A, int nb, float* img0, float* img1, int accumulate, int grid, cudaStream_t st);
int run_samples_out(const PassArgs& A, float* out, int grid, cudaStream_t st);
cudaError_t set_trace_smem_limits(int max_nodes);

// grad_over != nullptr: single-problem output; else each record's problem's F (which = 0) or dF (which = 1)
// Bounded-wait self-test: a barrier nothing completes, waited on with limit_ns; device status
// (MER_OK / MER_ERR_TIMEOUT) and the wait's duration
int run_wait_selftest(uint64_t limit_ns, int32_t* status, uint64_t* waited_ns, cudaStream_t st);
// Clears gradient texture `which` (0 F, 1 dF, 2 F_var, 3 dF_var) of every problem that has one.
int run_zero_grads(const ProblemDev* probs, int n_probs, int which, int grid, cudaStream_t st);
int run_scatter(uint32_t* cnt, const Record* rec, int64_t rcap, const ProblemDev* probs, int n_probs,
                float* grad_over, int which, int grid, cudaStream_t st);
// per-problem L2 loss and adjoint images of all problems (pix_pref: prefix of n_pix over problems)
// parts of the image loss kernel: the proportional image's adjoint image and loss, the FD pair's
// two adjoint images
constexpr int L2_PROP = 1, L2_FD = 2;
int run_l2(const ProblemDev* probs, const int64_t* pix_pref, int n_probs, int64_t total_pix, int parts,
           double* loss_acc, int grid, cudaStream_t st);
int run_philox(uint32_t k0, uint32_t k1, const uint32_t* ctr, int64_t n, uint32_t* out, cudaStream_t st);

}  // namespace mer

namespace mer {
int run_fill(float* p, int64_t n, float v, cudaStream_t st);
}  // namespace mer

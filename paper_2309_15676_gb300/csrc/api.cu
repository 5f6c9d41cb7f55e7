// C ABI of the library (mer.h): context, scene upload, pass orchestration, CUDA-graph
// capture of whole iterations, the standalone update and checkpointing.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "bvh.h"
#include "kernels.cuh"
#include "precond.cuh"
#include "update.cuh"
#include "wavefront.cuh"

using namespace mer;

struct Problem {
    int32_t id = 0;
    mer_hyper hyper{};
    int32_t max_depth = 1, spp_prop = 1, spp_fd = 0;
    int32_t width = 0, height = 0, n_pix = 0;
    int32_t C = 3, W = 1, H = 1;
    int64_t n_par = 0;
    float lo[8] = {0}, hi[8] = {0};
    bool meta = true;
    ProblemDev dev{};
    UpdSeg seg{};
    std::vector<void*> allocs;
    float *pslot[2] = {nullptr, nullptr}, *F = nullptr, *dF = nullptr, *m2f = nullptr, *m2d = nullptr;
    float *mean = nullptr, *var = nullptr, *ap = nullptr;
    // variant state (MER_META_* flags), NULL unless needed
    float *mu_f = nullptr, *mu_d = nullptr, *am = nullptr, *av = nullptr, *Fv = nullptr, *dFv = nullptr;
    Precond pc;                    // gradient preconditioner (precond_lambda > 0)
    bool precond = false;
    float *target = nullptr, *img = nullptr, *dimg = nullptr, *imgA = nullptr, *imgB = nullptr;
    float *dimgA = nullptr, *dimgB = nullptr;
};

// one set of wavefront buffers (a pass in flight uses one set)
struct Wave {
    int64_t qcap = 0, shcap = 0, rcap = 0;
    float* qf[2] = {nullptr, nullptr};
    uint32_t* qu[2] = {nullptr, nullptr};
    float* hitf = nullptr;
    int32_t* hitp = nullptr;
    float* shf = nullptr;
    uint32_t* shu = nullptr;
    uint32_t* cnt = nullptr;       // pass counters + error word
    float* lacc = nullptr;
    float* ltot = nullptr;
    Record* rec = nullptr;
    // hit store of the ADJ_FWD passes (sets 2 and 3), read by their replays (PassArgs::hs)
    float4* hs = nullptr;
    uint8_t* hvis = nullptr;
    int hs_depth = 0;
};

struct mer_ctx {
    int device = 0;
    cudaStream_t user = nullptr;   // caller's stream
    cudaStream_t st = nullptr;     // internal work stream (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    mer_config cfg{};
    std::string err = "no error";
    int sms = 1;
    std::vector<Problem*> probs;
    ProblemDev* d_probs = nullptr;
    ProbState* d_pstate = nullptr;
    double* d_loss = nullptr;
    bool any_uncorrelated = false;   // some problem uses MER_META_UNCORRELATED
    // pass tables
    int32_t *d_prop_prob = nullptr, *d_fd_prob = nullptr;
    int64_t *d_prop_off = nullptr, *d_fd_off = nullptr, *d_pix_pref = nullptr;
    int32_t n_fd = 0;
    int64_t P_prop = 0, P_fd = 0, total_pix = 0;
    int32_t maxD_prop = 0, maxD_fd = 0, maxD = 0;
    // wave sets: 0 proportional primal + replay (and API calls), 1 FD primal + replay,
    // 2 proportional PRB radiance pass, 3 FD PRB radiance pass
    Wave w[4];
    cudaStream_t sx[3] = {nullptr, nullptr, nullptr};   // extra internal streams for concurrent passes
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_loss[2] = {nullptr, nullptr};   // proportional / FD adjoint images ready
    // update
    UpdSeg* d_segs = nullptr;
    int64_t* d_blk_off = nullptr;
    double* d_partials = nullptr;
    int64_t upd_blocks = 0;
    // graph of one iteration
    cudaGraphExec_t gexec = nullptr;
    bool graph_dirty = true;
    LaunchShape shape{128, 0, 0, 1, 8};
    int64_t launches = 0;
    void* timer = nullptr;      // EventTimer while profiling
    bool counting = false;      // profiling mode 2: traversal kernels count their tests
    unsigned long long* d_stats = nullptr;
    bool failed = false;        // a kernel's bounded wait ran out: the context refuses further work
};

namespace {

thread_local std::string t_err = "no error";

const char* const kClassNames[KC_COUNT] = {
    "trace_1_primal", "trace_1_replay", "shade_1_primal", "shade_1_replay",
    "trace_2_primal", "trace_2_replay", "shade_2_primal", "shade_2_replay",
    "resolve", "l2_loss", "zero_grads", "scatter", "precond", "update", "update_finalize"};

// CUDA-event timer installed in mer::g_timer while profiling is enabled
struct EventTimer : KernelTimer {
    struct Rec {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    int64_t units[KC_COUNT] = {0};
    cudaEvent_t get() {
        if (pool.empty()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    void before(int cls, cudaStream_t st) override {
        Rec r{cls, get(), nullptr};
        cudaEventRecord(r.a, st);
        recs.push_back(r);
    }
    void after(int cls, cudaStream_t st) override {
        (void)cls;
        recs.back().b = get();
        cudaEventRecord(recs.back().b, st);
    }
    void add_units(int cls, int64_t n) override { units[cls] += n; }
    void read(mer_kernel_time* out, int max, int* n_out, const unsigned long long* stats) {
        double ms[KC_COUNT] = {0};
        int64_t cnt[KC_COUNT] = {0};
        for (Rec& r : recs) {
            cudaEventSynchronize(r.b);
            float t = 0.0f;
            cudaEventElapsedTime(&t, r.a, r.b);
            ms[r.cls] += t;
            cnt[r.cls]++;
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
        int k = 0;
        for (int c = 0; c < KC_COUNT; ++c) {
            const bool counted = stats && (stats[2 * c] || stats[2 * c + 1]);
            if (!cnt[c] && !counted && !units[c]) continue;
            if (k < max) {
                memset(&out[k], 0, sizeof out[k]);
                snprintf(out[k].name, sizeof out[k].name, "%s", kClassNames[c]);
                out[k].launches = cnt[c];
                out[k].units = units[c];
                out[k].total_ms = ms[c];
                if (stats) {
                    out[k].node_tests = (int64_t)stats[2 * c];
                    out[k].prim_tests = (int64_t)stats[2 * c + 1];
                }
            }
            ++k;
        }
        for (int64_t& u : units) u = 0;
        *n_out = std::min(k, max);
    }
    ~EventTimer() override {
        for (Rec& r : recs) {
            cudaEventDestroy(r.a);
            if (r.b) cudaEventDestroy(r.b);
        }
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
};

mer_status failv(mer_ctx* c, int code, const char* fmt, va_list ap) {
    char buf[1024];
    vsnprintf(buf, sizeof buf, fmt, ap);
    if (c) c->err = buf; else t_err = buf;
    return code;
}

mer_status fail(mer_ctx* c, int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    const mer_status s = failv(c, code, fmt, ap);
    va_end(ap);
    return s;
}

#define CK(ctx, call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MER_ERR_OOM : MER_ERR_CUDA, "%s: %s", #call, \
                        cudaGetErrorString(e_));                                                       \
    } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc((void**)p, count * sizeof(T));
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

// fences between the caller's stream and the internal stream
void enter(mer_ctx* c) {
    cudaEventRecord(c->ev_in, c->user);
    cudaStreamWaitEvent(c->st, c->ev_in, 0);
}
void leave(mer_ctx* c) {
    cudaEventRecord(c->ev_out, c->st);
    cudaStreamWaitEvent(c->user, c->ev_out, 0);
}

struct Guard {
    mer_ctx* c;
    explicit Guard(mer_ctx* c_) : c(c_) {
        cudaSetDevice(c->device);
        enter(c);
    }
    ~Guard() { leave(c); }
};

void free_wave(Wave& w) {
    for (int i = 0; i < 2; ++i) {
        dfree(w.qf[i]);
        dfree(w.qu[i]);
    }
    dfree(w.hitf); dfree(w.hitp); dfree(w.shf); dfree(w.shu); dfree(w.lacc); dfree(w.ltot);
    dfree(w.rec); dfree(w.cnt);
    dfree(w.hs); dfree(w.hvis);
    w = Wave();
}

void free_wavefront(mer_ctx* c) {
    for (Wave& w : c->w) free_wave(w);
}

mer_status alloc_wave(mer_ctx* c, Wave& w, int64_t Q, int64_t R, int hs_depth) {
    const int64_t S = 2 * Q;
    for (int i = 0; i < 2; ++i) {
        CK(c, dalloc(&w.qf[i], (size_t)(2 * QF_PER_BRANCH) * Q));
        CK(c, dalloc(&w.qu[i], (size_t)QU_WORDS * Q));
    }
    CK(c, dalloc(&w.hitf, (size_t)(2 * HF_PER_BRANCH) * Q));
    CK(c, dalloc(&w.hitp, (size_t)2 * Q));
    CK(c, dalloc(&w.shf, (size_t)(SF_SLOT + 2 * SF_PER_SLOT) * S));
    CK(c, dalloc(&w.shu, (size_t)(SU_REC + 2) * S));
    CK(c, dalloc(&w.lacc, (size_t)6 * Q));
    CK(c, dalloc(&w.ltot, (size_t)6 * Q));
    CK(c, dalloc(&w.rec, (size_t)R));
    CK(c, dalloc(&w.cnt, (size_t)CNT_WORDS));
    CK(c, cudaMemset(w.cnt, 0, sizeof(uint32_t) * CNT_WORDS));
    if (hs_depth > 0) {
        const size_t ne = (size_t)2 * hs_depth * Q;          // two branches
        CK(c, dalloc(&w.hs, ne));
        CK(c, dalloc(&w.hvis, ne));
        CK(c, cudaMemset(w.hs, 0xff, sizeof(float4) * ne));   // prim = -1 (miss) until written
        CK(c, cudaMemset(w.hvis, 0, ne));
        w.hs_depth = hs_depth;
    }
    w.qcap = Q;
    w.shcap = S;
    w.rcap = R;
    return MER_OK;
}

// four buffer sets so that independent passes can be in flight together; only sets 0 and 1
// run replay passes and need record buffers
mer_status ensure_wavefront(mer_ctx* c, int64_t need_paths, int maxD) {
    const int64_t want_q = std::max<int64_t>(need_paths, c->cfg.max_paths > 0 ? c->cfg.max_paths : 0);
    const int64_t want_r = 2 * want_q * std::max(1, maxD - 1);
    if (want_q <= c->w[0].qcap && want_r <= c->w[0].rcap && (!c->cfg.replay_hit_store || maxD <= c->w[2].hs_depth))
        return MER_OK;
    cudaStreamSynchronize(c->st);
    for (cudaStream_t s : c->sx) cudaStreamSynchronize(s);
    free_wavefront(c);
    const int64_t Q = std::max<int64_t>(want_q, 1024);
    const int64_t R = std::max<int64_t>(want_r, 1024);
    for (int i = 0; i < 4; ++i) {
        // sets 0 and 1 replay (records); sets 2 and 3 run the ADJ_FWD passes (hit store)
        const int hs_depth = (i < 2 || !c->cfg.replay_hit_store) ? 0 : std::max(1, maxD);
        mer_status s = alloc_wave(c, c->w[i], Q, i < 2 ? R : 1, hs_depth);
        if (s) return s;
    }
    c->graph_dirty = true;
    return MER_OK;
}

// grid of the simple grid-stride kernels (resolve, loss, scatter)
int grid_for(mer_ctx* c, int block) { return c->sms * (2048 / block); }

PassArgs base_args(mer_ctx* c, const Wave& w) {
    PassArgs A;
    memset(&A, 0, sizeof A);
    A.probs = c->d_probs;
    A.pstate = c->d_pstate;
    A.inl_prob = -1;
    A.iter_override = -1;
    A.qf[0] = w.qf[0]; A.qf[1] = w.qf[1];
    A.qu[0] = w.qu[0]; A.qu[1] = w.qu[1];
    A.qcap = w.qcap;
    A.hitf = w.hitf; A.hitp = w.hitp;
    A.shf = w.shf; A.shu = w.shu; A.shcap = w.shcap;
    A.cnt = w.cnt;
    A.lacc = w.lacc; A.ltot = w.ltot;
    A.rec = w.rec; A.rcap = w.rcap;
    A.smem_nodes = c->shape.smem_nodes;
    A.smem_prob = 0;
    A.stats = c->counting ? c->d_stats : nullptr;
    return A;
}

LaunchShape shape_of(mer_ctx* c) {
    LaunchShape L = c->shape;
    if (L.block <= 0) L.block = 128;
    L.per_sm = c->cfg.blocks_per_sm;
    L.sms = c->sms;
    return L;
}

// the hit store of wave set w (its ADJ_FWD pass writes it, the matching replay reads it)
void hit_store(PassArgs& A, const Wave& w) {
    A.hs = w.hs;
    A.hvis = w.hvis;
    A.hs_depth = w.hs_depth;
    A.hs_cap = w.qcap;
}

// zero the pass counters (not the error word) and run one pass on stream st
int pass(mer_ctx* c, cudaStream_t st, PassArgs A, int nb, int mode, int maxD) {
    cudaMemsetAsync(A.cnt, 0, CNT_ERR * sizeof(uint32_t), st);
    const LaunchShape L = shape_of(c);
    const int n = run_pass(A, nb, mode, maxD, L, st);   // kernel launches (the memset is not one)
    if (g_timer) {
        // work items of this pass: rays per depth and NEE rays, read back from the pass counters
        uint32_t h[CNT_WORDS];
        cudaMemcpyAsync(h, A.cnt, sizeof h, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        int64_t rays = A.n_paths, sh = 0;
        for (int k = 2; k <= maxD; ++k) rays += h[CNT_Q + k];
        for (int k = 1; k <= maxD; ++k) sh += h[CNT_S + k];
        const int rep = mode == MODE_REPLAY ? 1 : 0;
        if (!(rep && A.hs)) g_timer->add_units((nb == 1 ? KC_TRACE1_PRIMAL : KC_TRACE2_PRIMAL) + rep, rays + sh);
        g_timer->add_units((nb == 1 ? KC_SHADE1_PRIMAL : KC_SHADE2_PRIMAL) + rep, rays);
        if (mode == MODE_REPLAY) g_timer->add_units(KC_SCATTER, h[CNT_R]);
    }
    return n;
}

// the gradient part of one iteration for all problems (steps a1-a10), as a graph of passes in
// two independent chains that join before the update:
//   proportional: primal image [main stream, wave set 0] -> its loss and adjoint image (main)
//                 PRB radiance [stream x1, wave set 2]   -> (both done) replay [x1, set 0, L_total
//                 and hits of set 2] + scatter into F
//   FD pair:      primal image pair [x0, set 1] -> the pair's adjoint images (x0)
//                 PRB radiance pair [x2, set 3] -> (both done) replay pair [x2, set 1, L_total and
//                 hits of set 3] + scatter into dF
// Branches fork and join through events, so inside stream capture they become parallel graph
// branches. While per-kernel timing is on, everything runs on the main stream.
int enqueue_gradient(mer_ctx* c) {
    int n = 0;
    const int G = grid_for(c, 256);
    const bool have_fd = c->n_fd > 0 && c->P_fd > 0;
    const bool split = !g_timer;
    const int NP = (int)c->probs.size();
    cudaStream_t s[4] = {c->st, split ? c->sx[0] : c->st, split ? c->sx[1] : c->st, split ? c->sx[2] : c->st};
    auto prop_args = [&](int wi) {
        PassArgs A = base_args(c, c->w[wi]);
        A.entry_prob = c->d_prop_prob;
        A.path_off = c->d_prop_off;
        A.n_entries = NP;
        A.n_paths = c->P_prop;
        return A;
    };
    auto fd_args = [&](int wi) {
        PassArgs A = base_args(c, c->w[wi]);
        A.entry_prob = c->d_fd_prob;
        A.path_off = c->d_fd_off;
        A.n_entries = c->n_fd;
        A.n_paths = c->P_fd;
        A.fd_kind = 1;
        return A;
    };
    auto fork = [&](int branches) {
        if (!split) return;
        cudaEventRecord(c->ev_fork, s[0]);
        for (int b = 1; b < branches; ++b) cudaStreamWaitEvent(s[b], c->ev_fork, 0);
    };
    auto join = [&](int branches) {
        if (!split) return;
        for (int b = 1; b < branches; ++b) {
            cudaEventRecord(c->ev_join[b - 1], s[b]);
            cudaStreamWaitEvent(s[0], c->ev_join[b - 1], 0);
        }
    };
    auto zero = [&](int which, cudaStream_t st) {
        n += run_zero_grads(c->d_probs, NP, which, G, st);
        if (g_timer)
            for (Problem* p : c->probs) g_timer->add_units(KC_ZERO, p->n_par);
    };
    // One gradient evaluation: proportional samples into gradient texture wF and FD samples into
    // wD, drawn from the four gradient streams shifted by soff, loss accumulated into `loss`.
    auto evaluate = [&](uint32_t soff, int wF, int wD, double* loss) {
        cudaMemsetAsync(loss, 0, sizeof(double) * NP, s[0]);
        fork(4);
        // ---- proportional chain ----
        PassArgs P = prop_args(0);
        P.stream = MER_STREAM_PROP_PRIMAL + soff;
        n += pass(c, s[0], P, 1, MODE_PRIMAL, c->maxD_prop);
        n += run_resolve(P, 1, nullptr, nullptr, 0, G, s[0]);
        n += run_l2(c->d_probs, c->d_pix_pref, NP, c->total_pix, L2_PROP, loss, G, s[0]);
        if (split) cudaEventRecord(c->ev_loss[0], s[0]);
        PassArgs PR = prop_args(2);
        PR.stream = MER_STREAM_PROP_ADJ + soff;
        PR.lacc = c->w[2].ltot;                  // per-path radiance L_total of the replayed paths
        hit_store(PR, c->w[2]);
        n += pass(c, s[2], PR, 1, MODE_ADJ_FWD, c->maxD_prop);
        if (split) cudaStreamWaitEvent(s[2], c->ev_loss[0], 0);
        // proportional gradient <F_i>: replay from the same counters (in wave set 0, after the
        // primal pass left it), scatter into F (cleared right before, so that the reductions
        // find it in L2)
        P.stream = MER_STREAM_PROP_ADJ + soff;
        P.ltot = c->w[2].ltot;
        hit_store(P, c->w[2]);
        n += pass(c, s[2], P, 1, MODE_REPLAY, c->maxD_prop);
        zero(wF, s[2]);
        n += run_scatter(c->w[0].cnt, c->w[0].rec, c->w[0].rcap, c->d_probs, NP, nullptr, wF, G, s[2]);
        // ---- FD chain (Eq. est_triv) ----
        if (have_fd) {
            PassArgs D = fd_args(1);
            D.stream = MER_STREAM_FD_PRIMAL + soff;
            n += pass(c, s[1], D, 2, MODE_PRIMAL, c->maxD_fd);
            n += run_resolve(D, 2, nullptr, nullptr, 0, G, s[1]);
            n += run_l2(c->d_probs, c->d_pix_pref, NP, c->total_pix, L2_FD, loss, G, s[1]);
            if (split) cudaEventRecord(c->ev_loss[1], s[1]);
            PassArgs DR = fd_args(3);
            DR.stream = MER_STREAM_FD_ADJ + soff;
            DR.lacc = c->w[3].ltot;
            hit_store(DR, c->w[3]);
            n += pass(c, s[3], DR, 2, MODE_ADJ_FWD, c->maxD_fd);
            if (split) cudaStreamWaitEvent(s[3], c->ev_loss[1], 0);
            D.stream = MER_STREAM_FD_ADJ + soff;
            D.ltot = c->w[3].ltot;
            hit_store(D, c->w[3]);
            n += pass(c, s[3], D, 2, MODE_REPLAY, c->maxD_fd);
            zero(wD, s[3]);
            n += run_scatter(c->w[1].cnt, c->w[1].rec, c->w[1].rcap, c->d_probs, NP, nullptr, wD, G, s[3]);
        }
        join(4);
    };
    evaluate(0u, 0, 1, c->d_loss);
    // MER_META_UNCORRELATED: a second, independent evaluation (own streams) for the variances
    if (c->any_uncorrelated) evaluate(MER_STREAM_VAR_OFFSET, 2, 3, c->d_loss + MER_MAX_PROBLEMS);
    // gradient preconditioning of the problems that ask for it, before the update
    for (Problem* p : c->probs) {
        if (!p->precond) continue;
        if (g_timer) g_timer->before(KC_PRECOND, s[0]);
        for (float* gbuf : {p->F, p->meta ? p->dF : nullptr, p->Fv, p->dFv})
            if (gbuf) n += precond_apply(p->pc, gbuf, s[0]);
        if (g_timer) {
            g_timer->after(KC_PRECOND, s[0]);
            g_timer->add_units(KC_PRECOND, p->n_par);
        }
    }
    return n;
}

int enqueue_update(mer_ctx* c) {
    if (g_timer)
        for (Problem* p : c->probs) g_timer->add_units(KC_UPDATE, p->n_par);
    launch_update_ctx(c->d_segs, c->d_blk_off, (int)c->probs.size(), c->upd_blocks, c->d_pstate, c->d_partials, c->st);
    return 2;
}

mer_status check_err_word(mer_ctx* c) {
    for (Wave& w : c->w) {
        if (!w.cnt) continue;
        uint32_t e = 0;
        CK(c, cudaMemcpy(&e, w.cnt + CNT_ERR, sizeof e, cudaMemcpyDeviceToHost));
        if (e) {
            cudaMemset(w.cnt + CNT_ERR, 0, sizeof(uint32_t));
            // a bounded wait that ran out may have left copies in flight: nothing the context
            // computes from now on can be trusted
            if (e == MER_ERR_TIMEOUT) c->failed = true;
            return fail(c, (int)e, "a kernel reported %s (code %u)",
                        e == MER_ERR_TIMEOUT ? "a bounded wait that ran out" : "an out-of-capacity write", e);
        }
    }
    return MER_OK;
}

// rebuild the pass tables, problem table and update segments after the problem set changed
mer_status rebuild_tables(mer_ctx* c) {
    const int n = (int)c->probs.size();
    std::vector<ProblemDev> pd(n);
    std::vector<int32_t> prop_prob(n), fd_prob;
    std::vector<int64_t> prop_off(n + 1, 0), fd_off(1, 0), pix_pref(n + 1, 0);
    std::vector<UpdSeg> segs(n);
    std::vector<int64_t> blk_off(n + 1, 0);
    c->maxD_prop = c->maxD_fd = 0;
    c->any_uncorrelated = false;
    for (int i = 0; i < n; ++i) {
        Problem* p = c->probs[i];
        if (p->meta && (p->hyper.flags & MER_META_UNCORRELATED)) c->any_uncorrelated = true;
        pd[i] = p->dev;
        prop_prob[i] = i;
        prop_off[i + 1] = prop_off[i] + (int64_t)p->n_pix * p->spp_prop;
        c->maxD_prop = std::max(c->maxD_prop, p->max_depth);
        if (p->meta && p->spp_fd > 0) {
            fd_prob.push_back(i);
            fd_off.push_back(fd_off.back() + (int64_t)p->n_pix * p->spp_fd);
            c->maxD_fd = std::max(c->maxD_fd, p->max_depth);
        }
        pix_pref[i + 1] = pix_pref[i] + p->n_pix;
        segs[i] = p->seg;
        segs[i].prob = i;
        blk_off[i + 1] = blk_off[i] + update_blocks_for(p->n_par);
    }
    c->n_fd = (int)fd_prob.size();
    c->P_prop = prop_off[n];
    c->P_fd = fd_off.back();
    c->total_pix = pix_pref[n];
    c->upd_blocks = blk_off[n];
    c->maxD = std::max(c->maxD_prop, c->maxD_fd);
    cudaStreamSynchronize(c->st);
    dfree(c->d_probs); dfree(c->d_prop_prob); dfree(c->d_prop_off); dfree(c->d_fd_prob); dfree(c->d_fd_off);
    dfree(c->d_pix_pref); dfree(c->d_segs); dfree(c->d_blk_off); dfree(c->d_partials);
    CK(c, dalloc(&c->d_probs, n));
    CK(c, dalloc(&c->d_prop_prob, n));
    CK(c, dalloc(&c->d_prop_off, n + 1));
    CK(c, dalloc(&c->d_fd_prob, std::max<size_t>(1, fd_prob.size())));
    CK(c, dalloc(&c->d_fd_off, fd_off.size()));
    CK(c, dalloc(&c->d_pix_pref, n + 1));
    CK(c, dalloc(&c->d_segs, n));
    CK(c, dalloc(&c->d_blk_off, n + 1));
    CK(c, dalloc(&c->d_partials, std::max<int64_t>(1, c->upd_blocks)));
    CK(c, cudaMemcpy(c->d_probs, pd.data(), sizeof(ProblemDev) * n, cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->d_prop_prob, prop_prob.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->d_prop_off, prop_off.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice));
    if (!fd_prob.empty())
        CK(c, cudaMemcpy(c->d_fd_prob, fd_prob.data(), sizeof(int32_t) * fd_prob.size(), cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->d_fd_off, fd_off.data(), sizeof(int64_t) * fd_off.size(), cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->d_pix_pref, pix_pref.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->d_segs, segs.data(), sizeof(UpdSeg) * n, cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->d_blk_off, blk_off.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice));
    int64_t need = std::max(c->P_prop, c->P_fd);
    for (Problem* p : c->probs) need = std::max<int64_t>(need, p->n_pix);
    mer_status s = ensure_wavefront(c, need, c->maxD);
    if (s) return s;
    c->graph_dirty = true;
    return MER_OK;
}

mer_status reset_state(mer_ctx* c, Problem* p) {
    const size_t nb = sizeof(float) * (size_t)p->n_par;
    CK(c, cudaMemsetAsync(p->F, 0, nb, c->st));
    CK(c, cudaMemsetAsync(p->dF, 0, nb, c->st));
    CK(c, cudaMemsetAsync(p->m2f, 0, nb, c->st));
    CK(c, cudaMemsetAsync(p->m2d, 0, nb, c->st));
    CK(c, cudaMemsetAsync(p->mean, 0, nb, c->st));
    CK(c, cudaMemsetAsync(p->var, 0, nb, c->st));
    run_fill(p->ap, p->n_par, -INFINITY, c->st);
    for (float* a : {p->mu_f, p->mu_d, p->am, p->av, p->Fv, p->dFv})
        if (a) CK(c, cudaMemsetAsync(a, 0, nb, c->st));
    ProbState ps{};
    ps.coef = update_coef(p->hyper, 0, 0, 0, 0.0);
    CK(c, cudaMemcpyAsync(c->d_pstate + p->id, &ps, sizeof ps, cudaMemcpyHostToDevice, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    return MER_OK;
}

Problem* get_prob(mer_ctx* c, int32_t pid) {
    if (!c || pid < 0 || pid >= (int32_t)c->probs.size()) return nullptr;
    return c->probs[pid];
}

mer_status copy_in(mer_ctx* c, float* dst, const float* src, size_t n, int on_device) {
    if (!src) return fail(c, MER_ERR_INVALID_ARG, "null input pointer");
    CK(c, cudaMemcpyAsync(dst, src, n * sizeof(float), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          c->st));
    if (!on_device) CK(c, cudaStreamSynchronize(c->st));
    return MER_OK;
}

int32_t read_cur(mer_ctx* c, Problem* p) {
    ProbState ps{};
    cudaMemcpyAsync(&ps, c->d_pstate + p->id, sizeof ps, cudaMemcpyDeviceToHost, c->st);
    cudaStreamSynchronize(c->st);
    return ps.cur;
}

// single-problem pass helpers for the API calls (chunked over samples)
PassArgs single_args(mer_ctx* c, Problem* p, uint32_t stream, uint32_t iteration, int spp) {
    PassArgs A = base_args(c, c->w[0]);
    A.inl_prob = p->id;
    A.stream = stream;
    A.iter_override = (int32_t)iteration;
    A.spp_override = spp;
    A.smem_prob = p->id;
    return A;
}

int64_t chunk_spp(mer_ctx* c, Problem* p, int spp) {
    return std::max<int64_t>(1, std::min<int64_t>(spp, c->w[0].qcap / std::max(1, p->n_pix)));
}

}  // namespace

namespace mer {
int mer_internal_fail(int code, const char* msg) {
    t_err = msg;
    return code;
}
}  // namespace mer

// =====================================================================================
// exported entry points
// =====================================================================================
extern "C" {

mer_status mer_hyper_default(mer_hyper* h) {
    if (!h) return fail(nullptr, MER_ERR_INVALID_ARG, "null hyper");
    h->mode = MER_MODE_META;
    h->lr = 0.01f;
    h->beta_f = 0.99f;
    h->beta_d = 0.9f;
    h->eps = 1e-8f;
    h->eps_alpha = 1e-30f;
    h->beta1 = 0.9f;
    h->beta2 = 0.999f;
    h->flags = 0;
    return MER_OK;
}

const char* mer_last_error(const mer_ctx* ctx) { return ctx ? ctx->err.c_str() : t_err.c_str(); }

mer_status mer_create(const mer_config* cfg, void* cuda_stream, mer_ctx** out) {
    if (!out) return fail(nullptr, MER_ERR_INVALID_ARG, "null output");
    *out = nullptr;
    mer_config def{};
    const mer_config& C = cfg ? *cfg : def;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(nullptr, MER_ERR_CUDA, "no CUDA device available");
    if (C.device < 0 || C.device >= ndev) return fail(nullptr, MER_ERR_INVALID_ARG, "bad device %d", C.device);
    mer_ctx* c = new mer_ctx();
    c->cfg = C;
    c->device = C.device;
    c->user = (cudaStream_t)cuda_stream;
    cudaSetDevice(c->device);
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    c->shape.block = C.block_size > 0 ? C.block_size : 128;
    c->shape.smem_nodes = C.smem_nodes;
    c->shape.refill = C.trace_refill > 0 ? std::min(C.trace_refill, 32) : 8;
    cudaError_t e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
    if (!e) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
    if (!e) e = cudaMalloc(&c->d_pstate, sizeof(ProbState) * MER_MAX_PROBLEMS);
    if (!e) e = cudaMalloc(&c->d_loss, sizeof(double) * 2 * MER_MAX_PROBLEMS);   // loss, variance-sample loss
    for (int i = 0; i < 3 && !e; ++i) {
        e = cudaStreamCreateWithFlags(&c->sx[i], cudaStreamNonBlocking);
        if (!e) e = cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming);
        if (!e && i < 2) e = cudaEventCreateWithFlags(&c->ev_loss[i], cudaEventDisableTiming);
    }
    if (!e) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (!e) e = cudaMemset(c->d_loss, 0, sizeof(double) * 2 * MER_MAX_PROBLEMS);
    if (!e && c->shape.smem_nodes > 0) e = set_trace_smem_limits(c->shape.smem_nodes);
    if (e) {
        fail(nullptr, MER_ERR_CUDA, "context setup failed: %s", cudaGetErrorString(e));
        mer_destroy(c);
        return MER_ERR_CUDA;
    }
    *out = c;
    return MER_OK;
}

void mer_destroy(mer_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->st) cudaStreamSynchronize(c->st);
    mer_profile_enable(c, 0);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    for (Problem* p : c->probs) {
        for (void* a : p->allocs) dfree(a);
        delete p;
    }
    free_wavefront(c);
    dfree(c->d_probs); dfree(c->d_pstate); dfree(c->d_loss);
    dfree(c->d_prop_prob); dfree(c->d_prop_off); dfree(c->d_fd_prob); dfree(c->d_fd_off); dfree(c->d_pix_pref);
    dfree(c->d_segs); dfree(c->d_blk_off); dfree(c->d_partials);
    dfree(c->d_stats);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    for (int i = 0; i < 3; ++i) {
        if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
        if (i < 2 && c->ev_loss[i]) cudaEventDestroy(c->ev_loss[i]);
        if (c->sx[i]) cudaStreamDestroy(c->sx[i]);
    }
    if (c->st) cudaStreamDestroy(c->st);
    delete c;
}

mer_status mer_scene_add(mer_ctx* c, const mer_scene_desc* d, int32_t* problem_id) {
    if (!c || !d || !problem_id) return fail(c, MER_ERR_INVALID_ARG, "null argument");
    if ((int)c->probs.size() >= MER_MAX_PROBLEMS) return fail(c, MER_ERR_INVALID_ARG, "too many problems");
    if (d->n_tris < 0 || d->n_verts < 0 || d->n_spheres < 0 || d->n_mats <= 0 || d->n_quads < 0)
        return fail(c, MER_ERR_INVALID_ARG, "negative counts or no materials");
    if ((d->n_tris > 0 && (!d->positions || !d->uvs || !d->tris || !d->tri_mat || !d->tri_light)) ||
        (d->n_spheres > 0 && (!d->spheres || !d->sph_mat)) || !d->mat_type || !d->mat_textured || !d->mat_const ||
        (d->n_quads > 0 && !d->quads))
        return fail(c, MER_ERR_INVALID_ARG, "missing scene arrays");
    if (d->width <= 0 || d->height <= 0 || (int64_t)d->width * d->height > (int64_t)INT32_MAX)
        return fail(c, MER_ERR_INVALID_ARG, "bad image size");
    if (!(d->tex_c == 3 || d->tex_c == 5) || d->tex_w <= 0 || d->tex_h <= 0 || d->tex_w > 4094 || d->tex_h > 4094)
        return fail(c, MER_ERR_INVALID_ARG, "texture must be C in {3,5}, 1..4094 texels per side");
    if (d->max_depth < 1 || d->max_depth > MER_MAX_DEPTH) return fail(c, MER_ERR_INVALID_ARG, "max_depth out of range");
    if (d->spp_prop < 1 || d->spp_fd < 0) return fail(c, MER_ERR_INVALID_ARG, "bad spp");
    if (d->loss != MER_LOSS_L2 && d->loss != MER_LOSS_MRSE) return fail(c, MER_ERR_INVALID_ARG, "bad loss");
    for (int i = 0; i < d->n_mats; ++i) {
        if (d->mat_type[i] != 0 && d->mat_type[i] != 1) return fail(c, MER_ERR_INVALID_ARG, "bad material type");
        if (d->mat_type[i] == 1 && d->mat_textured[i] && d->tex_c != 5)
            return fail(c, MER_ERR_INVALID_ARG, "textured principled material needs a 5-channel texture");
    }
    for (int i = 0; i < d->n_tris; ++i) {
        for (int k = 0; k < 3; ++k)
            if (d->tris[3 * i + k] < 0 || d->tris[3 * i + k] >= d->n_verts)
                return fail(c, MER_ERR_INVALID_ARG, "triangle %d has a bad vertex index", i);
        if (d->tri_mat[i] < 0 || d->tri_mat[i] >= d->n_mats) return fail(c, MER_ERR_INVALID_ARG, "bad tri material");
        if (d->tri_light[i] < -1 || d->tri_light[i] >= d->n_quads) return fail(c, MER_ERR_INVALID_ARG, "bad tri light");
    }
    for (int i = 0; i < d->n_spheres; ++i)
        if (d->sph_mat[i] < 0 || d->sph_mat[i] >= d->n_mats || !(d->spheres[8 * i + 3] > 0.0f))
            return fail(c, MER_ERR_INVALID_ARG, "bad sphere %d", i);
    for (int i = 0; i < d->n_quads; ++i) {
        // the light's area density divides by |e1 x e2|; its emission must be a radiance
        const float* q = d->quads + 12 * i;
        const double cx = (double)q[4] * q[8] - (double)q[5] * q[7], cy = (double)q[5] * q[6] - (double)q[3] * q[8],
                     cz = (double)q[3] * q[7] - (double)q[4] * q[6];
        if (!(cx * cx + cy * cy + cz * cz > 0.0) || !(q[9] >= 0.0f && q[10] >= 0.0f && q[11] >= 0.0f) ||
            !std::isfinite(q[9] + q[10] + q[11]))
            return fail(c, MER_ERR_INVALID_ARG, "quad light %d has no area or a bad emission", i);
    }
    for (int k = 0; k < d->tex_c; ++k)
        if (!(d->clamp_lo[k] <= d->clamp_hi[k]))
            return fail(c, MER_ERR_INVALID_ARG, "parameter range of channel %d is empty", k);
    cudaSetDevice(c->device);

    Problem* p = new Problem();
    p->id = (int32_t)c->probs.size();
    p->hyper = d->hyper;
    if (p->hyper.lr == 0.0f && p->hyper.beta_f == 0.0f) {   // all-zero hyper: defaults (flags kept)
        const int32_t fl = p->hyper.flags;
        mer_hyper_default(&p->hyper);
        p->hyper.flags = fl;
    }
    if (const char* why = hyper_problem(p->hyper)) {
        delete p;
        return fail(c, MER_ERR_INVALID_ARG, "%s", why);
    }
    p->meta = p->hyper.mode == MER_MODE_META;
    p->max_depth = d->max_depth;
    p->spp_prop = d->spp_prop;
    p->spp_fd = p->meta ? d->spp_fd : 0;
    p->width = d->width;
    p->height = d->height;
    p->n_pix = d->width * d->height;
    p->C = d->tex_c;
    p->W = d->tex_w;
    p->H = d->tex_h;
    p->n_par = (int64_t)p->C * p->W * p->H;
    for (int k = 0; k < 8; ++k) {
        p->lo[k] = d->clamp_lo[k];
        p->hi[k] = d->clamp_hi[k];
    }
    auto bail = [&](mer_status s) {
        for (void* a : p->allocs) dfree(a);
        delete p;
        return s;
    };
    auto alloc = [&](auto** ptr, size_t count) -> cudaError_t {
        cudaError_t e = dalloc(ptr, std::max<size_t>(count, 1));
        if (!e) p->allocs.push_back((void*)*ptr);
        return e;
    };
#define AK(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_) return bail(fail(c, MER_ERR_OOM, "allocation failed: %s", cudaGetErrorString(e_))); \
    } while (0)

    // ---- geometry: BVH over triangles, leaf-ordered triangle records, attributes ----
    ProblemDev& D = p->dev;
    memset(&D, 0, sizeof D);
    D.n_tris = d->n_tris;
    D.n_sph = d->n_spheres;
    D.n_quads = d->n_quads;
    D.has_env = d->has_env ? 1 : 0;
    D.n_lights = d->n_quads + D.has_env;
    for (int k = 0; k < 3; ++k) D.env[k] = d->has_env ? d->env[k] : 0.0f;
    if (d->n_tris > 0) {
        std::vector<HostNode> hn;
        std::vector<int> order;
        const int root2 = build_bvh(d->positions, d->tris, d->n_tris, hn, order);
        std::vector<HostNode4> h4;
        collapse_bvh4(hn, root2, h4);
        if (3 * bvh4_levels(h4) > TRAV_STACK)
            return bail(fail(c, MER_ERR_INVALID_ARG,
                             "mer_scene_add: the triangle BVH has %d levels; the traversal stack holds %d (at most %d "
                             "levels)", bvh4_levels(h4), TRAV_STACK, TRAV_STACK / 3));
        std::vector<Node> nodes(h4.size());
        for (size_t i = 0; i < h4.size(); ++i) {
            const HostNode4& h = h4[i];
            Node& n = nodes[i];
            n.lx = make_float4(h.lo[0][0], h.lo[1][0], h.lo[2][0], h.lo[3][0]);
            n.hx = make_float4(h.hi[0][0], h.hi[1][0], h.hi[2][0], h.hi[3][0]);
            n.ly = make_float4(h.lo[0][1], h.lo[1][1], h.lo[2][1], h.lo[3][1]);
            n.hy = make_float4(h.hi[0][1], h.hi[1][1], h.hi[2][1], h.hi[3][1]);
            n.lz = make_float4(h.lo[0][2], h.lo[1][2], h.lo[2][2], h.lo[3][2]);
            n.hz = make_float4(h.hi[0][2], h.hi[1][2], h.hi[2][2], h.hi[3][2]);
            n.child = make_int4(h.child[0], h.child[1], h.child[2], h.child[3]);
            n.pad = make_int4(0, 0, 0, 0);
        }
        std::vector<TriGeo> tg(d->n_tris);
        std::vector<TriAttr> ta(d->n_tris);
        for (int t = 0; t < d->n_tris; ++t) {
            const int* T = d->tris + 3 * t;
            const float* a = d->positions + 3 * T[0];
            const float* b = d->positions + 3 * T[1];
            const float* cc = d->positions + 3 * T[2];
            double e1[3], e2[3];
            for (int k = 0; k < 3; ++k) {
                e1[k] = (double)b[k] - a[k];
                e2[k] = (double)cc[k] - a[k];
            }
            double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
            const double ln = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            TriAttr& A = ta[t];
            for (int k = 0; k < 3; ++k) A.n[k] = ln > 0 ? (float)(n[k] / ln) : (k == 2 ? 1.0f : 0.0f);
            for (int v = 0; v < 3; ++v) {
                A.uv[2 * v] = d->uvs[2 * T[v]];
                A.uv[2 * v + 1] = d->uvs[2 * T[v] + 1];
            }
            A.mat = d->tri_mat[t];
            A.light = d->tri_light[t];
            A.pad = 0;
        }
        for (int k = 0; k < d->n_tris; ++k) {
            const int t = order[k];
            const int* T = d->tris + 3 * t;
            const float* a = d->positions + 3 * T[0];
            const float* b = d->positions + 3 * T[1];
            const float* cc = d->positions + 3 * T[2];
            int tid = t;
            float tidf;
            memcpy(&tidf, &tid, 4);
            tg[k].v0 = make_float4(a[0], a[1], a[2], tidf);
            tg[k].e1 = make_float4((float)((double)b[0] - a[0]), (float)((double)b[1] - a[1]),
                                   (float)((double)b[2] - a[2]), 0.0f);
            tg[k].e2 = make_float4((float)((double)cc[0] - a[0]), (float)((double)cc[1] - a[1]),
                                   (float)((double)cc[2] - a[2]), 0.0f);
        }
        Node* dn;
        TriGeo* dt;
        TriAttr* da;
        AK(alloc(&dn, nodes.size()));
        AK(alloc(&dt, tg.size()));
        AK(alloc(&da, ta.size()));
        AK(cudaMemcpy(dn, nodes.data(), sizeof(Node) * nodes.size(), cudaMemcpyHostToDevice));
        AK(cudaMemcpy(dt, tg.data(), sizeof(TriGeo) * tg.size(), cudaMemcpyHostToDevice));
        AK(cudaMemcpy(da, ta.data(), sizeof(TriAttr) * ta.size(), cudaMemcpyHostToDevice));
        D.nodes = dn;
        D.n_nodes = (int32_t)nodes.size();
        D.tris = dt;
        D.attr = da;
    }
    {
        std::vector<Sphere> sp(d->n_spheres);
        for (int i = 0; i < d->n_spheres; ++i) {
            const float* S = d->spheres + 8 * i;
            sp[i].cr = make_float4(S[0], S[1], S[2], S[3]);
            sp[i].uvr = make_float4(S[4], S[5], S[6], S[7]);
            sp[i].mat = d->sph_mat[i];
        }
        std::vector<Material> mt(d->n_mats);
        for (int i = 0; i < d->n_mats; ++i) {
            mt[i].type = d->mat_type[i];
            mt[i].textured = d->mat_textured[i];
            for (int k = 0; k < 5; ++k) mt[i].c[k] = d->mat_const[5 * i + k];
            mt[i].pad = 0;
        }
        std::vector<QuadLight> ql(d->n_quads);
        for (int i = 0; i < d->n_quads; ++i) {
            const float* Q = d->quads + 12 * i;
            QuadLight& L = ql[i];
            for (int k = 0; k < 3; ++k) {
                L.p0[k] = Q[k];
                L.e1[k] = Q[3 + k];
                L.e2[k] = Q[6 + k];
                L.le[k] = Q[9 + k];
            }
            const double n[3] = {(double)Q[4] * Q[8] - (double)Q[5] * Q[7], (double)Q[5] * Q[6] - (double)Q[3] * Q[8],
                                 (double)Q[3] * Q[7] - (double)Q[4] * Q[6]};
            const double a = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            if (!(a > 0)) return bail(fail(c, MER_ERR_INVALID_ARG, "degenerate quad light %d", i));
            for (int k = 0; k < 3; ++k) L.n[k] = (float)(n[k] / a);
            L.area = (float)a;
        }
        Sphere* ds;
        Material* dm;
        QuadLight* dq;
        AK(alloc(&ds, sp.size()));
        AK(alloc(&dm, mt.size()));
        AK(alloc(&dq, ql.size()));
        if (!sp.empty()) AK(cudaMemcpy(ds, sp.data(), sizeof(Sphere) * sp.size(), cudaMemcpyHostToDevice));
        AK(cudaMemcpy(dm, mt.data(), sizeof(Material) * mt.size(), cudaMemcpyHostToDevice));
        if (!ql.empty()) AK(cudaMemcpy(dq, ql.data(), sizeof(QuadLight) * ql.size(), cudaMemcpyHostToDevice));
        D.sph = ds;
        D.mats = dm;
        D.quads = dq;
    }
    // camera: pinhole, vertical fov, row 0 at the top
    {
        double eye[3], f[3], up[3], r[3], u[3];
        for (int k = 0; k < 3; ++k) {
            eye[k] = d->eye[k];
            f[k] = (double)d->target[k] - d->eye[k];
            up[k] = d->up[k];
        }
        double lf = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        for (double& x : f) x /= lf;
        r[0] = f[1] * up[2] - f[2] * up[1];
        r[1] = f[2] * up[0] - f[0] * up[2];
        r[2] = f[0] * up[1] - f[1] * up[0];
        const double lr = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (!(lf > 0) || !(lr > 0) || !(d->fov_deg > 0.0f && d->fov_deg < 180.0f))
            return bail(fail(c, MER_ERR_INVALID_ARG, "degenerate camera"));
        for (double& x : r) x /= lr;
        u[0] = r[1] * f[2] - r[2] * f[1];
        u[1] = r[2] * f[0] - r[0] * f[2];
        u[2] = r[0] * f[1] - r[1] * f[0];
        const double th = std::tan(0.5 * (double)d->fov_deg * 3.14159265358979323846 / 180.0);
        const double asp = (double)d->width / (double)d->height;
        for (int k = 0; k < 3; ++k) {
            D.cam_o[k] = (float)eye[k];
            D.cam_f[k] = (float)f[k];
            D.cam_r[k] = (float)(r[k] * th * asp);
            D.cam_u[k] = (float)(u[k] * th);
        }
    }
    D.width = d->width;
    D.height = d->height;
    D.n_pix = p->n_pix;
    D.tex_c = p->C;
    D.tex_w = p->W;
    D.tex_h = p->H;
    D.n_par = p->n_par;
    D.max_depth = p->max_depth;
    D.spp_prop = p->spp_prop;
    D.spp_fd = p->spp_fd;
    D.seed = d->seed;
    D.key_id = d->key_id;
    D.loss_kind = d->loss;
    D.fd_shared = (p->meta && (p->hyper.flags & MER_META_FD_SHARED_PATH)) ? 1 : 0;
    // ---- optimiser state and images ----
    const size_t np = (size_t)p->n_par, npx = (size_t)p->n_pix * 3;
    AK(alloc(&p->pslot[0], np));
    AK(alloc(&p->pslot[1], np));
    AK(alloc(&p->F, np));
    AK(alloc(&p->dF, np));
    AK(alloc(&p->m2f, np));
    AK(alloc(&p->m2d, np));
    AK(alloc(&p->mean, np));
    AK(alloc(&p->var, np));
    AK(alloc(&p->ap, np));
    const int vfl = p->meta ? p->hyper.flags : 0;
    if (vfl & MER_META_CENTRED) {
        AK(alloc(&p->mu_f, np));
        AK(alloc(&p->mu_d, np));
    }
    if (vfl & MER_META_NAIVE_ADAM) {
        AK(alloc(&p->am, np));
        AK(alloc(&p->av, np));
    }
    if (vfl & MER_META_UNCORRELATED) {
        AK(alloc(&p->Fv, np));
        AK(alloc(&p->dFv, np));
    }
    if (p->hyper.precond_lambda > 0.0f) {
        const cudaError_t pe = precond_init(p->pc, p->C, p->H, p->W, p->hyper.precond_lambda);
        for (void* a : {(void*)p->pc.ax_w.fft_tw, (void*)p->pc.ax_w.dct_tw, (void*)p->pc.ax_w.cos4,
                        (void*)p->pc.ax_h.fft_tw, (void*)p->pc.ax_h.dct_tw, (void*)p->pc.ax_h.cos4, (void*)p->pc.St,
                        (void*)p->pc.T1, (void*)p->pc.T2})
            if (a) p->allocs.push_back(a);   // freed with the problem, also on the error path
        AK(pe);
        p->precond = true;
    }
    AK(alloc(&p->target, npx));
    AK(alloc(&p->img, npx));
    AK(alloc(&p->dimg, npx));
    if (p->meta) {
        AK(alloc(&p->imgA, npx));
        AK(alloc(&p->imgB, npx));
        AK(alloc(&p->dimgA, npx));
        AK(alloc(&p->dimgB, npx));
    }
    AK(cudaMemset(p->pslot[0], 0, np * 4));
    AK(cudaMemset(p->pslot[1], 0, np * 4));
    AK(cudaMemset(p->target, 0, npx * 4));
    D.pslot[0] = p->pslot[0];
    D.pslot[1] = p->pslot[1];
    D.F = p->F;
    D.dF = p->dF;
    D.Fv = p->Fv;
    D.dFv = p->dFv;
    D.target = p->target;
    D.img = p->img;
    D.dimg = p->dimg;
    D.imgA = p->imgA;
    D.imgB = p->imgB;
    D.dimgA = p->dimgA;
    D.dimgB = p->dimgB;
    UpdSeg& S = p->seg;
    memset(&S, 0, sizeof S);
    S.pA = p->pslot[0];
    S.pB = p->pslot[1];
    S.F = p->F;
    S.dF = p->dF;
    S.m2f = p->m2f;
    S.m2d = p->m2d;
    S.mean = p->mean;
    S.var = p->var;
    S.ap = p->ap;
    S.mu_f = p->mu_f;
    S.mu_d = p->mu_d;
    S.am = p->am;
    S.av = p->av;
    S.Fv = p->Fv;
    S.dFv = p->dFv;
    S.n = p->n_par;
    S.C = p->C;
    S.prob = p->id;
    S.zero_grads = 0;        // the gradient step clears F and dF right before their scatters
    for (int k = 0; k < 8; ++k) {
        S.lo[k] = p->lo[k];
        S.hi[k] = p->hi[k];
    }
    S.hyper = p->hyper;
#undef AK
    c->probs.push_back(p);
    mer_status s = reset_state(c, p);
    if (!s) s = rebuild_tables(c);
    if (s) {
        c->probs.pop_back();
        for (void* a : p->allocs) dfree(a);
        delete p;
        return s;
    }
    *problem_id = p->id;
    return MER_OK;
}

mer_status mer_params_set(mer_ctx* c, int32_t pid, const float* hwc, int32_t on_device) {
    Problem* p = get_prob(c, pid);
    if (!p) return fail(c, MER_ERR_INVALID_ARG, "bad problem id");
    Guard g(c);
    mer_status s = copy_in(c, p->pslot[0], hwc, p->n_par, on_device);
    if (s) return s;
    CK(c, cudaMemcpyAsync(p->pslot[1], p->pslot[0], p->n_par * 4, cudaMemcpyDeviceToDevice, c->st));
    return reset_state(c, p);
}

mer_status mer_params_get(mer_ctx* c, int32_t pid, float* out, int32_t on_device) {
    Problem* p = get_prob(c, pid);
    if (!p || !out) return fail(c, MER_ERR_INVALID_ARG, "bad problem id or output");
    Guard g(c);
    const int cur = read_cur(c, p);
    CK(c, cudaMemcpyAsync(out, p->pslot[cur], p->n_par * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          c->st));
    if (!on_device) CK(c, cudaStreamSynchronize(c->st));
    return MER_OK;
}

mer_status mer_wait_selftest(double limit_s, double* waited_s) {
    if (!(limit_s > 0.0) || limit_s > 1.0) return fail(nullptr, MER_ERR_INVALID_ARG, "limit must be in (0, 1] s");
    int32_t* d_status = nullptr;
    uint64_t* d_ns = nullptr;
    cudaError_t e = cudaMalloc(&d_status, sizeof(int32_t));
    if (!e) e = cudaMalloc(&d_ns, sizeof(uint64_t));
    if (!e) {
        run_wait_selftest((uint64_t)(limit_s * 1e9), d_status, d_ns, nullptr);
        e = cudaGetLastError();
    }
    int32_t st = MER_ERR_CUDA;
    uint64_t ns = 0;
    if (!e) e = cudaMemcpy(&st, d_status, sizeof st, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(&ns, d_ns, sizeof ns, cudaMemcpyDeviceToHost);
    cudaFree(d_status);
    cudaFree(d_ns);
    if (e) return fail(nullptr, MER_ERR_CUDA, "wait self-test: %s", cudaGetErrorString(e));
    if (waited_s) *waited_s = (double)ns * 1e-9;
    return st;
}

mer_status mer_params_force(mer_ctx* c, int32_t pid, const float* hwc, int32_t on_device) {
    Problem* p = get_prob(c, pid);
    if (!p || !hwc) return fail(c, MER_ERR_INVALID_ARG, "bad problem id or input");
    Guard g(c);
    const int cur = read_cur(c, p);
    mer_status s = copy_in(c, p->pslot[cur], hwc, p->n_par, on_device);
    if (s) return s;
    CK(c, launch_force_step(p->pslot[cur], p->pslot[cur ^ 1], p->n_par, c->d_pstate + p->id, p->hyper, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    return MER_OK;
}

mer_status mer_target_set(mer_ctx* c, int32_t pid, const float* img, int32_t on_device) {
    Problem* p = get_prob(c, pid);
    if (!p) return fail(c, MER_ERR_INVALID_ARG, "bad problem id");
    Guard g(c);
    return copy_in(c, p->target, img, (size_t)p->n_pix * 3, on_device);
}

mer_status mer_target_set_async(mer_ctx* c, int32_t pid, const float* img) {
    Problem* p = get_prob(c, pid);
    if (!p || !img) return fail(c, MER_ERR_INVALID_ARG, "bad arguments to mer_target_set_async");
    Guard g(c);
    CK(c, cudaMemcpyAsync(p->target, img, sizeof(float) * 3 * (size_t)p->n_pix, cudaMemcpyHostToDevice, c->st));
    return MER_OK;
}

mer_status mer_loss_async(mer_ctx* c, int32_t pid, double* loss_host) {
    Problem* p = get_prob(c, pid);
    if (!p || !loss_host) return fail(c, MER_ERR_INVALID_ARG, "bad arguments to mer_loss_async");
    Guard g(c);
    CK(c, cudaMemcpyAsync(loss_host, c->d_loss + p->id, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    return MER_OK;
}

mer_status mer_render(mer_ctx* c, int32_t pid, const float* tex, int32_t spp, uint32_t stream, uint32_t iteration,
                      float* img) {
    Problem* p = get_prob(c, pid);
    if (!p || !img || spp < 1 || stream > MER_STREAM_MAX) return fail(c, MER_ERR_INVALID_ARG, "bad arguments to mer_render");
    Guard g(c);
    const int64_t ch = chunk_spp(c, p, spp);
    for (int64_t s0 = 0; s0 < spp; s0 += ch) {
        const int64_t ns = std::min<int64_t>(ch, spp - s0);
        PassArgs A = single_args(c, p, stream, iteration, spp);
        A.tex_over[0] = tex;
        A.n_paths = ns * p->n_pix;
        A.sample_base = (int32_t)s0;
        pass(c, c->st, A, 1, MODE_PRIMAL, p->max_depth);
        run_resolve(A, 1, img, nullptr, s0 > 0, grid_for(c, 256), c->st);
    }
    CK(c, cudaGetLastError());
    return MER_OK;
}

mer_status mer_target_render(mer_ctx* c, int32_t pid, const float* tex, int32_t spp) {
    Problem* p = get_prob(c, pid);
    if (!p || !tex) return fail(c, MER_ERR_INVALID_ARG, "bad arguments to mer_target_render");
    return mer_render(c, pid, tex, spp, MER_STREAM_TARGET, 0, p->target);
}

mer_status mer_render_samples(mer_ctx* c, int32_t pid, const float* tex, int32_t spp, uint32_t stream,
                              uint32_t iteration, float* out) {
    Problem* p = get_prob(c, pid);
    if (!p || !out || spp < 1 || stream > MER_STREAM_MAX)
        return fail(c, MER_ERR_INVALID_ARG, "bad arguments to mer_render_samples");
    Guard g(c);
    const int64_t ch = chunk_spp(c, p, spp);
    for (int64_t s0 = 0; s0 < spp; s0 += ch) {
        const int64_t ns = std::min<int64_t>(ch, spp - s0);
        PassArgs A = single_args(c, p, stream, iteration, spp);
        A.tex_over[0] = tex;
        A.n_paths = ns * p->n_pix;
        A.sample_base = (int32_t)s0;
        pass(c, c->st, A, 1, MODE_PRIMAL, p->max_depth);
        run_samples_out(A, out, grid_for(c, 256), c->st);
    }
    CK(c, cudaGetLastError());
    return MER_OK;
}

mer_status mer_render_pair(mer_ctx* c, int32_t pid, const float* texA, const float* texB, int32_t spp, uint32_t stream,
                           uint32_t iteration, float* imgA, float* imgB) {
    Problem* p = get_prob(c, pid);
    if (!p || !texA || !texB || !imgA || !imgB || spp < 1 || stream > MER_STREAM_MAX)
        return fail(c, MER_ERR_INVALID_ARG, "bad arguments to mer_render_pair");
    Guard g(c);
    const int64_t ch = chunk_spp(c, p, spp);
    for (int64_t s0 = 0; s0 < spp; s0 += ch) {
        const int64_t ns = std::min<int64_t>(ch, spp - s0);
        PassArgs A = single_args(c, p, stream, iteration, spp);
        A.tex_over[0] = texA;
        A.tex_over[1] = texB;
        A.n_paths = ns * p->n_pix;
        A.sample_base = (int32_t)s0;
        pass(c, c->st, A, 2, MODE_PRIMAL, p->max_depth);
        run_resolve(A, 2, imgA, imgB, s0 > 0, grid_for(c, 256), c->st);
    }
    CK(c, cudaGetLastError());
    return MER_OK;
}

static mer_status adjoint_impl(mer_ctx* c, Problem* p, int nb, const float* texA, const float* texB,
                               const float* dA, const float* dB, int32_t spp, uint32_t stream, uint32_t iteration,
                               float* grad) {
    if ((uintptr_t)grad & 15u) return fail(c, MER_ERR_INVALID_ARG, "gradient output must be 16-byte aligned");
    Guard g(c);
    CK(c, cudaMemsetAsync(grad, 0, sizeof(float) * p->n_par, c->st));
    const int64_t ch = chunk_spp(c, p, spp);
    for (int64_t s0 = 0; s0 < spp; s0 += ch) {
        const int64_t ns = std::min<int64_t>(ch, spp - s0);
        PassArgs A = single_args(c, p, stream, iteration, spp);
        A.tex_over[0] = texA;
        A.tex_over[1] = texB;
        A.dimg_over[0] = dA;
        A.dimg_over[1] = dB;
        A.n_paths = ns * p->n_pix;
        A.sample_base = (int32_t)s0;
        A.lacc = c->w[0].ltot;
        pass(c, c->st, A, nb, MODE_ADJ_FWD, p->max_depth);
        A.lacc = c->w[0].lacc;
        A.ltot = c->w[0].ltot;
        pass(c, c->st, A, nb, MODE_REPLAY, p->max_depth);
        run_scatter(c->w[0].cnt, c->w[0].rec, c->w[0].rcap, c->d_probs, (int)c->probs.size(), grad, 0, grid_for(c, 256),
                    c->st);
    }
    CK(c, cudaGetLastError());
    return MER_OK;
}

mer_status mer_adjoint(mer_ctx* c, int32_t pid, const float* tex, const float* dimg, int32_t spp, uint32_t stream,
                       uint32_t iteration, float* grad) {
    Problem* p = get_prob(c, pid);
    if (!p || !dimg || !grad || spp < 1 || stream > MER_STREAM_MAX)
        return fail(c, MER_ERR_INVALID_ARG, "bad arguments to mer_adjoint");
    return adjoint_impl(c, p, 1, tex, nullptr, dimg, nullptr, spp, stream, iteration, grad);
}

mer_status mer_adjoint_pair(mer_ctx* c, int32_t pid, const float* texA, const float* texB, const float* dA,
                            const float* dB, int32_t spp, uint32_t stream, uint32_t iteration, float* grad) {
    Problem* p = get_prob(c, pid);
    if (!p || !texA || !texB || !dA || !dB || !grad || spp < 1 || stream > MER_STREAM_MAX)
        return fail(c, MER_ERR_INVALID_ARG, "bad arguments to mer_adjoint_pair");
    return adjoint_impl(c, p, 2, texA, texB, dA, dB, spp, stream, iteration, grad);
}

mer_status mer_gradient_step(mer_ctx* c) {
    if (!c || c->probs.empty()) return fail(c, MER_ERR_STATE, "no problems");
    if (c->failed) return fail(c, MER_ERR_STATE, "a kernel ran out of a bounded wait earlier; destroy this context");
    Guard g(c);
    c->launches = enqueue_gradient(c);
    CK(c, cudaGetLastError());
    return MER_OK;
}

mer_status mer_update_step(mer_ctx* c) {
    if (!c || c->probs.empty()) return fail(c, MER_ERR_STATE, "no problems");
    if (c->failed) return fail(c, MER_ERR_STATE, "a kernel ran out of a bounded wait earlier; destroy this context");
    Guard g(c);
    c->launches = enqueue_update(c);
    CK(c, cudaGetLastError());
    return MER_OK;
}

mer_status mer_iterate(mer_ctx* c, int32_t n_iters, int32_t use_graph) {
    if (!c || c->probs.empty()) return fail(c, MER_ERR_STATE, "no problems");
    if (c->failed) return fail(c, MER_ERR_STATE, "a kernel ran out of a bounded wait earlier; destroy this context");
    if (n_iters < 0) return fail(c, MER_ERR_INVALID_ARG, "negative iteration count");
    Guard g(c);
    if (!use_graph) {
        for (int i = 0; i < n_iters; ++i) {
            c->launches = enqueue_gradient(c);
            c->launches += enqueue_update(c);
        }
        CK(c, cudaGetLastError());
        return MER_OK;
    }
    if (c->graph_dirty || !c->gexec) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        KernelTimer* saved_timer = g_timer;
        g_timer = nullptr;   // no event timing inside a captured graph
        CK(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
        int n = enqueue_gradient(c);
        n += enqueue_update(c);
        cudaError_t e = cudaStreamEndCapture(c->st, &graph);
        g_timer = saved_timer;
        if (e) return fail(c, MER_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e) return fail(c, MER_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
        c->launches = n;
        c->graph_dirty = false;
    }
    for (int i = 0; i < n_iters; ++i) CK(c, cudaGraphLaunch(c->gexec, c->st));
    return MER_OK;
}

mer_status mer_grads_get(mer_ctx* c, int32_t pid, float* F_out, float* dF_out, int32_t on_device) {
    Problem* p = get_prob(c, pid);
    if (!p) return fail(c, MER_ERR_INVALID_ARG, "bad problem id");
    Guard g(c);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (F_out) CK(c, cudaMemcpyAsync(F_out, p->F, p->n_par * 4, k, c->st));
    if (dF_out) CK(c, cudaMemcpyAsync(dF_out, p->dF, p->n_par * 4, k, c->st));
    if (!on_device) CK(c, cudaStreamSynchronize(c->st));
    return MER_OK;
}

mer_status mer_stats(mer_ctx* c, int32_t pid, mer_iter_stats* out) {
    Problem* p = get_prob(c, pid);
    if (!p || !out) return fail(c, MER_ERR_INVALID_ARG, "bad problem id or output");
    Guard g(c);
    ProbState ps{};
    double la = 0.0;
    CK(c, cudaMemcpyAsync(&ps, c->d_pstate + pid, sizeof ps, cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaMemcpyAsync(&la, c->d_loss + pid, sizeof la, cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    out->iteration = ps.iteration;
    out->loss = la;
    out->dpi_norm2 = ps.dpi_norm2;
    out->count_f = ps.count_f;
    out->count_d = ps.count_d;
    out->paths_per_iter = (int64_t)p->n_pix * (3 * p->spp_prop + 6 * p->spp_fd);
    return check_err_word(c);
}

mer_status mer_state_get(mer_ctx* c, int32_t pid, mer_state_view* out) {
    Problem* p = get_prob(c, pid);
    if (!p || !out) return fail(c, MER_ERR_INVALID_ARG, "bad problem id or output");
    Guard g(c);
    const int cur = read_cur(c, p);
    out->pi_cur = p->pslot[cur];
    out->pi_prev = p->pslot[cur ^ 1];
    out->F = p->F;
    out->dF = p->dF;
    out->m2f = p->m2f;
    out->m2d = p->m2d;
    out->mean = p->mean;
    out->var = p->var;
    out->alpha_prev = p->ap;
    out->mu_f = p->mu_f;
    out->mu_d = p->mu_d;
    out->adam_m = p->am;
    out->adam_v = p->av;
    out->F_var = p->Fv;
    out->dF_var = p->dFv;
    out->n = p->n_par;
    return MER_OK;
}

mer_status mer_profile_enable(mer_ctx* c, int32_t enable) {
    if (!c || enable < 0 || enable > 2) return fail(c, MER_ERR_INVALID_ARG, "bad arguments");
    cudaSetDevice(c->device);
    if (enable && !c->timer) {
        EventTimer* t = new EventTimer();
        c->timer = t;
        g_timer = t;
    } else if (!enable && c->timer) {
        EventTimer* t = (EventTimer*)c->timer;
        if (g_timer == t) g_timer = nullptr;
        delete t;
        c->timer = nullptr;
    }
    if (enable == 2 && !c->d_stats) {
        CK(c, dalloc(&c->d_stats, 2 * KC_COUNT));
        CK(c, cudaMemset(c->d_stats, 0, sizeof(unsigned long long) * 2 * KC_COUNT));
    }
    c->counting = enable == 2;
    c->graph_dirty = true;
    return MER_OK;
}

mer_status mer_profile_read(mer_ctx* c, mer_kernel_time* out, int32_t max_entries, int32_t* n_out) {
    if (!c || !out || !n_out || max_entries < 0) return fail(c, MER_ERR_INVALID_ARG, "bad arguments");
    if (!c->timer) return fail(c, MER_ERR_STATE, "profiling is not enabled");
    cudaSetDevice(c->device);
    unsigned long long h[2 * KC_COUNT] = {0};
    if (c->counting && c->d_stats) {
        CK(c, cudaStreamSynchronize(c->st));
        CK(c, cudaMemcpy(h, c->d_stats, sizeof h, cudaMemcpyDeviceToHost));
        CK(c, cudaMemset(c->d_stats, 0, sizeof h));
    }
    int n = 0;
    ((EventTimer*)c->timer)->read(out, max_entries, &n, c->counting ? h : nullptr);
    *n_out = n;
    return MER_OK;
}

mer_status mer_launch_count(mer_ctx* c, int64_t* out) {
    if (!c || !out) return fail(c, MER_ERR_INVALID_ARG, "null argument");
    *out = c->launches;
    return MER_OK;
}

mer_status mer_precondition(int32_t C, int32_t H, int32_t W, float lambda, float* g, void* stream) {
    if (C < 1 || C > MER_MAX_CHANNELS || H < 1 || W < 1 || H > 4094 || W > 4094 || !g || !(lambda >= 0.0f) ||
        !std::isfinite(lambda))
        return fail(nullptr, MER_ERR_INVALID_ARG, "bad arguments to mer_precondition");
    if (lambda == 0.0f) return MER_OK;
    Precond pc;
    cudaError_t e = precond_init(pc, C, H, W, lambda);
    if (!e) {
        precond_apply(pc, g, (cudaStream_t)stream);
        e = cudaGetLastError();
    }
    if (!e) e = cudaStreamSynchronize((cudaStream_t)stream);
    precond_free(pc);
    if (e) return fail(nullptr, MER_ERR_CUDA, "mer_precondition: %s", cudaGetErrorString(e));
    return MER_OK;
}

mer_status mer_philox(uint32_t k0, uint32_t k1, const uint32_t* ctr, int64_t n, uint32_t* out, void* stream) {
    if (n < 0 || (n > 0 && (!ctr || !out))) return fail(nullptr, MER_ERR_INVALID_ARG, "bad arguments to mer_philox");
    run_philox(k0, k1, ctr, n, out, (cudaStream_t)stream);
    const cudaError_t e = cudaGetLastError();
    if (e) return fail(nullptr, MER_ERR_CUDA, "mer_philox: %s", cudaGetErrorString(e));
    return MER_OK;
}

// --------------------------------------------------------------------------------------
// standalone update: scratch for the per-block partial norms is owned by the library,
// one growing buffer per device
// --------------------------------------------------------------------------------------
static std::mutex g_scratch_mu;
static std::vector<std::pair<double*, int64_t>> g_scratch;   // per device

mer_status mer_meta_step_raw(const mer_hyper* hyper, int64_t n, int32_t C, const float* lo, const float* hi,
                             const float* pi, float* pi_next, float* F, float* dF, float* m2f, float* m2d, float* mean,
                             float* var, float* alpha_prev, int32_t iteration, int32_t count_f, int32_t count_d,
                             double dpi_norm2, int32_t zero_grads, double* out, void* stream) {
    mer_update_arrays A;
    memset(&A, 0, sizeof A);
    A.pi = pi; A.pi_next = pi_next; A.F = F; A.dF = dF; A.m2f = m2f; A.m2d = m2d; A.mean = mean; A.var = var;
    A.alpha_prev = alpha_prev;
    return mer_meta_step_raw_ex(hyper, n, C, lo, hi, &A, iteration, count_f, count_d, dpi_norm2, zero_grads, out,
                                stream);
}

mer_status mer_meta_step_raw_ex(const mer_hyper* hyper, int64_t n, int32_t C, const float* lo, const float* hi,
                                const mer_update_arrays* arrays, int32_t iteration, int32_t count_f,
                                int32_t count_d, double dpi_norm2, int32_t zero_grads, double* out, void* stream) {
    UpdSeg S;
    if (const char* why = raw_update_seg(hyper, n, C, lo, hi, arrays, zero_grads, out, &S))
        return fail(nullptr, MER_ERR_INVALID_ARG, "mer_meta_step_raw: %s", why);
    const int64_t nb = update_blocks_for(n);
    int dev = 0;
    cudaGetDevice(&dev);
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if ((int)g_scratch.size() <= dev) g_scratch.resize(dev + 1, {nullptr, 0});
        auto& sl = g_scratch[dev];
        if (sl.second < std::max<int64_t>(nb, 1)) {
            if (sl.first) {
                cudaDeviceSynchronize();
                cudaFree(sl.first);
            }
            sl.first = nullptr;
            sl.second = 0;
            const int64_t want = std::max<int64_t>(nb, 1024);
            if (cudaMalloc(&sl.first, sizeof(double) * want) != cudaSuccess)
                return fail(nullptr, MER_ERR_OOM, "scratch allocation failed");
            sl.second = want;
        }
        scratch = sl.first;
    }
    const cudaError_t e = launch_update_raw(S, iteration, count_f, count_d, dpi_norm2, scratch, nb, out,
                                            (cudaStream_t)stream);
    if (e) return fail(nullptr, MER_ERR_CUDA, "mer_meta_step_raw: %s", cudaGetErrorString(e));
    return MER_OK;
}

// --------------------------------------------------------------------------------------
// checkpoint: per problem ProbState + the nine parameter-shaped arrays (+ the variant state
// its flags allocate)
// --------------------------------------------------------------------------------------
static std::vector<float*> ckpt_arrays(Problem* p) {
    std::vector<float*> v = {p->pslot[0], p->pslot[1], p->F, p->dF, p->m2f, p->m2d, p->mean, p->var, p->ap};
    for (float* a : {p->mu_f, p->mu_d, p->am, p->av, p->Fv, p->dFv})
        if (a) v.push_back(a);
    return v;
}

mer_status mer_checkpoint_save(mer_ctx* c, void* buf, size_t* len) {
    if (!c || !len) return fail(c, MER_ERR_INVALID_ARG, "null argument");
    size_t need = sizeof(uint64_t) * 2;
    for (Problem* p : c->probs) need += sizeof(ProbState) + ckpt_arrays(p).size() * sizeof(float) * (size_t)p->n_par;
    if (!buf) {
        *len = need;
        return MER_OK;
    }
    if (*len < need) return fail(c, MER_ERR_INVALID_ARG, "checkpoint buffer too small (%zu < %zu)", *len, need);
    Guard g(c);
    char* w = (char*)buf;
    const uint64_t hdr[2] = {0x4d4552434b505431ull, (uint64_t)c->probs.size()};
    memcpy(w, hdr, sizeof hdr);
    w += sizeof hdr;
    for (Problem* p : c->probs) {
        CK(c, cudaMemcpyAsync(w, c->d_pstate + p->id, sizeof(ProbState), cudaMemcpyDeviceToHost, c->st));
        w += sizeof(ProbState);
        for (float* a : ckpt_arrays(p)) {
            CK(c, cudaMemcpyAsync(w, a, sizeof(float) * p->n_par, cudaMemcpyDeviceToHost, c->st));
            w += sizeof(float) * p->n_par;
        }
    }
    CK(c, cudaStreamSynchronize(c->st));
    *len = need;
    return MER_OK;
}

mer_status mer_checkpoint_load(mer_ctx* c, const void* buf, size_t len) {
    if (!c || !buf) return fail(c, MER_ERR_INVALID_ARG, "null argument");
    size_t need = sizeof(uint64_t) * 2;
    for (Problem* p : c->probs) need += sizeof(ProbState) + ckpt_arrays(p).size() * sizeof(float) * (size_t)p->n_par;
    uint64_t hdr[2];
    if (len < sizeof hdr) return fail(c, MER_ERR_INVALID_ARG, "checkpoint too short");
    memcpy(hdr, buf, sizeof hdr);
    if (hdr[0] != 0x4d4552434b505431ull || hdr[1] != c->probs.size() || len != need)
        return fail(c, MER_ERR_INVALID_ARG, "checkpoint does not match this context's problems");
    Guard g(c);
    const char* r = (const char*)buf + sizeof hdr;
    for (Problem* p : c->probs) {
        CK(c, cudaMemcpyAsync(c->d_pstate + p->id, r, sizeof(ProbState), cudaMemcpyHostToDevice, c->st));
        r += sizeof(ProbState);
        for (float* a : ckpt_arrays(p)) {
            CK(c, cudaMemcpyAsync(a, r, sizeof(float) * p->n_par, cudaMemcpyHostToDevice, c->st));
            r += sizeof(float) * p->n_par;
        }
    }
    CK(c, cudaStreamSynchronize(c->st));
    return MER_OK;
}

mer_status mer_autotune(mer_ctx* c, int32_t trial_iters, char* desc, size_t desc_len) {
    if (!c || c->probs.empty()) return fail(c, MER_ERR_STATE, "no problems");
    if (trial_iters < 1) trial_iters = 1;
    // candidates: block size x blocks per SM x shared-memory node staging
    const int blocks[] = {64, 128, 256};   // <= the kernels' launch bounds
    const int per_sm[] = {2, 4, 8, 16};
    const int smem[] = {0, 128, 512};   // 128-byte nodes: 16 KB, 64 KB
    // every trial runs full iterations on a checkpoint of the state, restored afterwards
    size_t len = 0;
    mer_status s = mer_checkpoint_save(c, nullptr, &len);
    if (s) return s;
    std::vector<char> saved(len);
    s = mer_checkpoint_save(c, saved.data(), &len);
    if (s) return s;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    LaunchShape best_shape = c->shape;
    int best_per_sm = c->cfg.blocks_per_sm;
    for (int b : blocks)
        for (int ps : per_sm)
            for (int sm : smem) {
                if (b * ps > 2048) continue;
                if (sm > 0 && (set_trace_smem_limits(sm) != cudaSuccess)) continue;
                c->shape.block = b;
                c->shape.smem_nodes = sm;
                c->cfg.blocks_per_sm = ps;
                c->graph_dirty = true;
                // warm-up (also captures the graph); a shape that fails is skipped
                if (mer_iterate(c, 1, 1)) {
                    mer_checkpoint_load(c, saved.data(), saved.size());
                    continue;
                }
                cudaEventRecord(e0, c->st);
                const mer_status ts = mer_iterate(c, trial_iters, 1);
                cudaEventRecord(e1, c->st);
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ts == MER_OK && cudaGetLastError() == cudaSuccess && ms < best) {
                    best = ms;
                    best_shape = c->shape;
                    best_per_sm = ps;
                }
                mer_checkpoint_load(c, saved.data(), saved.size());
            }
    // then the traversal's refill threshold at the best shape
    c->shape = best_shape;
    c->cfg.blocks_per_sm = best_per_sm;
    for (int rf : {4, 8, 16, 24}) {
        c->shape.refill = rf;
        c->graph_dirty = true;
        if (mer_iterate(c, 1, 1)) {
            mer_checkpoint_load(c, saved.data(), saved.size());
            continue;
        }
        cudaEventRecord(e0, c->st);
        const mer_status ts = mer_iterate(c, trial_iters, 1);
        cudaEventRecord(e1, c->st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ts == MER_OK && cudaGetLastError() == cudaSuccess && ms < best) {
            best = ms;
            best_shape.refill = rf;
        }
        mer_checkpoint_load(c, saved.data(), saved.size());
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->shape = best_shape;
    c->cfg.blocks_per_sm = best_per_sm;
    c->graph_dirty = true;
    if (desc && desc_len)
        snprintf(desc, desc_len, "block=%d blocks_per_sm=%d smem_nodes=%d refill=%d ms_per_iter=%.4f",
                 best_shape.block, best_per_sm, best_shape.smem_nodes, best_shape.refill, best / trial_iters);
    return mer_checkpoint_load(c, saved.data(), saved.size());
}

}  // extern "C"

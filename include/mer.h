/*
 * mer.h — C ABI of the GB300 library for meta-estimated inverse path tracing.
 *
 * Implements the data-parallel hot path of "Joint Sampling and Optimisation for
 * Inverse Rendering" (Balint, Myszkowski, Seidel, Singh; SIGGRAPH Asia 2023):
 * Monte Carlo estimation of texture gradients of an image loss by path tracing with
 * Path Replay Backpropagation (Sec. 6 setup), in two kinds — proportional samples
 * <F_i> (Sec. 3, Eq. est_def) and finite-difference samples <dF_i> that replay the
 * same random numbers at pi_i and pi_{i-1} (Sec. 3, Eq. est_triv) — feeding the
 * variance-weighted meta-estimator (Eqs. recurrent_meta, alpha, varest, vardiff,
 * varmeta, alpha_clip_2) and its update rule replacing Adam's moments (Sec. 5).
 *
 * Conventions for every entry point:
 *  - Every call returns a mer_status and never throws across the ABI. On failure
 *    mer_last_error(ctx) gives a message (context-free calls: mer_last_error(NULL)).
 *  - "device" pointers are CUDA device addresses on the context's device; they are
 *    borrowed for the duration of the call (including its asynchronous GPU work on
 *    the context stream). "host" pointers are read or written before the call returns.
 *  - Work is enqueued on the stream given at mer_create (or the stream argument of
 *    the context-free calls) and is asynchronous unless stated otherwise.
 *  - Textures / parameters are HWC float32: element (y, x, c) at (y*W + x)*C + c,
 *    with C = 3 (Lambert albedo RGB) or C = 5 (base colour RGB, metalness, roughness).
 *  - Images are row-major float32 RGB: pixel (py, px) at (py*width + px)*3.
 *  - Random numbers: Philox4x32-10 with key (seed, key_id) and counter
 *    (pixel, sample, iteration, stream<<16 | vertex<<4 | block); uniforms are
 *    (x >> 8) * 2^-24. Streams: MER_STREAM_*.
 *
 * Steps of one iteration, as the comments below number them:
 *  a1 Philox streams; a2 camera rays; a3 BVH traversal and intersection; a4 surface
 *  interaction (texture fetch, BSDF parameters); a5 next-event estimation with MIS; a6 BSDF
 *  sample and continuation; a7 image and loss adjoint; a8 path-replay adjoint; a9 the FD pair
 *  at pi_i and pi_{i-1}; a10 scatter of texel gradients; a11 the fused update; a12 batching of
 *  problems and graph capture of the iteration.
 */
#ifndef MER_H
#define MER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int mer_status;
#define MER_OK 0
#define MER_ERR_INVALID_ARG 1
#define MER_ERR_CUDA 2
#define MER_ERR_OOM 3
#define MER_ERR_TIMEOUT 4
#define MER_ERR_BOUNDS 5
#define MER_ERR_STATE 6
#define MER_ERR_NAN 7

/* optimiser of a problem */
#define MER_MODE_META 0  /* meta-estimator + its update rule (Sec. 5): 1 FD + spp_prop proportional */
#define MER_MODE_ADAM 1  /* plain fresh-sample gradients with Adam (Sec. 5, Eqs. adam_*) */

/* Philox stream ids (fourth counter word, bits 16..31) */
#define MER_STREAM_PROP_PRIMAL 0u /* primal image used for the proportional sample's loss adjoint */
#define MER_STREAM_PROP_ADJ 1u    /* proportional sample's path replay */
#define MER_STREAM_FD_PRIMAL 2u   /* primal image pair of the FD sample (same numbers at pi_i, pi_{i-1}) */
#define MER_STREAM_FD_ADJ 3u      /* adjoint pair of the FD sample */
#define MER_STREAM_TARGET 4u      /* target rendering */
#define MER_STREAM_EVAL 5u        /* loss evaluation renders */
/* MER_META_UNCORRELATED draws its independent variance samples from the four gradient streams
 * shifted by this offset (streams 8..11) */
#define MER_STREAM_VAR_OFFSET 8u
/* largest stream id a caller may pass (the id fills the counter word's upper 16 bits); larger ids
 * give MER_ERR_INVALID_ARG */
#define MER_STREAM_MAX 0xFFFFu

/* Image loss of step a7 (N pixels, 3 channels, target T, image I):
 *  L2    L = 1/(3N) sum (I - T)^2,               dL/dI = 2 (I - T) / (3N)
 *  MRSE  L = 1/(3N) sum (I - T)^2 / (T^2 + 0.01), dL/dI = 2 (I - T) / ((T^2 + 0.01) 3N)
 *        (the relative loss of Sec. 6's setup, normalised by the target only, so that the
 *        adjoint stays linear in the independent primal image) */
#define MER_LOSS_L2 0
#define MER_LOSS_MRSE 1

#define MER_MAX_CHANNELS 5
#define MER_MAX_DEPTH 16
#define MER_MAX_PROBLEMS 256

/* Hyper-parameters of one problem's optimiser. Defaults (mer_hyper_default):
 * lr 0.01, beta_f 0.99, beta_d 0.9 (Sec. 4.1 "large beta_F", Sec. 4.2 "small beta_D"),
 * eps 1e-8 and eps_alpha 1e-30 (appendix pseudocode), beta1 0.9 / beta2 0.999 (Adam). */
/* Variants of the META update (bits of mer_hyper.flags; 0 = the method as stated):
 *  PER_ELEMENT   the step size of Sec. 4.2 read per element, |pi_i - pi_{i-1}| (the appendix
 *                loop writes sqrt(dpi_i^2)), instead of the Euclidean norm of the problem's
 *                step; an element whose own step was zero keeps Var_D and adds Var[<dF>] = 0
 *  NO_CLIP       Eq. alpha_clip_2 not applied (ablation "alpha clipping", Sec. 6)
 *  CENTRED       non-zero-centred variances max(m2 - mu^2, 0), mu a start-up-corrected EMA of
 *                the sample beside each Moment2 (ablation "zero-centred EMAs", Sec. 6)
 *  GROWING_BETA  beta_F of the k-th Var[<F>] step grown as max(beta_F, k/(k+1)), start-up
 *                correction (1 - beta_k) / (1 - prod_{j<=k} beta_j) (appendix A)
 *  NAIVE_ADAM    <F_i>_M fed to Adam's moments (beta1, beta2, bias-corrected) instead of the
 *                update rule of Sec. 5 (the naive coupling Sec. 5 argues against)
 *  UNCORRELATED  Var[<F>] and Var[<dF>]_D stepped with independent samples F_var, dF_var of
 *                the same estimators (ablation "sample reuse", Sec. 6); <F_i>_M still uses F, dF
 *  FD_SHARED_PATH  the FD sample of Eq. est_triv read literally: the pi_{i-1} branch follows the
 *                path sampled at pi_i (directions, lobe choices, light samples) and divides its
 *                integrand by that path's density and MIS weights, instead of replaying the same
 *                random numbers with its own sampling; identical to the replay wherever sampling
 *                does not depend on the parameters (e.g. Lambertian albedo) */
#define MER_META_PER_ELEMENT 1
#define MER_META_NO_CLIP 2
#define MER_META_CENTRED 4
#define MER_META_GROWING_BETA 8
#define MER_META_NAIVE_ADAM 16
#define MER_META_UNCORRELATED 32
#define MER_META_FD_SHARED_PATH 64

typedef struct mer_hyper {
    int32_t mode;      /* MER_MODE_META or MER_MODE_ADAM */
    float lr;          /* eta */
    float beta_f;      /* EMA decay of Var[<F_i>]   (Eq. varest) */
    float beta_d;      /* EMA decay of Var[<dF_i>]_D (Sec. 4.2) */
    float eps;         /* step epsilon (update rule of Sec. 5) */
    float eps_alpha;   /* added to the alpha denominator (appendix pseudocode) */
    float beta1;       /* Adam first moment */
    float beta2;       /* Adam second moment */
    int32_t flags;     /* MER_META_* variant bits (META mode only; 0 = as stated) */
    float precond_lambda; /* > 0: texture gradients (F, dF and any variance samples) are replaced by
                           * (I + lambda L)^{-1} g per channel before the update, L the Neumann graph
                           * Laplacian of the texel grid (the gradient preconditioning of the
                           * experiments of Sec. 6, after Nicolet et al. 2021); 0 = off */
} mer_hyper;

/* Scene of one problem. All arrays are HOST arrays, copied by mer_scene_add (the caller
 * keeps ownership). Triangles index shared vertices; quads are parallelogram area lights
 * (p0, e1, e2, Le; emitting on the side of e1 x e2) whose geometry must also be present as
 * triangles carrying the light's index in tri_light. */
typedef struct mer_scene_desc {
    int32_t n_verts, n_tris;
    const float* positions;   /* [n_verts][3] */
    const float* uvs;         /* [n_verts][2] */
    const int32_t* tris;      /* [n_tris][3] vertex indices */
    const int32_t* tri_mat;   /* [n_tris] material index */
    const int32_t* tri_light; /* [n_tris] quad-light index or -1 */
    int32_t n_spheres;
    const float* spheres;     /* [n_spheres][8]: centre xyz, radius, u0, u1, v0, v1 (uv rectangle) */
    const int32_t* sph_mat;   /* [n_spheres] */
    int32_t n_mats;
    const int32_t* mat_type;  /* [n_mats] 0 Lambert, 1 principled */
    const int32_t* mat_textured; /* [n_mats] 1: parameters from the problem's texture */
    const float* mat_const;   /* [n_mats][5] parameters of untextured materials */
    int32_t n_quads;
    const float* quads;       /* [n_quads][12]: p0, e1, e2, Le */
    int32_t has_env;
    float env[3];             /* constant environment radiance */
    float eye[3], target[3], up[3];
    float fov_deg;            /* vertical field of view, degrees in (0, 180); eye != target and up not
                               * parallel to target - eye, else MER_ERR_INVALID_ARG */
    int32_t width, height;
    int32_t tex_c, tex_h, tex_w; /* parameter texture shape: C in {3, 5}, 1..4094 texels per side
                                  * (a gradient record packs texel coordinates in 12 bits);
                                  * otherwise MER_ERR_INVALID_ARG */
    float clamp_lo[8], clamp_hi[8]; /* per-channel parameter range applied after each step */
    int32_t max_depth;        /* path segments (1 = emitters only, 2 = direct light) */
    int32_t spp_prop, spp_fd; /* samples per pixel and iteration */
    uint32_t seed, key_id;    /* Philox key */
    int32_t loss;             /* MER_LOSS_* image loss of step a7 (0 = L2) */
    mer_hyper hyper;
} mer_scene_desc;

typedef struct mer_config {
    int32_t device;           /* CUDA device ordinal */
    int32_t block_size;       /* threads per block of the wavefront kernels (0 = default 128) */
    int32_t blocks_per_sm;    /* persistent-grid occupancy target (0 = default) */
    int32_t smem_nodes;       /* BVH nodes staged in shared memory per block (0 = off) */
    int64_t max_paths;        /* capacity hint for path queues (0 = size from the scenes) */
    /* 0 (default): the iteration's replays regenerate every path from its counters and trace its
     * rays again, so no per-vertex state outlives a kernel (path replay as the checkpointing,
     * Sec. 6 setup: PRB). 1: a variant in which the PRB radiance passes keep each path vertex's
     * closest hit and NEE visibility (16 B + 1 B per vertex and branch) and the replays read them
     * instead of tracing (same hits, no traversal launches in the replays). The estimates are the
     * same either way; mer_adjoint and mer_adjoint_pair always re-trace. */
    int32_t replay_hit_store;
    /* traversal launches: a warp's idle lanes take new rays once at least this many of its 32
     * lanes are idle (1..32; 0 = default 8; mer_autotune picks it) */
    int32_t trace_refill;
} mer_config;

typedef struct mer_iter_stats {
    int64_t iteration;        /* optimisation iterations completed */
    double loss;              /* L2 loss of the last proportional primal image */
    double dpi_norm2;         /* ||pi_i - pi_{i-1}||^2 of the last applied step */
    int32_t count_f, count_d; /* Moment2 step counts of Var[<F>] and Var[<dF>]_D */
    int64_t paths_per_iter;   /* path traversals of one iteration (all passes) */
} mer_iter_stats;

typedef struct mer_ctx mer_ctx;

/* Default hyper-parameters (see mer_hyper). Host-only, never fails. */
mer_status mer_hyper_default(mer_hyper* out);

/* Create a context on cfg->device that enqueues on cuda_stream (a cudaStream_t; NULL =
 * legacy default stream). Owns all device buffers it allocates. */
mer_status mer_create(const mer_config* cfg, void* cuda_stream, mer_ctx** out);
void mer_destroy(mer_ctx* ctx);
/* Last error message of ctx (or of the calling thread's context-free calls if ctx is NULL).
 * Never NULL. */
const char* mer_last_error(const mer_ctx* ctx);

/* Add one inverse-rendering problem: copies the scene, builds its BVH on the host (binned
 * SAH) and uploads it; parameters start at zero and the optimiser state is reset. Returns
 * its id in *problem_id (0, 1, ... in call order). Synchronous. */
mer_status mer_scene_add(mer_ctx* ctx, const mer_scene_desc* desc, int32_t* problem_id);

/* Set the parameters pi_0 = pi_{-1} of a problem from an HWC texture (host or device
 * pointer per on_device) and reset its optimiser state to iteration 0. */
mer_status mer_params_set(mer_ctx* ctx, int32_t pid, const float* hwc, int32_t on_device);
/* Copy the current parameters pi_i out (host pointer: synchronous; device: asynchronous). */
mer_status mer_params_get(mer_ctx* ctx, int32_t pid, float* hwc_out, int32_t on_device);
/* ---- Emissive-absorptive volume (the high-dimensional experiment of Sec. 6) ----
 * A voxel grid of emission (RGB) and density over the box [lo, hi], seen from n_views pinhole
 * cameras (width x height each; images stacked view-major, RGB fp32) and rendered by a jittered
 * ray march: L = sum_k T_k (1 - exp(-sigma_k * step)) e_k + T_end * background with
 * T_{k+1} = T_k exp(-sigma_k * step); sample k at t0 + (k + u) * step, u one Philox uniform per ray
 * (vertex 1; the pixel jitter is vertex 0), samples past the box exit skipped. Parameters: device
 * float4 per voxel (emission RGB, density) at ((z * ny + y) * nx + x), 16-byte aligned; trilinear
 * interpolation, clamp-to-edge, voxel centres at (i + 1/2) / n across the box. Pixel index =
 * view * width * height + y * width + x; counters as for surfaces (pixel, sample, iteration,
 * stream). */
typedef struct mer_volume_desc {
    int32_t nx, ny, nz;
    float lo[3], hi[3];
    int32_t n_views, width, height;
    const float* cameras;     /* HOST [n_views][10]: eye xyz, target xyz, up xyz, fov_deg (vertical,
                               * in (0, 180)); a degenerate camera gives MER_ERR_INVALID_ARG */
    float step;               /* march step, world units (> 0) */
    float background[3];
    uint32_t seed, key_id;    /* Philox key */
} mer_volume_desc;
typedef struct mer_volume mer_volume;
mer_status mer_volume_create(const mer_volume_desc* desc, int32_t device, mer_volume** out);
void mer_volume_destroy(mer_volume* vol);
/* img_dev [n_views * height * width * 3] = mean over spp samples (asynchronous on cuda_stream) */
mer_status mer_volume_render(mer_volume* vol, const float* params_dev, int32_t spp, uint32_t stream,
                             uint32_t iteration, float* img_dev, void* cuda_stream);
/* grad_dev (voxel float4s, caller-zeroed) += d/dparams of sum_p dimg[p] . I_p by replay of the
 * same counters: a radiance pass that records (sigma_k, dimg . e_k) per march step into a buffer
 * the volume owns (allocated on the first call, 8 B per step of each ray in flight; so adjoint
 * calls and optimiser iterations on one volume must be ordered on one stream or synchronised),
 * then the replay from those records */
mer_status mer_volume_adjoint(mer_volume* vol, const float* params_dev, const float* dimg_dev, int32_t spp,
                              uint32_t stream, uint32_t iteration, float* grad_dev, void* cuda_stream);
/* FD pair (Eq. est_triv): the same counters at paramsA and paramsB; grad_dev += g_A - g_B */
mer_status mer_volume_adjoint_pair(mer_volume* vol, const float* paramsA_dev, const float* paramsB_dev,
                                   const float* dimgA_dev, const float* dimgB_dev, int32_t spp, uint32_t stream,
                                   uint32_t iteration, float* grad_dev, void* cuda_stream);
/* Image loss of n_pix RGB pixels (MER_LOSS_L2 or MER_LOSS_MRSE, as in step a7): *loss_dev (device
 * double) = the loss, dimg_dev = dLoss/dimg. */
mer_status mer_image_loss(int32_t kind, int64_t n_pix, const float* img_dev, const float* target_dev,
                          float* dimg_dev, double* loss_dev, void* cuda_stream);

/* Failure detection of the bounded waits (the scatter's record staging waits on shared-memory
 * barriers with a wall-time limit and reports MER_ERR_TIMEOUT instead of hanging): runs one
 * such wait on a barrier that nothing completes, with limit_s in (0, 1] seconds, on the current
 * device. Returns MER_ERR_TIMEOUT when the wait gave up as designed (MER_OK would mean the
 * barrier completed); *waited_s receives how long it waited. The paper has no counterpart. */
mer_status mer_wait_selftest(double limit_s, double* waited_s);

/* Replaces pi_{i+1}, the parameters the last update step produced, by the caller's values (HWC,
 * host or device) and sets ||pi_{i+1} - pi_i||^2 and the next update's coefficients from them,
 * so that the estimators run along a prescribed parameter trajectory instead of the optimiser's
 * (the experiments of Sec. 6 "variance reduction without lag" and "approximation accuracy" move
 * the parameters along a fixed schedule without an optimiser). The meta-estimator state, the
 * Moment2 counts and the iteration are left as they are. Synchronous. */
mer_status mer_params_force(mer_ctx* ctx, int32_t pid, const float* hwc, int32_t on_device);
/* Set the target image ([height][width][3]). */
mer_status mer_target_set(mer_ctx* ctx, int32_t pid, const float* img, int32_t on_device);
/* Asynchronous forms for a host loop that keeps steps in flight (both enqueue on the context
 * stream, fenced to the caller's stream, and return at once):
 *  mer_target_set_async: target from host memory img_host ([height][width][3], page-locked for
 *    the copy to be asynchronous), which must stay unchanged until the context's work up to this
 *    call has completed;
 *  mer_loss_async: *loss_host (host memory, page-locked) receives the problem's loss of its last
 *    gradient step once the context's work up to this call has completed. */
mer_status mer_target_set_async(mer_ctx* ctx, int32_t pid, const float* img_host);
mer_status mer_loss_async(mer_ctx* ctx, int32_t pid, double* loss_host);
/* Render the target image from the given parameters (device HWC texture) with spp samples
 * of stream MER_STREAM_TARGET at iteration 0, and store it as the target. */
mer_status mer_target_render(mer_ctx* ctx, int32_t pid, const float* tex_dev, int32_t spp);

/* Primal render of problem pid with the device texture tex_dev (NULL = current parameters):
 * img_dev[p] = (1/spp) sum_s L(pixel p, sample s) with counters (p, s, iteration, stream). */
mer_status mer_render(mer_ctx* ctx, int32_t pid, const float* tex_dev, int32_t spp, uint32_t stream,
                      uint32_t iteration, float* img_dev);
/* Per-sample radiance: out_dev[(s*n_pix + p)*3 + c] for s < spp. */
mer_status mer_render_samples(mer_ctx* ctx, int32_t pid, const float* tex_dev, int32_t spp, uint32_t stream,
                              uint32_t iteration, float* out_dev);
/* Adjoint of mer_render by path replay: grad_dev (texture-shaped, overwritten) =
 * d/dtex sum_p sum_c dimg_dev[p,c] * img[p,c], where img is the render with the same
 * (tex, spp, stream, iteration). Paths are recomputed from their counters (no stored vertices). */
mer_status mer_adjoint(mer_ctx* ctx, int32_t pid, const float* tex_dev, const float* dimg_dev, int32_t spp,
                       uint32_t stream, uint32_t iteration, float* grad_dev);
/* FD pair of Eq. est_triv for one problem: grad_dev = d/dtex J(texA) - d/dtex J(texB) where both
 * terms replay the same counters; dimgA/dimgB are the adjoint images of each side. */
mer_status mer_adjoint_pair(mer_ctx* ctx, int32_t pid, const float* texA_dev, const float* texB_dev,
                            const float* dimgA_dev, const float* dimgB_dev, int32_t spp, uint32_t stream,
                            uint32_t iteration, float* grad_dev);
/* The two primal images of the FD pair (same counters at texA and texB). */
mer_status mer_render_pair(mer_ctx* ctx, int32_t pid, const float* texA_dev, const float* texB_dev,
                           int32_t spp, uint32_t stream, uint32_t iteration, float* imgA_dev, float* imgB_dev);

/* Steps a1-a10 of one iteration for every problem: the proportional gradient <F_i> and (META
 * problems, iteration >= 1) the FD gradient <dF_i>, accumulated into the context's F and dF,
 * each cleared right before its scatter (after the call they hold this step's gradients). */
mer_status mer_gradient_step(mer_ctx* ctx);
/* Copy a problem's current F and dF (texture-shaped) out (host: synchronous). */
mer_status mer_grads_get(mer_ctx* ctx, int32_t pid, float* F_out, float* dF_out, int32_t on_device);
/* Step a11 for every problem: the fused meta-estimator (or Adam) update, pi_{i+1} written over
 * pi_{i-1}, ||pi_{i+1} - pi_i||^2 reduced, iteration advanced. F and dF are left as they are
 * (the next gradient step clears them). */
mer_status mer_update_step(mer_ctx* ctx);
/* n_iters full iterations (gradient + update) of all problems; use_graph = 1 replays one
 * captured CUDA graph per iteration (captured on first use). */
mer_status mer_iterate(mer_ctx* ctx, int32_t n_iters, int32_t use_graph);
/* Statistics of a problem (synchronous). Also reads the kernels' error word: a capacity overrun
 * returns MER_ERR_BOUNDS and a bounded wait that ran out MER_ERR_TIMEOUT. After MER_ERR_TIMEOUT
 * the context's results can no longer be trusted (a scatter block may have left with copies in
 * flight), and mer_gradient_step, mer_update_step and mer_iterate refuse it (MER_ERR_STATE):
 * destroy the context. */
mer_status mer_stats(mer_ctx* ctx, int32_t pid, mer_iter_stats* out);

/* Optimiser state of a problem (parameter-shaped device arrays owned by the context) for
 * inspection and tests: pi_cur, pi_prev, F, dF, m2f, m2d, mean, var, alpha_prev. */
typedef struct mer_state_view {
    float *pi_cur, *pi_prev, *F, *dF, *m2f, *m2d, *mean, *var, *alpha_prev;
    /* variant state, NULL unless the problem's flags need it: CENTRED first moments, NAIVE_ADAM
     * moments, UNCORRELATED variance samples */
    float *mu_f, *mu_d, *adam_m, *adam_v, *F_var, *dF_var;
    int64_t n;                /* parameters of the problem (H*W*C) */
} mer_state_view;
mer_status mer_state_get(mer_ctx* ctx, int32_t pid, mer_state_view* out);

/* Standalone fused update of step a11 over n parameters (one problem), every array a device
 * array of n floats; pi_next may not alias pi. Per element: Var[<F>] Moment2 step (Eq. varest
 * with start-up correction count_f+1), if iteration >= 1 and dpi_norm2 > 0 the Var[<dF>]_D
 * Moment2 step of dF/||dpi|| (count_d+1) and Var[<dF>] = m2d*dpi_norm2 (Eq. vardiff), then the
 * meta-estimator of the appendix pseudocode (Eqs. recurrent_meta, alpha, alpha_clip_2, varmeta)
 * and the update dpi = -lr*mean/(sqrt(var)+eps), clamped channel-wise (channel = index % C) to
 * [lo[c], hi[c]]. ADAM mode uses mean/var as Adam's m/v and iteration+1 as its step count.
 * zero_grads = 1 clears F and dF. *dpi_norm2_out (device double) receives ||pi_next - pi||^2.
 * Variant flags without arrays of their own work here (PER_ELEMENT, with pi_next holding pi_{i-1}
 * on entry; NO_CLIP; GROWING_BETA); CENTRED, NAIVE_ADAM and UNCORRELATED are rejected
 * (MER_ERR_INVALID_ARG): use mer_meta_step_raw_ex.
 * Scratch: the per-block partial sums of the deterministic norm reduction go to one buffer per
 * device that the library owns and shares between all calls of mer_meta_step_raw and
 * mer_meta_step_raw_ex on that device (n/4096 doubles, grown on demand). Calls ordered on one
 * stream are safe; calls that overlap on the GPU (different streams with no ordering between
 * them) race on it and give wrong norms. Growing it (a call with a larger n than any before on
 * this device) synchronises the device and frees the old buffer, so a caller that must not
 * allocate or synchronise uses mer_meta_step_raw_noalloc. */
mer_status mer_meta_step_raw(const mer_hyper* hyper, int64_t n, int32_t C, const float* lo, const float* hi,
                             const float* pi, float* pi_next, float* F, float* dF, float* m2f, float* m2d,
                             float* mean, float* var, float* alpha_prev, int32_t iteration, int32_t count_f,
                             int32_t count_d, double dpi_norm2, int32_t zero_grads, double* dpi_norm2_out,
                             void* cuda_stream);

/* Device arrays of the standalone update (n floats each, 16-byte aligned). pi_next may not alias
 * pi; with MER_META_PER_ELEMENT it holds pi_{i-1} on entry (as the context's second parameter
 * slot does). The variant arrays are read only when their flag is set and may be NULL otherwise:
 * mu_f, mu_d (CENTRED, start at 0), adam_m, adam_v (NAIVE_ADAM, start at 0), F_var, dF_var
 * (UNCORRELATED, this iteration's independent samples). */
typedef struct mer_update_arrays {
    const float* pi;
    float *pi_next, *F, *dF, *m2f, *m2d, *mean, *var, *alpha_prev;
    float *mu_f, *mu_d, *adam_m, *adam_v;
    const float *F_var, *dF_var;
} mer_update_arrays;

/* mer_meta_step_raw with every variant of hyper->flags: arrays as described above, scalars as
 * in mer_meta_step_raw (ADAM mode ignores the flags). Rejects (MER_ERR_INVALID_ARG) a flag whose
 * arrays are missing. Shares mer_meta_step_raw's per-device scratch (same race rule). */
mer_status mer_meta_step_raw_ex(const mer_hyper* hyper, int64_t n, int32_t C, const float* lo, const float* hi,
                                const mer_update_arrays* arrays, int32_t iteration, int32_t count_f,
                                int32_t count_d, double dpi_norm2, int32_t zero_grads, double* dpi_norm2_out,
                                void* cuda_stream);

/* The same update as mer_meta_step_raw, for callers that must not allocate device memory:
 * applications that reserve all device memory up front or hand it out through their own pool
 * (a library allocation would go around it or fail), and real-time loops where an allocation,
 * and the device synchronisation that freeing a grown buffer implies, is not allowed.
 * The paper has no counterpart; this is an interface variant only.
 * Arguments, layout, results and tolerances are exactly those of mer_meta_step_raw.
 * Scratch: the per-block partial norms go to a fixed array compiled into the library (512 KiB
 * of device memory on every GPU that loads it, held until the process exits), so n may be at
 * most 268,435,456 parameters; larger n fails with MER_ERR_INVALID_ARG. It calls no cudaMalloc,
 * cudaFree or other allocating routine. The first call on a device looks up the array's device
 * address once (cudaGetSymbolAddress, with that device current); make that first call before any
 * stream capture. All calls share the one array: calls that overlap on the GPU (different
 * streams, no ordering between them) race and give wrong norms; calls ordered on one stream are
 * safe. Nothing in the array needs to start at zero (every call writes all the entries it reads).
 * The looked-up address is kept for the life of the process: do not use this entry point on a
 * device after cudaDeviceReset (or from another driver context on the same device). */
mer_status mer_meta_step_raw_noalloc(const mer_hyper* hyper, int64_t n, int32_t C, const float* lo, const float* hi,
                                     const float* pi, float* pi_next, float* F, float* dF, float* m2f, float* m2d,
                                     float* mean, float* var, float* alpha_prev, int32_t iteration, int32_t count_f,
                                     int32_t count_d, double dpi_norm2, int32_t zero_grads, double* dpi_norm2_out,
                                     void* cuda_stream);

/* Gradient preconditioning of Sec. 6 (texture gradients preconditioned after Nicolet et al. 2021)
 * on its own: g <- (I + lambda L)^{-1} g in place, g a device HWC array of C x H x W floats
 * (C in 1..5, 1 <= H, W <= 4094), L the Neumann graph Laplacian of the W x H texel grid per
 * channel, lambda >= 0 finite (0 leaves g unchanged). The same kernels as the iteration's
 * preconditioning (a DCT-II solve: FFT-based along a power-of-two side, a direct sum otherwise).
 * Allocates its tables and scratch for the call and returns after the result is written
 * (synchronous on cuda_stream). */
mer_status mer_precondition(int32_t C, int32_t H, int32_t W, float lambda, float* g_dev, void* cuda_stream);

/* Philox4x32-10 of n counters: ctr_dev [n][4] u32, out_dev [n][4] u32, key (k0, k1). */
mer_status mer_philox(uint32_t k0, uint32_t k1, const uint32_t* ctr_dev, int64_t n, uint32_t* out_dev,
                      void* cuda_stream);

/* Checkpoint: the optimiser state of every problem (parameters, moments, scalars) as an opaque
 * host blob. With buf NULL, *len receives the size. Synchronous. Restoring into a context with
 * the same scenes continues bit-identically. */
mer_status mer_checkpoint_save(mer_ctx* ctx, void* buf, size_t* len);
mer_status mer_checkpoint_load(mer_ctx* ctx, const void* buf, size_t len);

/* Autotune launch shapes (block size, blocks per SM, shared-memory BVH staging) of the
 * wavefront kernels by timing trial iterations; the choice is kept in the context and its
 * description written to desc (may be NULL). Changes no optimisation state. */
mer_status mer_autotune(mer_ctx* ctx, int32_t trial_iters, char* desc, size_t desc_len);

/* Number of the library's own kernel launches the last mer_iterate / mer_gradient_step +
 * mer_update_step enqueued per iteration (for launch accounting; memsets and cuBLAS calls are not
 * counted). */
mer_status mer_launch_count(mer_ctx* ctx, int64_t* launches_per_iter);

/* Per-kernel timing (diagnostic). While enabled, every launch of the wavefront, scatter, loss and
 * update kernels made outside graph capture (by ctx, or by mer_meta_step_raw) is bracketed by CUDA
 * events on the stream it is launched on, and pass counters are read back after each pass (this
 * synchronises). Not for concurrent use from several threads. */
typedef struct mer_kernel_time {
    char name[32];
    int64_t launches;
    int64_t units;      /* work items: rays (extend/shade/shadow), records (scatter), parameters (update),
                           paths (resolve), pixels (loss) */
    double total_ms;    /* sum of event-measured launch durations (timing mode) */
    int64_t node_tests; /* counting mode: BVH node tests (two child boxes each) of extend/shadow */
    int64_t prim_tests; /* counting mode: triangle and sphere tests of extend/shadow */
} mer_kernel_time;
/* enable: 0 off, 1 timing (events around launches), 2 counting (traversal kernels count their
 * node and primitive tests; launches are not timed). */
mer_status mer_profile_enable(mer_ctx* ctx, int32_t enable);
/* Synchronises, writes up to max_entries launch classes that ran (in a fixed order) and clears them. */
mer_status mer_profile_read(mer_ctx* ctx, mer_kernel_time* out, int32_t max_entries, int32_t* n_out);

/* Optimiser of a volume's voxel parameters toward target images (the 256^3 emissive-absorptive
 * experiment of Sec. 6) by the meta-estimator (MER_MODE_META) or Adam (MER_MODE_ADAM). It owns two
 * parameter slots (pi_i and pi_{i-1}), F, dF, the optimiser state and its images. One iteration:
 * the proportional sample <F_i> (render pi_i on MER_STREAM_PROP_PRIMAL, loss adjoint, replay on
 * MER_STREAM_PROP_ADJ), in META mode concurrently the FD sample <dF_i> of Eq. est_triv (pi_i and
 * pi_{i-1} rendered on the same MER_STREAM_FD_PRIMAL rays, both loss adjoints, paired replay on
 * MER_STREAM_FD_ADJ), then the fused update a11 over the 4 nvox parameters (channel c = index % 4
 * clamped to [lo[c], hi[c]]). Every per-iteration scalar (iteration, slot, step counts, ||dpi||^2,
 * the update's coefficients) stays on the device, so mer_volume_opt_iterate with use_graph = 1
 * replays one captured graph. hyper->flags: every MER_META_* variant (UNCORRELATED repeats both
 * samples on the streams + MER_STREAM_VAR_OFFSET; FD_SHARED_PATH changes nothing, no sampling
 * decision of the march depends on the parameters); precond_lambda must be 0.
 * target: device image [n_views][height][width][3] (copied); init: device voxels (copied into
 * both slots, 16-byte aligned). vol must outlive the optimiser. Synchronous. */
typedef struct mer_volume_opt mer_volume_opt;
mer_status mer_volume_opt_create(mer_volume* vol, const mer_hyper* hyper, int32_t loss_kind, int32_t spp_f,
                                 int32_t spp_d, const float* lo4, const float* hi4, const float* target_dev,
                                 const float* init_dev, mer_volume_opt** out);
void mer_volume_opt_destroy(mer_volume_opt* opt);
/* Both slots = params_dev (device, copied); the optimiser state and iteration count reset. Synchronous. */
mer_status mer_volume_opt_set_params(mer_volume_opt* opt, const float* params_dev);
/* n_iters iterations, ordered after earlier work on cuda_stream, which waits for them (asynchronous;
 * the optimiser's own streams run the work). use_graph = 1: one graph captured on first use. */
mer_status mer_volume_opt_iterate(mer_volume_opt* opt, int32_t n_iters, int32_t use_graph, void* cuda_stream);
/* iteration, loss of the last proportional primal image, ||dpi||^2, step counts; paths_per_iter =
 * ray marches per iteration (a rendered ray counts one, a replayed one two). Synchronous. */
mer_status mer_volume_opt_stats(mer_volume_opt* opt, mer_iter_stats* out);
/* Device pointers of the optimiser's arrays (valid until destroy; pi_cur / pi_prev as of the
 * last completed iteration; NULL where the mode and flags keep no such array). Synchronous. */
mer_status mer_volume_opt_state(mer_volume_opt* opt, mer_state_view* out);
/* Kernel launches (and memsets) one iteration enqueues. */
mer_status mer_volume_opt_launches(mer_volume_opt* opt, int32_t* out);

#ifdef __cplusplus
}
#endif
#endif /* MER_H */

// Emissive-absorptive volume (the high-dimensional experiment of Sec. 6): a voxel grid of
// emission (RGB) and density over an axis-aligned box, seen from several pinhole views and
// rendered by a jittered ray march
//   L = sum_k T_k (1 - exp(-sigma_k delta)) e_k + T_end * background,  T_{k+1} = T_k exp(-sigma_k delta),
// sample k at t0 + (k + u) delta with one Philox uniform u per ray (vertex 1), samples past the
// exit skipped. Voxel parameters are one float4 each (emission RGB, density) at
// ((z ny + y) nx + x); trilinear, clamp-to-edge, voxel centres at (i + 1/2) / n across the box.
// The adjoint marches each ray twice from the same counters: a radiance pass that records
// (sigma_k, adj . e_k) per step (8 bytes per step of each ray in flight, in a buffer the volume
// owns) and a replay that reads the records back instead of the voxels:
// dL/de_k = T_k a_k, dL/dsigma_k = delta ((1 - a_k) T_k e_k - L_after_k), distributed to the
// eight voxels by the trilinear weights with fire-and-forget float4 reductions.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "mer_internal.cuh"
#include "update.cuh"

namespace mer {

struct VolCam {
    float o[3], f[3], r[3], u[3];   // eye, forward, right * tan(fov/2) * aspect, up * tan(fov/2)
};

struct VolDev {
    int nx, ny, nz, views, width, height;
    float lo[3], scale[3];          // grid coordinate = (p - lo) * scale - 1/2
    float hi[3];
    float step;
    float bg[3];
    uint32_t seed, key_id;
    const VolCam* cams;
};

__device__ __forceinline__ bool vol_box(const VolDev& V, v3 o, v3 d, float& t0, float& t1) {
    float a = 0.0f, b = INFINITY;
    const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (dd[k] == 0.0f) {
            if (oo[k] < V.lo[k] || oo[k] > V.hi[k]) return false;
            continue;
        }
        float ta = (V.lo[k] - oo[k]) / dd[k], tb = (V.hi[k] - oo[k]) / dd[k];
        if (ta > tb) { const float t = ta; ta = tb; tb = t; }
        a = fmaxf(a, ta);
        b = fminf(b, tb);
    }
    t0 = a;
    t1 = b;
    return b > a;
}

struct Taps {
    int idx[8];
    float w[8];
};

__device__ __forceinline__ void vol_taps(const VolDev& V, v3 p, Taps& T) {
    const float pp[3] = {p.x, p.y, p.z};
    const int n[3] = {V.nx, V.ny, V.nz};
    int i0[3], i1[3];
    float f[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float g = (pp[k] - V.lo[k]) * V.scale[k] - 0.5f;
        const float fl = floorf(g);
        f[k] = g - fl;
        const int a = (int)fl;
        i0[k] = min(max(a, 0), n[k] - 1);
        i1[k] = min(max(a + 1, 0), n[k] - 1);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int x = (c & 1) ? i1[0] : i0[0], y = (c & 2) ? i1[1] : i0[1], z = (c & 4) ? i1[2] : i0[2];
        const float wx = (c & 1) ? f[0] : 1.0f - f[0], wy = (c & 2) ? f[1] : 1.0f - f[1];
        const float wz = (c & 4) ? f[2] : 1.0f - f[2];
        T.idx[c] = (z * V.ny + y) * V.nx + x;
        T.w[c] = wx * wy * wz;
    }
}

__device__ __forceinline__ void red4(float4* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

__device__ __forceinline__ void vol_ray(const VolDev& V, uint32_t pixel, uint32_t sample, uint32_t iter, uint32_t stream,
                                        v3& o, v3& d, float& u) {
    const uint32_t per_view = (uint32_t)V.width * (uint32_t)V.height;
    const uint32_t view = pixel / per_view, local = pixel - view * per_view;
    const uint4 r = draw(V.seed, V.key_id, pixel, sample, iter, stream, 0, 0);
    const VolCam& C = V.cams[view];
    const uint32_t px = local % (uint32_t)V.width, py = local / (uint32_t)V.width;
    const float sx = 2.0f * ((float)px + u01(r.x)) / (float)V.width - 1.0f;
    const float sy = 1.0f - 2.0f * ((float)py + u01(r.y)) / (float)V.height;
    o = mk(C.o[0], C.o[1], C.o[2]);
    d = normalize(mk(C.f[0], C.f[1], C.f[2]) + mk(C.r[0], C.r[1], C.r[2]) * sx + mk(C.u[0], C.u[1], C.u[2]) * sy);
    u = u01(draw(V.seed, V.key_id, pixel, sample, iter, stream, 1, 0).x);
}

// Radiance of one parameter vector along one ray. With REC (the adjoint's radiance pass), step k
// (k < max_steps) also records sigma_k and adj . e_k at rec[k * slots] — one float2 plane
// [max_steps][slots] per branch, the caller offsetting rec by its plane and thread slot — and the
// march stops after max_steps; returns the step count.
template <bool REC>
__device__ __forceinline__ int vol_march(const VolDev& V, const float4* __restrict__ par, v3 o, v3 d, float u, v3& Lout,
                                         v3 adj = v3{}, float2* rec = nullptr, int64_t slots = 0, int max_steps = 0) {
    v3 L = mk(0, 0, 0);
    float T = 1.0f;
    float t0, t1;
    int k = 0;
    if (vol_box(V, o, d, t0, t1)) {
        const float dl = V.step;
        for (;; ++k) {
            if (REC && k >= max_steps) break;
            const float t = t0 + ((float)k + u) * dl;
            if (!(t < t1)) break;
            Taps tp;
            vol_taps(V, o + d * t, tp);
            float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f, sd = 0.0f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float4 q = __ldg(par + tp.idx[c]);
                e0 = fmaf(tp.w[c], q.x, e0);
                e1 = fmaf(tp.w[c], q.y, e1);
                e2 = fmaf(tp.w[c], q.z, e2);
                sd = fmaf(tp.w[c], q.w, sd);
            }
            const float tr = expf(-sd * dl), a = 1.0f - tr;
            L = L + mk(e0, e1, e2) * (T * a);
            T *= tr;
            if (REC) rec[(int64_t)k * slots] = make_float2(sd, adj.x * e0 + adj.y * e1 + adj.z * e2);
        }
    }
    Lout = L + mk(V.bg[0], V.bg[1], V.bg[2]) * T;
    return k;
}

// Replay of the first n steps of the ray from the radiance pass's records (no parameter reads):
// with T_k, a_k = 1 - exp(-sigma_k delta) and the running s_k = sum_{i<=k} T_i a_i adj . e_i,
//   dLoss/de_k = T_k a_k adj,   dLoss/dsigma_k = delta (exp(-sigma_k delta) T_k adj . e_k - (adjL - s_k)),
// adjL = adj . (total radiance) per branch; branch 1 of a pair enters with sign -1. The branches'
// sum goes to the eight taps by one vector reduction each. (Summing shared corners of consecutive
// steps in registers first issues fewer reductions but diverges per lane and measured slower.)
template <int NB>
__device__ __forceinline__ void vol_replay(const VolDev& V, v3 o, v3 d, float u, int n, const float2* rec,
                                           int64_t slots, int64_t plane, const v3* adj, const float* adjL,
                                           float4* grad) {
    float t0, t1;
    if (n <= 0 || !vol_box(V, o, d, t0, t1)) return;
    const float dl = V.step;
    float T[NB], acc[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        T[j] = 1.0f;
        acc[j] = 0.0f;
    }
    for (int k = 0; k < n; ++k) {
        const float t = t0 + ((float)k + u) * dl;
        Taps tp;
        vol_taps(V, o + d * t, tp);
        float sd[NB], se[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const float2 r = rec[j * plane + (int64_t)k * slots];
            sd[j] = r.x;
            se[j] = r.y;
        }
        float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f, g3 = 0.0f;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const float sg = j == 0 ? 1.0f : -1.0f;
            const float tr = expf(-sd[j] * dl), a = 1.0f - tr;
            const float ta = T[j] * a;
            acc[j] = fmaf(ta, se[j], acc[j]);
            g0 = fmaf(sg * ta, adj[j].x, g0);
            g1 = fmaf(sg * ta, adj[j].y, g1);
            g2 = fmaf(sg * ta, adj[j].z, g2);
            g3 = fmaf(sg * dl, tr * T[j] * se[j] - (adjL[j] - acc[j]), g3);
            T[j] *= tr;
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) red4(grad + tp.idx[c], tp.w[c] * g0, tp.w[c] * g1, tp.w[c] * g2, tp.w[c] * g3);
    }
}

// Pixel of the i-th ray of a launch: views whose sides are multiples of 16 are walked in 16 x 16
// tiles (a block of 256 rays is one compact bundle that shares voxels across both image axes),
// others row by row.
__device__ __forceinline__ uint32_t vol_pixel(const VolDev& V, uint32_t i) {
    if ((V.width & 15) || (V.height & 15)) return i;
    const uint32_t per_view = (uint32_t)V.width * (uint32_t)V.height;
    const uint32_t view = i / per_view, r = i - view * per_view;
    const uint32_t tiles_x = (uint32_t)V.width >> 4;
    const uint32_t tile = r >> 8, k = r & 255u;
    const uint32_t ty = tile / tiles_x, tx = tile - ty * tiles_x;
    return view * per_view + ((ty << 4) + (k >> 4)) * (uint32_t)V.width + (tx << 4) + (k & 15u);
}

// The parameter vectors and iteration of a launch: given explicitly, or (ps != nullptr) the
// optimiser's two slots, pi_i = slot[ps->cur] and pi_{i-1} = the other, at iteration ps->iteration,
// read on the device so that one captured graph serves every iteration.
struct VolSel {
    const float4* a;
    const float4* b;            // second vector of a pair, or nullptr
    const float4* slot[2];
    const ProbState* ps;
    uint32_t iter;
    int32_t pair;
};

__device__ __forceinline__ void vol_resolve(const VolSel& S, const float4*& a, const float4*& b, uint32_t& iter) {
    if (S.ps) {
        const int c = S.ps->cur & 1;
        a = S.slot[c];
        b = S.pair ? S.slot[c ^ 1] : nullptr;
        iter = (uint32_t)S.ps->iteration;
    } else {
        a = S.a;
        b = S.b;
        iter = S.iter;
    }
}

// one thread per pixel, spp samples; with a pair the same rays are marched through both vectors,
// one after the other
template <int NB>
__global__ void __launch_bounds__(256) k_vol_render(VolDev V, VolSel S, int spp, uint32_t stream, float* imgA,
                                                    float* imgB) {
    const float4* par[2];
    uint32_t iter;
    vol_resolve(S, par[0], par[1], iter);
    const int64_t N = (int64_t)V.views * V.width * V.height;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float inv = 1.0f / (float)spp;
    float* img[2] = {imgA, imgB};
    for (int64_t pi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pi < N; pi += stride) {
        const int64_t p = vol_pixel(V, (uint32_t)pi);
        v3 acc[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) acc[j] = mk(0, 0, 0);
        for (int s = 0; s < spp; ++s) {
            v3 o, d;
            float u;
            vol_ray(V, (uint32_t)p, (uint32_t)s, iter, stream, o, d, u);
            v3 L;
            vol_march<false>(V, par[0], o, d, u, L);
            acc[0] = acc[0] + L;
            if (NB == 2) {
                vol_march<false>(V, par[1], o, d, u, L);
                acc[NB - 1] = acc[NB - 1] + L;
            }
        }
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            img[j][3 * p + 0] = acc[j].x * inv;
            img[j][3 * p + 1] = acc[j].y * inv;
            img[j][3 * p + 2] = acc[j].z * inv;
        }
    }
}

// one thread per (pixel, sample): the radiance pass, recording each step, then the replay from the
// records; with a pair (NB = 2) the second branch's radiance pass follows the first's (same
// counters at the second parameter vector) and one replay handles both, the second subtracted.
// Thread slot q owns records rec[j * plane + k * slots + q], plane = max_steps * slots.
template <int NB>
__global__ void __launch_bounds__(256) k_vol_adjoint(VolDev V, VolSel S, const float* __restrict__ dA,
                                                     const float* __restrict__ dB, int spp, uint32_t stream,
                                                     float4* grad, float2* rec, int64_t slots, int max_steps) {
    const float4* par[2];
    uint32_t iter;
    vol_resolve(S, par[0], par[1], iter);
    const int64_t N = (int64_t)V.views * V.width * V.height;
    const int64_t total = N * spp;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t plane = (int64_t)max_steps * slots;
    const float inv = 1.0f / (float)spp;
    const float* dimg[2] = {dA, dB};
    for (int64_t i = q; i < total; i += stride) {
        const int64_t pi = i / spp;
        const uint32_t s = (uint32_t)(i - pi * spp);
        const int64_t p = vol_pixel(V, (uint32_t)pi);
        v3 o, d;
        float u;
        vol_ray(V, (uint32_t)p, s, iter, stream, o, d, u);
        v3 adj[NB];
        float adjL[NB];
        int n = 0;
#pragma unroll 1
        for (int j = 0; j < NB; ++j) {      // not unrolled: one copy of the march, like the single kernel
            const float* dj = j ? dimg[NB - 1] : dimg[0];
            const v3 aj = mk(dj[3 * p] * inv, dj[3 * p + 1] * inv, dj[3 * p + 2] * inv);
            v3 L;
            n = vol_march<true>(V, j ? par[1] : par[0], o, d, u, L, aj, rec + j * plane + q, slots, max_steps);
            const float al = aj.x * L.x + aj.y * L.y + aj.z * L.z;
            if (j == 0) {
                adj[0] = aj;
                adjL[0] = al;
            } else {
                adj[NB - 1] = aj;
                adjL[NB - 1] = al;
            }
        }
        vol_replay<NB>(V, o, d, u, n, rec + q, slots, plane, adj, adjL, grad);
    }
}

// image loss: L2 (kind 0) or MRSE (kind 1, each term / (T^2 + 0.01)); loss accumulated in FP64
__global__ void __launch_bounds__(256) k_image_loss(int kind, int64_t n_pix, const float* __restrict__ img,
                                                    const float* __restrict__ tgt, float* dimg, double* loss) {
    const int64_t n = 3 * n_pix, stride = (int64_t)gridDim.x * blockDim.x;
    const float sc = 2.0f / (3.0f * (float)n_pix);
    double l = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float t = tgt[i];
        const float w = kind == MER_LOSS_MRSE ? 1.0f / (t * t + 0.01f) : 1.0f;
        const float r = img[i] - t;
        dimg[i] = sc * r * w;
        l += (double)r * (double)r * (double)w;
    }
    if (!loss) return;
    __shared__ double part[8];
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < 8; ++w) b += part[w];
        atomicAdd(loss, b / (3.0 * (double)n_pix));     // one atomic per block
    }
}

}  // namespace mer

using namespace mer;

struct mer_volume {
    int device = 0;
    VolDev dev{};
    VolCam* d_cams = nullptr;
    int64_t n_vox = 0;
    int max_steps = 0;           // bound on the march steps of any ray through the box
    // radiance-pass records of the adjoint (index 0: single, 1: pair), allocated on first use:
    // one [max_steps][slots] float2 plane per branch, slots = the persistent grid's threads
    void* rec[2] = {nullptr, nullptr};
    int64_t rec_slots[2] = {0, 0};
    int rec_blocks[2] = {0, 0};
};

extern "C" mer_status mer_volume_create(const mer_volume_desc* d, int32_t device, mer_volume** out) {
    if (!d || !out || !d->cameras || d->nx < 1 || d->ny < 1 || d->nz < 1 || d->n_views < 1 || d->width < 1 ||
        d->height < 1 || !(d->step > 0.0f))
        return mer_internal_fail(MER_ERR_INVALID_ARG, "bad volume description");
    for (int k = 0; k < 3; ++k)
        if (!(d->hi[k] > d->lo[k])) return mer_internal_fail(MER_ERR_INVALID_ARG, "empty volume box");
    if ((int64_t)d->nx * d->ny * d->nz >= ((int64_t)1 << 31) ||
        (int64_t)d->n_views * d->width * d->height >= ((int64_t)1 << 32))
        return mer_internal_fail(MER_ERR_INVALID_ARG, "volume or image too large");
    for (int i = 0; i < d->n_views; ++i) {
        // eye != target, up not parallel to the view direction, field of view in (0, 180) degrees
        const float* c = d->cameras + 10 * i;
        const double f[3] = {(double)c[3] - c[0], (double)c[4] - c[1], (double)c[5] - c[2]};
        const double r[3] = {f[1] * c[8] - f[2] * c[7], f[2] * c[6] - f[0] * c[8], f[0] * c[7] - f[1] * c[6]};
        if (!(f[0] * f[0] + f[1] * f[1] + f[2] * f[2] > 0.0) || !(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] > 0.0) ||
            !(c[9] > 0.0f && c[9] < 180.0f))
            return mer_internal_fail(MER_ERR_INVALID_ARG, "degenerate volume camera");
    }
    if (cudaSetDevice(device) != cudaSuccess) return mer_internal_fail(MER_ERR_CUDA, "bad device");
    mer_volume* v = new mer_volume();
    v->device = device;
    VolDev& V = v->dev;
    V.nx = d->nx; V.ny = d->ny; V.nz = d->nz;
    V.views = d->n_views; V.width = d->width; V.height = d->height;
    const int n[3] = {d->nx, d->ny, d->nz};
    for (int k = 0; k < 3; ++k) {
        V.lo[k] = d->lo[k];
        V.hi[k] = d->hi[k];
        V.scale[k] = (float)(n[k] / ((double)d->hi[k] - (double)d->lo[k]));
        V.bg[k] = d->background[k];
    }
    V.step = d->step;
    V.seed = d->seed;
    V.key_id = d->key_id;
    std::vector<VolCam> cams(d->n_views);
    for (int i = 0; i < d->n_views; ++i) {
        const float* c = d->cameras + 10 * i;
        double f[3] = {c[3] - c[0], c[4] - c[1], c[5] - c[2]};
        double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        for (double& x : f) x /= fl;
        double r[3] = {f[1] * c[8] - f[2] * c[7], f[2] * c[6] - f[0] * c[8], f[0] * c[7] - f[1] * c[6]};
        double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        for (double& x : r) x /= rl;
        double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
        const double th = std::tan(0.5 * c[9] * 3.14159265358979323846 / 180.0);
        const double asp = (double)d->width / (double)d->height;
        for (int k = 0; k < 3; ++k) {
            cams[i].o[k] = c[k];
            cams[i].f[k] = (float)f[k];
            cams[i].r[k] = (float)(r[k] * th * asp);
            cams[i].u[k] = (float)(u[k] * th);
        }
    }
    cudaError_t e = cudaMalloc(&v->d_cams, sizeof(VolCam) * cams.size());
    if (!e) e = cudaMemcpy(v->d_cams, cams.data(), sizeof(VolCam) * cams.size(), cudaMemcpyHostToDevice);
    if (e) {
        cudaFree(v->d_cams);
        delete v;
        return mer_internal_fail(MER_ERR_CUDA, cudaGetErrorString(e));
    }
    V.cams = v->d_cams;
    v->n_vox = (int64_t)d->nx * d->ny * d->nz;
    // steps k with t0 + (k + u) delta < t1 number at most floor((t1 - t0) / delta) + 1, and t1 - t0 is
    // at most the box diagonal; one more for rounding
    double diag2 = 0.0;
    for (int k = 0; k < 3; ++k) diag2 += ((double)d->hi[k] - d->lo[k]) * ((double)d->hi[k] - d->lo[k]);
    const double ms = std::floor(std::sqrt(diag2) / (double)d->step) + 2.0;
    if (ms > 1e6) {
        cudaFree(v->d_cams);
        delete v;
        return mer_internal_fail(MER_ERR_INVALID_ARG, "march step too small for the volume box");
    }
    v->max_steps = (int)ms;
    *out = v;
    return MER_OK;
}

extern "C" void mer_volume_destroy(mer_volume* v) {
    if (!v) return;
    cudaSetDevice(v->device);
    cudaFree(v->d_cams);
    cudaFree(v->rec[0]);
    cudaFree(v->rec[1]);
    delete v;
}

// the adjoint's persistent grid (SMs x resident blocks) and its record buffer, for NB branches
template <int NB>
static cudaError_t vol_ensure_rec(mer_volume* v) {
    const int i = NB - 1;
    if (v->rec[i]) return cudaSuccess;
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_vol_adjoint<NB>, 256, 0);
    if (e) return e;
    const int blocks = std::max(1, sms * std::max(occ, 1));
    const int64_t slots = (int64_t)blocks * 256;
    e = cudaMalloc(&v->rec[i], (size_t)NB * (size_t)slots * (size_t)v->max_steps * sizeof(float2));
    if (e) {
        v->rec[i] = nullptr;
        return e;
    }
    v->rec_slots[i] = slots;
    v->rec_blocks[i] = blocks;
    return cudaSuccess;
}

template <int NB>
static cudaError_t vol_launch_adjoint(mer_volume* v, const VolSel& S, const float* dA, const float* dB, int spp,
                                      uint32_t stream, float* grad, cudaStream_t st) {
    const cudaError_t e = vol_ensure_rec<NB>(v);
    if (e) return e;
    const int i = NB - 1;
    const int64_t total = (int64_t)v->dev.views * v->dev.width * v->dev.height * spp;
    const int blocks = (int)std::min<int64_t>(v->rec_blocks[i], (total + 255) / 256);
    k_vol_adjoint<NB><<<std::max(blocks, 1), 256, 0, st>>>(v->dev, S, dA, dB, spp, stream, reinterpret_cast<float4*>(grad),
                                                           static_cast<float2*>(v->rec[i]),
                                                           v->rec_slots[i], v->max_steps);
    return cudaGetLastError();
}

static int vol_grid(int64_t n) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

extern "C" mer_status mer_volume_render(mer_volume* v, const float* params, int32_t spp, uint32_t stream,
                                        uint32_t iteration, float* img, void* cuda_stream) {
    if (!v || !params || !img || spp < 1 || !aligned16(params) || stream > MER_STREAM_MAX)
        return mer_internal_fail(MER_ERR_INVALID_ARG, "bad arguments to mer_volume_render");
    cudaSetDevice(v->device);
    const int64_t N = (int64_t)v->dev.views * v->dev.width * v->dev.height;
    VolSel S{};
    S.a = reinterpret_cast<const float4*>(params);
    S.iter = iteration;
    k_vol_render<1><<<vol_grid(N), 256, 0, (cudaStream_t)cuda_stream>>>(v->dev, S, spp, stream, img, nullptr);
    const cudaError_t e = cudaGetLastError();
    return e ? mer_internal_fail(MER_ERR_CUDA, cudaGetErrorString(e)) : MER_OK;
}

static mer_status vol_adjoint(mer_volume* v, const float* pA, const float* pB, const float* dA, const float* dB,
                              int32_t spp, uint32_t stream, uint32_t iteration, float* grad, void* cuda_stream) {
    if (!v || !pA || !dA || !grad || spp < 1 || !aligned16(pA) || !aligned16(grad) || (pB && (!dB || !aligned16(pB))) ||
        stream > MER_STREAM_MAX)
        return mer_internal_fail(MER_ERR_INVALID_ARG, "bad arguments to mer_volume_adjoint");
    cudaSetDevice(v->device);
    VolSel S{};
    S.a = reinterpret_cast<const float4*>(pA);
    S.b = reinterpret_cast<const float4*>(pB);
    S.iter = iteration;
    const cudaError_t e = pB ? vol_launch_adjoint<2>(v, S, dA, dB, spp, stream, grad, (cudaStream_t)cuda_stream)
                             : vol_launch_adjoint<1>(v, S, dA, dB, spp, stream, grad, (cudaStream_t)cuda_stream);
    return e ? mer_internal_fail(MER_ERR_CUDA, cudaGetErrorString(e)) : MER_OK;
}

extern "C" mer_status mer_volume_adjoint(mer_volume* v, const float* params, const float* dimg, int32_t spp,
                                         uint32_t stream, uint32_t iteration, float* grad, void* cuda_stream) {
    return vol_adjoint(v, params, nullptr, dimg, nullptr, spp, stream, iteration, grad, cuda_stream);
}

extern "C" mer_status mer_volume_adjoint_pair(mer_volume* v, const float* pA, const float* pB, const float* dA,
                                              const float* dB, int32_t spp, uint32_t stream, uint32_t iteration,
                                              float* grad, void* cuda_stream) {
    if (!pB) return mer_internal_fail(MER_ERR_INVALID_ARG, "mer_volume_adjoint_pair needs both parameter vectors");
    return vol_adjoint(v, pA, pB, dA, dB, spp, stream, iteration, grad, cuda_stream);
}

extern "C" mer_status mer_image_loss(int32_t kind, int64_t n_pix, const float* img, const float* target, float* dimg,
                                     double* loss, void* cuda_stream) {
    if (n_pix < 1 || !img || !target || !dimg || !loss || (kind != MER_LOSS_L2 && kind != MER_LOSS_MRSE))
        return mer_internal_fail(MER_ERR_INVALID_ARG, "bad arguments to mer_image_loss");
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaMemsetAsync(loss, 0, sizeof(double), st);
    k_image_loss<<<vol_grid(3 * n_pix), 256, 0, st>>>(kind, n_pix, img, target, dimg, loss);
    const cudaError_t e = cudaGetLastError();
    return e ? mer_internal_fail(MER_ERR_CUDA, cudaGetErrorString(e)) : MER_OK;
}

// ---------------------------------------------------------------------------------------
// Optimiser of a volume's voxels toward target images (mer_volume_opt_*). One iteration, all
// on the device and capturable as one graph:
//   branch 1 (proportional <F>): render pi_i (PROP_PRIMAL), loss adjoint, replay (PROP_ADJ) into F;
//   branch 2 (META, FD <dF>):   render pi_i and pi_{i-1} on the same rays (FD_PRIMAL), both loss
//                                adjoints, paired replay (FD_ADJ) into dF;
//   UNCORRELATED: each branch repeats itself on streams + MER_STREAM_VAR_OFFSET into F_var, dF_var;
//   then the fused update of the texture problems (one segment, C = 4) with its finalize, which
//   advances the iteration, swaps the slots and computes the next coefficients on the device.
// ---------------------------------------------------------------------------------------

struct mer_volume_opt {
    mer_volume* vol = nullptr;
    int device = 0;
    mer_hyper h{};
    int32_t loss_kind = 0, spp_f = 1, spp_d = 1;
    bool meta = true;
    int64_t n = 0, n_pix = 0;
    float* slot[2] = {nullptr, nullptr};
    float *F = nullptr, *dF = nullptr, *m2f = nullptr, *m2d = nullptr, *mean = nullptr, *var = nullptr, *ap = nullptr;
    float *mu_f = nullptr, *mu_d = nullptr, *am = nullptr, *av = nullptr, *Fv = nullptr, *dFv = nullptr;
    float *target = nullptr, *imgP = nullptr, *dP = nullptr, *imgA = nullptr, *imgB = nullptr, *dA = nullptr,
          *dB = nullptr;
    ProbState* d_ps = nullptr;
    UpdSeg* d_seg = nullptr;
    int64_t* d_blk_off = nullptr;
    double* d_partials = nullptr;
    int64_t nblocks = 0;
    cudaStream_t st = nullptr, st2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int launches = 0;
    std::vector<void*> allocs;
};

static cudaError_t vopt_alloc(mer_volume_opt* o, float** p, int64_t n) {
    const cudaError_t e = cudaMalloc(p, sizeof(float) * (size_t)std::max<int64_t>(n, 1));
    if (!e) o->allocs.push_back(*p);
    return e;
}

static void vopt_free(mer_volume_opt* o) {
    cudaSetDevice(o->device);
    if (o->gexec) cudaGraphExecDestroy(o->gexec);
    for (void* a : o->allocs) cudaFree(a);
    cudaFree(o->d_ps);
    cudaFree(o->d_seg);
    cudaFree(o->d_blk_off);
    cudaFree(o->d_partials);
    for (cudaEvent_t e : {o->ev_fork, o->ev_join, o->ev_in, o->ev_out})
        if (e) cudaEventDestroy(e);
    if (o->st) cudaStreamDestroy(o->st);
    if (o->st2) cudaStreamDestroy(o->st2);
    delete o;
}

static VolSel vopt_sel(const mer_volume_opt* o, int pair) {
    VolSel S{};
    S.slot[0] = reinterpret_cast<const float4*>(o->slot[0]);
    S.slot[1] = reinterpret_cast<const float4*>(o->slot[1]);
    S.ps = o->d_ps;
    S.pair = pair;
    return S;
}

// one branch: (pair ? FD : proportional) sample of the current iteration into grad (cleared first)
static int vopt_branch(mer_volume_opt* o, int pair, uint32_t soff, float* grad, double* loss, cudaStream_t s) {
    const VolDev& V = o->vol->dev;
    const int spp = pair ? o->spp_d : o->spp_f;
    const uint32_t sp = (pair ? MER_STREAM_FD_PRIMAL : MER_STREAM_PROP_PRIMAL) + soff;
    const uint32_t sa = (pair ? MER_STREAM_FD_ADJ : MER_STREAM_PROP_ADJ) + soff;
    const VolSel S = vopt_sel(o, pair);
    const int g3 = vol_grid(3 * o->n_pix);
    cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)o->n, s);
    if (pair) {
        k_vol_render<2><<<vol_grid(o->n_pix), 256, 0, s>>>(V, S, spp, sp, o->imgA, o->imgB);
        k_image_loss<<<g3, 256, 0, s>>>(o->loss_kind, o->n_pix, o->imgA, o->target, o->dA, nullptr);
        k_image_loss<<<g3, 256, 0, s>>>(o->loss_kind, o->n_pix, o->imgB, o->target, o->dB, nullptr);
        vol_launch_adjoint<2>(o->vol, S, o->dA, o->dB, spp, sa, grad, s);
        return 4;
    }
    if (loss) cudaMemsetAsync(loss, 0, sizeof(double), s);
    k_vol_render<1><<<vol_grid(o->n_pix), 256, 0, s>>>(V, S, spp, sp, o->imgP, nullptr);
    k_image_loss<<<g3, 256, 0, s>>>(o->loss_kind, o->n_pix, o->imgP, o->target, o->dP, loss);
    vol_launch_adjoint<1>(o->vol, S, o->dP, nullptr, spp, sa, grad, s);
    return 3;
}

static int vopt_enqueue(mer_volume_opt* o) {
    int n = 0;
    const bool unc = o->meta && (o->h.flags & MER_META_UNCORRELATED);
    if (o->meta) {
        cudaEventRecord(o->ev_fork, o->st);
        cudaStreamWaitEvent(o->st2, o->ev_fork, 0);
        n += vopt_branch(o, 1, 0, o->dF, nullptr, o->st2);
        if (unc) n += vopt_branch(o, 1, MER_STREAM_VAR_OFFSET, o->dFv, nullptr, o->st2);
        cudaEventRecord(o->ev_join, o->st2);
    }
    n += vopt_branch(o, 0, 0, o->F, &o->d_ps->loss, o->st);
    if (unc) n += vopt_branch(o, 0, MER_STREAM_VAR_OFFSET, o->Fv, nullptr, o->st);
    if (o->meta) cudaStreamWaitEvent(o->st, o->ev_join, 0);
    if (g_timer) g_timer->add_units(KC_UPDATE, o->n);
    launch_update_ctx(o->d_seg, o->d_blk_off, 1, o->nblocks, o->d_ps, o->d_partials, o->st);
    return n + 2;
}

static mer_status vopt_reset(mer_volume_opt* o, const float* params) {
    const size_t nb = sizeof(float) * (size_t)o->n;
    cudaError_t e = cudaMemcpyAsync(o->slot[0], params, nb, cudaMemcpyDeviceToDevice, o->st);
    if (!e) e = cudaMemcpyAsync(o->slot[1], params, nb, cudaMemcpyDeviceToDevice, o->st);
    for (float* a : {o->F, o->dF, o->m2f, o->m2d, o->mean, o->var, o->mu_f, o->mu_d, o->am, o->av, o->Fv, o->dFv})
        if (!e && a) e = cudaMemsetAsync(a, 0, nb, o->st);
    if (!e) run_fill(o->ap, o->n, -INFINITY, o->st);
    ProbState ps{};
    ps.coef = update_coef(o->h, 0, 0, 0, 0.0);
    if (!e) e = cudaMemcpyAsync(o->d_ps, &ps, sizeof ps, cudaMemcpyHostToDevice, o->st);
    if (!e) e = cudaStreamSynchronize(o->st);
    return e ? mer_internal_fail(MER_ERR_CUDA, cudaGetErrorString(e)) : MER_OK;
}

extern "C" mer_status mer_volume_opt_create(mer_volume* vol, const mer_hyper* hyper, int32_t loss_kind, int32_t spp_f,
                                            int32_t spp_d, const float* lo, const float* hi, const float* target,
                                            const float* init, mer_volume_opt** out) {
    if (!vol || !hyper || !lo || !hi || !target || !init || !out || !aligned16(init))
        return mer_internal_fail(MER_ERR_INVALID_ARG, "bad arguments to mer_volume_opt_create");
    if (const char* why = hyper_problem(*hyper)) return mer_internal_fail(MER_ERR_INVALID_ARG, why);
    if (hyper->precond_lambda != 0.0f)
        return mer_internal_fail(MER_ERR_INVALID_ARG, "gradient preconditioning applies to textures only");
    if (loss_kind != MER_LOSS_L2 && loss_kind != MER_LOSS_MRSE)
        return mer_internal_fail(MER_ERR_INVALID_ARG, "unknown loss kind");
    if (spp_f < 1 || (hyper->mode == MER_MODE_META && spp_d < 1))
        return mer_internal_fail(MER_ERR_INVALID_ARG, "samples per pixel must be >= 1");
    for (int k = 0; k < 4; ++k)
        if (!(lo[k] <= hi[k])) return mer_internal_fail(MER_ERR_INVALID_ARG, "clamp range lo > hi");
    if (cudaSetDevice(vol->device) != cudaSuccess) return mer_internal_fail(MER_ERR_CUDA, "bad device");
    mer_volume_opt* o = new mer_volume_opt();
    o->vol = vol;
    o->device = vol->device;
    o->h = *hyper;
    o->meta = hyper->mode == MER_MODE_META;
    o->loss_kind = loss_kind;
    o->spp_f = spp_f;
    o->spp_d = o->meta ? spp_d : 0;
    o->n = 4 * vol->n_vox;
    o->n_pix = (int64_t)vol->dev.views * vol->dev.width * vol->dev.height;
    const int fl = o->meta ? hyper->flags : 0;
    cudaError_t e = cudaStreamCreateWithFlags(&o->st, cudaStreamNonBlocking);
    if (!e) e = cudaStreamCreateWithFlags(&o->st2, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&o->ev_fork, &o->ev_join, &o->ev_in, &o->ev_out})
        if (!e) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    for (float** a : {&o->slot[0], &o->slot[1], &o->F, &o->m2f, &o->mean, &o->ap})
        if (!e) e = vopt_alloc(o, a, o->n);
    if (o->meta)
        for (float** a : {&o->dF, &o->m2d, &o->var})
            if (!e) e = vopt_alloc(o, a, o->n);
    if (fl & MER_META_CENTRED)
        for (float** a : {&o->mu_f, &o->mu_d})
            if (!e) e = vopt_alloc(o, a, o->n);
    if (fl & MER_META_NAIVE_ADAM)
        for (float** a : {&o->am, &o->av})
            if (!e) e = vopt_alloc(o, a, o->n);
    if (fl & MER_META_UNCORRELATED)
        for (float** a : {&o->Fv, &o->dFv})
            if (!e) e = vopt_alloc(o, a, o->n);
    for (float** a : {&o->target, &o->imgP, &o->dP, &o->imgA, &o->imgB, &o->dA, &o->dB})
        if (!e) e = vopt_alloc(o, a, 3 * o->n_pix);
    o->nblocks = update_blocks_for(o->n);
    if (!e) e = vol_ensure_rec<1>(vol);          // allocated here, not inside a graph capture
    if (!e && o->meta) e = vol_ensure_rec<2>(vol);
    if (!e) e = cudaMalloc(&o->d_ps, sizeof(ProbState));
    if (!e) e = cudaMalloc(&o->d_seg, sizeof(UpdSeg));
    if (!e) e = cudaMalloc(&o->d_blk_off, 2 * sizeof(int64_t));
    if (!e) e = cudaMalloc(&o->d_partials, sizeof(double) * (size_t)std::max<int64_t>(1, o->nblocks));
    if (e) {
        vopt_free(o);
        return mer_internal_fail(e == cudaErrorMemoryAllocation ? MER_ERR_OOM : MER_ERR_CUDA, cudaGetErrorString(e));
    }
    UpdSeg S;
    memset(&S, 0, sizeof S);
    S.pA = o->slot[0];
    S.pB = o->slot[1];
    S.F = o->F;
    S.dF = o->dF;
    S.m2f = o->m2f;
    S.m2d = o->m2d;
    S.mean = o->mean;
    S.var = o->var;
    S.ap = o->ap;
    S.mu_f = o->mu_f;
    S.mu_d = o->mu_d;
    S.am = o->am;
    S.av = o->av;
    S.Fv = o->Fv;
    S.dFv = o->dFv;
    S.n = o->n;
    S.C = 4;
    S.prob = 0;
    S.zero_grads = 0;        // each branch clears its gradient before its replay
    for (int k = 0; k < 8; ++k) {
        S.lo[k] = k < 4 ? lo[k] : 0.0f;
        S.hi[k] = k < 4 ? hi[k] : 0.0f;
    }
    S.hyper = o->h;
    S.hyper.flags = fl;
    o->h.flags = fl;
    const int64_t boff[2] = {0, o->nblocks};
    e = cudaMemcpy(o->d_seg, &S, sizeof S, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(o->d_blk_off, boff, sizeof boff, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(o->target, target, sizeof(float) * 3 * (size_t)o->n_pix, cudaMemcpyDeviceToDevice);
    if (e) {
        vopt_free(o);
        return mer_internal_fail(MER_ERR_CUDA, cudaGetErrorString(e));
    }
    const mer_status s = vopt_reset(o, init);
    if (s) {
        vopt_free(o);
        return s;
    }
    *out = o;
    return MER_OK;
}

extern "C" void mer_volume_opt_destroy(mer_volume_opt* o) {
    if (!o) return;
    cudaStreamSynchronize(o->st);
    vopt_free(o);
}

extern "C" mer_status mer_volume_opt_set_params(mer_volume_opt* o, const float* params) {
    if (!o || !params || !aligned16(params)) return mer_internal_fail(MER_ERR_INVALID_ARG, "bad parameters");
    cudaSetDevice(o->device);
    return vopt_reset(o, params);
}

extern "C" mer_status mer_volume_opt_iterate(mer_volume_opt* o, int32_t n_iters, int32_t use_graph,
                                             void* cuda_stream) {
    if (!o || n_iters < 0) return mer_internal_fail(MER_ERR_INVALID_ARG, "bad arguments to mer_volume_opt_iterate");
    cudaSetDevice(o->device);
    const cudaStream_t user = (cudaStream_t)cuda_stream;
    cudaEventRecord(o->ev_in, user);
    cudaStreamWaitEvent(o->st, o->ev_in, 0);
    cudaError_t e = cudaSuccess;
    if (!use_graph) {
        for (int i = 0; i < n_iters; ++i) o->launches = vopt_enqueue(o);
        e = cudaGetLastError();
    } else {
        if (!o->gexec) {
            cudaGraph_t graph = nullptr;
            KernelTimer* saved = g_timer;
            g_timer = nullptr;   // no event timing inside a captured graph
            e = cudaStreamBeginCapture(o->st, cudaStreamCaptureModeThreadLocal);
            if (!e) {
                const int n = vopt_enqueue(o);
                e = cudaStreamEndCapture(o->st, &graph);
                if (!e) e = cudaGraphInstantiate(&o->gexec, graph, 0);
                if (graph) cudaGraphDestroy(graph);
                if (!e) o->launches = n;
            }
            g_timer = saved;
        }
        for (int i = 0; i < n_iters && !e; ++i) e = cudaGraphLaunch(o->gexec, o->st);
    }
    cudaEventRecord(o->ev_out, o->st);
    cudaStreamWaitEvent(user, o->ev_out, 0);
    return e ? mer_internal_fail(MER_ERR_CUDA, cudaGetErrorString(e)) : MER_OK;
}

extern "C" mer_status mer_volume_opt_stats(mer_volume_opt* o, mer_iter_stats* out) {
    if (!o || !out) return mer_internal_fail(MER_ERR_INVALID_ARG, "bad arguments to mer_volume_opt_stats");
    cudaSetDevice(o->device);
    ProbState ps;
    cudaError_t e = cudaMemcpyAsync(&ps, o->d_ps, sizeof ps, cudaMemcpyDeviceToHost, o->st);
    if (!e) e = cudaStreamSynchronize(o->st);
    if (e) return mer_internal_fail(MER_ERR_CUDA, cudaGetErrorString(e));
    out->iteration = ps.iteration;
    out->loss = ps.loss;
    out->dpi_norm2 = ps.dpi_norm2;
    out->count_f = ps.count_f;
    out->count_d = ps.count_d;
    // ray marches: render + radiance/replay pair per proportional sample, twice that per FD sample
    const int64_t per = o->n_pix * (3 * (int64_t)o->spp_f + 6 * (int64_t)o->spp_d);
    out->paths_per_iter = (o->meta && (o->h.flags & MER_META_UNCORRELATED)) ? 2 * per : per;
    return MER_OK;
}

extern "C" mer_status mer_volume_opt_state(mer_volume_opt* o, mer_state_view* out) {
    if (!o || !out) return mer_internal_fail(MER_ERR_INVALID_ARG, "bad arguments to mer_volume_opt_state");
    cudaSetDevice(o->device);
    int32_t cur = 0;
    cudaError_t e = cudaMemcpyAsync(&cur, &o->d_ps->cur, sizeof cur, cudaMemcpyDeviceToHost, o->st);
    if (!e) e = cudaStreamSynchronize(o->st);
    if (e) return mer_internal_fail(MER_ERR_CUDA, cudaGetErrorString(e));
    memset(out, 0, sizeof *out);
    out->pi_cur = o->slot[cur & 1];
    out->pi_prev = o->slot[(cur & 1) ^ 1];
    out->F = o->F;
    out->dF = o->dF;
    out->m2f = o->m2f;
    out->m2d = o->m2d;
    out->mean = o->mean;
    out->var = o->var;
    out->alpha_prev = o->ap;
    out->mu_f = o->mu_f;
    out->mu_d = o->mu_d;
    out->adam_m = o->am;
    out->adam_v = o->av;
    out->F_var = o->Fv;
    out->dF_var = o->dFv;
    out->n = o->n;
    return MER_OK;
}

extern "C" mer_status mer_volume_opt_launches(mer_volume_opt* o, int32_t* out) {
    if (!o || !out) return mer_internal_fail(MER_ERR_INVALID_ARG, "bad arguments to mer_volume_opt_launches");
    *out = o->launches;
    return MER_OK;
}

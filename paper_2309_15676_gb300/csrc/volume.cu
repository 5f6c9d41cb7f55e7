// Emissive-absorptive volume (the high-dimensional experiment of Sec. 6): a voxel grid of
// emission (RGB) and density over an axis-aligned box, seen from several pinhole views and
// rendered by a jittered ray march
//   L = sum_k T_k (1 - exp(-sigma_k delta)) e_k + T_end * background,  T_{k+1} = T_k exp(-sigma_k delta),
// sample k at t0 + (k + u) delta with one Philox uniform u per ray (vertex 1), samples past the
// exit skipped. Voxel parameters are one float4 each (emission RGB, density) at
// ((z ny + y) nx + x); trilinear, clamp-to-edge, voxel centres at (i + 1/2) / n across the box.
// The adjoint replays the march from the same counters with the ray's total radiance (O(1)
// memory): dL/de_k = T_k a_k, dL/dsigma_k = delta ((1 - a_k) T_k e_k - L_after_k), distributed to
// the eight voxels by the trilinear weights with fire-and-forget float4 reductions.
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

// mode 0: radiance; mode 1: replay adding sg * dLoss/dparams into grad (sg = +1 or -1)
template <int MODE>
__device__ __forceinline__ v3 vol_march(const VolDev& V, const float4* __restrict__ par, v3 o, v3 d, float u, v3 Ltot,
                                        v3 adj, float sg, float4* grad) {
    v3 L = mk(0, 0, 0);
    float T = 1.0f;
    float t0, t1;
    if (vol_box(V, o, d, t0, t1)) {
        const float dl = V.step;
        for (int k = 0;; ++k) {
            const float t = t0 + ((float)k + u) * dl;
            if (!(t < t1)) break;
            Taps tp;
            vol_taps(V, o + d * t, tp);
            float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f, s = 0.0f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float4 q = __ldg(par + tp.idx[c]);
                e0 = fmaf(tp.w[c], q.x, e0);
                e1 = fmaf(tp.w[c], q.y, e1);
                e2 = fmaf(tp.w[c], q.z, e2);
                s = fmaf(tp.w[c], q.w, s);
            }
            const float tr = expf(-s * dl), a = 1.0f - tr;
            L = L + mk(e0, e1, e2) * (T * a);
            if (MODE == 1) {
                const float ta = T * a;
                const float ge0 = sg * adj.x * ta, ge1 = sg * adj.y * ta, ge2 = sg * adj.z * ta;
                const float gs = sg * dl * (adj.x * (tr * T * e0 - (Ltot.x - L.x)) + adj.y * (tr * T * e1 - (Ltot.y - L.y)) +
                                            adj.z * (tr * T * e2 - (Ltot.z - L.z)));
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    red4(grad + tp.idx[c], tp.w[c] * ge0, tp.w[c] * ge1, tp.w[c] * ge2, tp.w[c] * gs);
            }
            T *= tr;
        }
    }
    return L + mk(V.bg[0], V.bg[1], V.bg[2]) * T;
}

__global__ void __launch_bounds__(256) k_vol_render(VolDev V, const float4* __restrict__ par, int spp, uint32_t stream,
                                                    uint32_t iter, float* img) {
    const int64_t N = (int64_t)V.views * V.width * V.height;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += stride) {
        v3 acc = mk(0, 0, 0);
        for (int s = 0; s < spp; ++s) {
            v3 o, d;
            float u;
            vol_ray(V, (uint32_t)p, (uint32_t)s, iter, stream, o, d, u);
            acc = acc + vol_march<0>(V, par, o, d, u, mk(0, 0, 0), mk(0, 0, 0), 0.0f, nullptr);
        }
        const float inv = 1.0f / (float)spp;
        img[3 * p + 0] = acc.x * inv;
        img[3 * p + 1] = acc.y * inv;
        img[3 * p + 2] = acc.z * inv;
    }
}

// one thread per (pixel, sample): radiance pass(es), then the replay(s); with parB the pair's
// second branch is subtracted (same counters at the second parameter vector)
__global__ void __launch_bounds__(256) k_vol_adjoint(VolDev V, const float4* __restrict__ parA,
                                                     const float4* __restrict__ parB, const float* __restrict__ dA,
                                                     const float* __restrict__ dB, int spp, uint32_t stream,
                                                     uint32_t iter, float4* grad) {
    const int64_t N = (int64_t)V.views * V.width * V.height;
    const int64_t total = N * spp;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float inv = 1.0f / (float)spp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int64_t p = i / spp;
        const uint32_t s = (uint32_t)(i - p * spp);
        v3 o, d;
        float u;
        vol_ray(V, (uint32_t)p, s, iter, stream, o, d, u);
        const v3 adjA = mk(dA[3 * p] * inv, dA[3 * p + 1] * inv, dA[3 * p + 2] * inv);
        const v3 LA = vol_march<0>(V, parA, o, d, u, mk(0, 0, 0), mk(0, 0, 0), 0.0f, nullptr);
        vol_march<1>(V, parA, o, d, u, LA, adjA, 1.0f, grad);
        if (parB) {
            const v3 adjB = mk(dB[3 * p] * inv, dB[3 * p + 1] * inv, dB[3 * p + 2] * inv);
            const v3 LB = vol_march<0>(V, parB, o, d, u, mk(0, 0, 0), mk(0, 0, 0), 0.0f, nullptr);
            vol_march<1>(V, parB, o, d, u, LB, adjB, -1.0f, grad);
        }
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
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l / (3.0 * (double)n_pix));
}

}  // namespace mer

using namespace mer;

struct mer_volume {
    int device = 0;
    VolDev dev{};
    VolCam* d_cams = nullptr;
    int64_t n_vox = 0;
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
    *out = v;
    return MER_OK;
}

extern "C" void mer_volume_destroy(mer_volume* v) {
    if (!v) return;
    cudaSetDevice(v->device);
    cudaFree(v->d_cams);
    delete v;
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
    if (!v || !params || !img || spp < 1 || !aligned16(params))
        return mer_internal_fail(MER_ERR_INVALID_ARG, "bad arguments to mer_volume_render");
    cudaSetDevice(v->device);
    const int64_t N = (int64_t)v->dev.views * v->dev.width * v->dev.height;
    k_vol_render<<<vol_grid(N), 256, 0, (cudaStream_t)cuda_stream>>>(v->dev, reinterpret_cast<const float4*>(params), spp,
                                                                        stream, iteration, img);
    const cudaError_t e = cudaGetLastError();
    return e ? mer_internal_fail(MER_ERR_CUDA, cudaGetErrorString(e)) : MER_OK;
}

static mer_status vol_adjoint(mer_volume* v, const float* pA, const float* pB, const float* dA, const float* dB,
                              int32_t spp, uint32_t stream, uint32_t iteration, float* grad, void* cuda_stream) {
    if (!v || !pA || !dA || !grad || spp < 1 || !aligned16(pA) || !aligned16(grad) || (pB && (!dB || !aligned16(pB))))
        return mer_internal_fail(MER_ERR_INVALID_ARG, "bad arguments to mer_volume_adjoint");
    cudaSetDevice(v->device);
    const int64_t N = (int64_t)v->dev.views * v->dev.width * v->dev.height;
    k_vol_adjoint<<<vol_grid(N * spp), 256, 0, (cudaStream_t)cuda_stream>>>(
        v->dev, reinterpret_cast<const float4*>(pA), reinterpret_cast<const float4*>(pB), dA, dB, spp, stream, iteration,
        reinterpret_cast<float4*>(grad));
    const cudaError_t e = cudaGetLastError();
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

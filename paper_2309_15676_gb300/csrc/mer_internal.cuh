// Internal device-side definitions of the GB300 library: random numbers, vector math,
// scene layout in HBM, materials. Everything here is FP32 (no fast-math: the library is
// built with IEEE division/sqrt and denormals preserved).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mer.h"

namespace mer {

constexpr int MAXC = MER_MAX_CHANNELS;
constexpr int MAX_DEPTH = MER_MAX_DEPTH;
constexpr float PI_F = 3.14159265358979323846f;
constexpr float INV_PI_F = 0.318309886183790671538f;

// ---------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC 2011): 10 rounds of two 32x32->64 multiplies on
// words 0 and 2 with the published multipliers, Weyl-sequence key schedule.
// ---------------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1) {
    const uint32_t MA = 0xD2511F53u, MB = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hiA = mulhi32(MA, x.x), loA = MA * x.x;
        const uint32_t hiB = mulhi32(MB, x.z), loB = MB * x.z;
        x = make_uint4(hiB ^ x.y ^ k0, loB, hiA ^ x.w ^ k1, loA);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return x;
}

__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * 0x1p-24f; }

// counter word 3: stream << 16 | vertex << 4 | block
__device__ __forceinline__ uint4 draw(uint32_t k0, uint32_t k1, uint32_t pixel, uint32_t sample,
                                      uint32_t iter, uint32_t stream, uint32_t vertex, uint32_t block) {
    return philox4x32_10(make_uint4(pixel, sample, iter, (stream << 16) | (vertex << 4) | block), k0, k1);
}

// ---------------------------------------------------------------------------------
// small vector type
// ---------------------------------------------------------------------------------
struct v3 {
    float x, y, z;
};
__host__ __device__ __forceinline__ v3 mk(float x, float y, float z) { return v3{x, y, z}; }
__host__ __device__ __forceinline__ v3 operator+(v3 a, v3 b) { return v3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__host__ __device__ __forceinline__ v3 operator-(v3 a, v3 b) { return v3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__host__ __device__ __forceinline__ v3 operator*(v3 a, float s) { return v3{a.x * s, a.y * s, a.z * s}; }
__host__ __device__ __forceinline__ v3 operator-(v3 a) { return v3{-a.x, -a.y, -a.z}; }
__host__ __device__ __forceinline__ float dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ __forceinline__ v3 cross(v3 a, v3 b) {
    return v3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ v3 normalize(v3 a) { return a * (1.0f / sqrtf(dot(a, a))); }

// ---------------------------------------------------------------------------------
// scene layout in HBM (per problem; ProblemDev holds the pointers)
// ---------------------------------------------------------------------------------
// Four-wide BVH node, 128 B: the four children's boxes stored in the parent, one slab per
// float4 (component k = child k), so one node fetch (seven 16-byte loads) tests all four.
// child >= 0: inner node index; child < 0: leaf ~((first << 3) | (count - 1)) over the
// leaf-ordered triangles [first, first + count); NODE_EMPTY: unused slot.
constexpr int NODE_EMPTY = 0x7fffffff;
// Traversal stack entries per thread: a nearest-first walk defers at most three children per inner
// level, so trees of up to TRAV_STACK / 3 inner levels are accepted (mer_scene_add refuses deeper).
constexpr int TRAV_STACK = 64;
struct __align__(16) Node {
    float4 lx, hx, ly, hy, lz, hz;
    int4 child;
    int4 pad;
};

// leaf-ordered triangle, 48 B: v0 (w = original primitive id as int bits), e1, e2
struct TriGeo {
    float4 v0, e1, e2;
};

// per original-order triangle shading attributes, 48 B
struct TriAttr {
    float n[3];        // unit geometric normal, along e1 x e2
    float uv[6];       // uv of v0, v1, v2
    int32_t mat;       // material index
    int32_t light;     // quad-light index or -1
    int32_t pad;
};

struct Sphere {
    float4 cr;         // centre, radius
    float4 uvr;        // u0, u1, v0, v1
    int32_t mat;       // material index
    int32_t pad[3];
};

struct Material {
    int32_t type;      // 0 Lambert, 1 principled
    int32_t textured;
    float c[5];
    int32_t pad;
};

struct QuadLight {
    float p0[3], e1[3], e2[3];
    float le[3];
    float n[3];        // unit normal along e1 x e2
    float area;
};

// One problem's description on the device. Each problem owns its buffers; the table of
// ProblemDev entries is what the batched kernels index by problem id.
struct ProblemDev {
    // geometry (local indices: triangles [0, n_tris), spheres, materials and lights of this problem)
    const Node* nodes;         // root at 0 (nullptr: no triangles)
    int32_t n_nodes;
    const TriGeo* tris;
    const TriAttr* attr;
    const Sphere* sph;
    const Material* mats;
    const QuadLight* quads;
    int32_t n_tris, n_sph, n_quads;
    int32_t n_lights;          // n_quads + has_env
    int32_t has_env;
    float env[3];
    float cam_o[3], cam_f[3], cam_r[3], cam_u[3];  // r scaled by tan(fov/2)*aspect, u by tan(fov/2)
    int32_t width, height, n_pix;
    int32_t tex_c, tex_w, tex_h;
    int64_t n_par;             // H*W*C
    int32_t max_depth, spp_prop, spp_fd;
    uint32_t seed, key_id;
    // parameter-shaped arrays: two parameter slots (pi_i in pslot[cur], pi_{i-1} in the other),
    // gradient accumulators of the proportional and the finite-difference samples
    float* pslot[2];
    float* F;
    float* dF;
    int32_t loss_kind;         // MER_LOSS_*
    int32_t fd_shared;         // FD pairs: the pi_{i-1} branch follows the pi_i path (MER_META_FD_SHARED_PATH)
    float* Fv;                 // MER_META_UNCORRELATED: independent samples of F and dF (else NULL)
    float* dFv;
    // per-pixel arrays [n_pix][3]
    const float* target;
    float* img;                // proportional primal image
    float* dimg;               // its adjoint image dLoss/dI
    float* imgA;               // FD primal pair images (pi_i, pi_{i-1}) and their adjoint images
    float* imgB;
    float* dimgA;
    float* dimgB;
};

// per-problem scalars that live on the device (read and advanced by kernels, so that a
// captured iteration needs no host round trip)
// per-problem scalars of the fused update for the coming iteration (start-up corrections, the
// step-norm terms, Adam's bias corrections), computed once per problem and iteration
struct UpdCoef {
    float cF, cD, norm2, inv_norm, c1, c2;
    int32_t stepD, pad;
};

struct ProbState {
    int32_t iteration;         // optimisation iteration i
    int32_t count_f, count_d;  // Moment2 step counts
    int32_t cur;               // which parameter slot (0/1) holds pi_i; the other holds pi_{i-1}
    double dpi_norm2;          // ||pi_i - pi_{i-1}||^2 of the applied step
    double loss;               // L2 loss of the proportional primal image of the last gradient step
    double loss_acc;           // accumulator used by the loss kernel
    UpdCoef coef;              // this iteration's update coefficients (set at reset and by the
                               // previous update's finalize)
};

// ---------------------------------------------------------------------------------
// orthonormal basis around a unit normal (Duff et al. 2017, JCGT 6(1))
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void basis(v3 n, v3& t, v3& b) {
    const float s = copysignf(1.0f, n.z);
    const float a = -1.0f / (s + n.z);
    const float q = n.x * n.y * a;
    t = mk(1.0f + s * n.x * n.x * a, s * q, -s * n.x);
    b = mk(q, s + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ v3 local_to_world(v3 n, float x, float y, float z) {
    v3 t, b;
    basis(n, t, b);
    return t * x + b * y + n * z;
}

// cosine-weighted hemisphere direction around n
__device__ __forceinline__ v3 cosine_dir(v3 n, float u1, float u2) {
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    const float r = sqrtf(u1);
    return local_to_world(n, r * c, r * s, sqrtf(fmaxf(0.0f, 1.0f - u1)));
}

// ---------------------------------------------------------------------------------
// materials: Lambert f = rho/pi; principled f = (1-m) bc/pi + D F G1(o) G1(i) / (4 co ci)
// with GGX D (alpha = rough^2), Schlick F (F0 = 0.04 (1-m) + bc m), separable Smith G1;
// specular lobe sampled with probability (1+m)/2 (Walter et al. 2007 D*cos sampling).
// ---------------------------------------------------------------------------------
struct MatEval {
    int type;
    float th[MAXC];   // bc.rgb (or albedo), metal, rough
};

// GGX D with k = cos^2 a^2 + sin^2, sin^2 taken from |n x h|^2 so that it keeps its
// relative precision near the specular peak (1 - cos^2 would cancel in FP32)
__device__ __forceinline__ float ggx_k(float a2, float ch, float sh2) { return ch * ch * a2 + sh2; }
__device__ __forceinline__ float ggx_d(float a2, float ch, float sh2) {
    const float k = ggx_k(a2, ch, sh2);
    return a2 / (PI_F * k * k);
}
__device__ __forceinline__ float sin2(v3 n, v3 h) {
    const v3 c = cross(n, h);
    return dot(c, c);
}

__device__ __forceinline__ float smith_g1(float a2, float c) {
    return 2.0f * c / (c + sqrtf(a2 + (1.0f - a2) * c * c));
}

__device__ __forceinline__ float pow5(float x) {
    const float x2 = x * x;
    return x2 * x2 * x;
}

// Half vector of (wo, wi). A direction the GGX lobe sampled comes with its half vector, which
// the evaluation uses as is: recomputing it from wo + wi loses about eps / (wo . h) of relative
// precision (wo + wi = 2 (wo . h) h), which the steep GGX peak of a low roughness amplifies.
__device__ __forceinline__ v3 half_vec(v3 wo, v3 wi) { return normalize(wo + wi); }

// value f (RGB). n faces wo; h = the half vector of (wo, wi).
__device__ __forceinline__ v3 bsdf_f(const MatEval& m, v3 n, v3 wo, v3 wi, v3 h) {
    const float co = dot(n, wo), ci = dot(n, wi);
    if (co <= 0.0f || ci <= 0.0f) return mk(0, 0, 0);
    if (m.type == 0) return mk(m.th[0] * INV_PI_F, m.th[1] * INV_PI_F, m.th[2] * INV_PI_F);
    const float metal = m.th[3], r = m.th[4];
    const float a = r * r, a2 = a * a;
    const float ch = dot(n, h), vh = dot(wi, h);
    const float S = ggx_d(a2, ch, sin2(n, h)) * smith_g1(a2, co) * smith_g1(a2, ci) / (4.0f * co * ci);
    const float fw = pow5(1.0f - vh);
    const float kd = (1.0f - metal) * INV_PI_F;
    float f[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float F0 = 0.04f * (1.0f - metal) + m.th[c] * metal;
        f[c] = kd * m.th[c] + S * (F0 + (1.0f - F0) * fw);
    }
    return mk(f[0], f[1], f[2]);
}

// value and derivatives df[j][c] = d f_c / d theta_j
__device__ __forceinline__ v3 bsdf_f_grad(const MatEval& m, v3 n, v3 wo, v3 wi, v3 h, float df[MAXC][3]) {
#pragma unroll
    for (int j = 0; j < MAXC; ++j) df[j][0] = df[j][1] = df[j][2] = 0.0f;
    const float co = dot(n, wo), ci = dot(n, wi);
    if (co <= 0.0f || ci <= 0.0f) return mk(0, 0, 0);
    if (m.type == 0) {
        df[0][0] = df[1][1] = df[2][2] = INV_PI_F;
        return mk(m.th[0] * INV_PI_F, m.th[1] * INV_PI_F, m.th[2] * INV_PI_F);
    }
    const float metal = m.th[3], r = m.th[4];
    const float a = r * r, a2 = a * a;
    const float ch = dot(n, h), vh = dot(wi, h);
    const float k = ggx_k(a2, ch, sin2(n, h));
    const float D = a2 / (PI_F * k * k);
    const float so = sqrtf(a2 + (1.0f - a2) * co * co), si = sqrtf(a2 + (1.0f - a2) * ci * ci);
    const float Go = 2.0f * co / (co + so), Gi = 2.0f * ci / (ci + si);
    const float inv4 = 1.0f / (4.0f * co * ci);
    const float S = D * Go * Gi * inv4;
    const float fw = pow5(1.0f - vh);
    // dS/drough through alpha = rough^2
    const float dD = (2.0f * a / (PI_F * k * k)) * (1.0f - 2.0f * a2 * ch * ch / k);
    const float dGo = -2.0f * co * (a * (1.0f - co * co) / so) / ((co + so) * (co + so));
    const float dGi = -2.0f * ci * (a * (1.0f - ci * ci) / si) / ((ci + si) * (ci + si));
    const float dS = (dD * Go * Gi + D * (dGo * Gi + Go * dGi)) * inv4 * (2.0f * r);
    const float kd = (1.0f - metal) * INV_PI_F;
    float f[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float bc = m.th[c];
        const float F0 = 0.04f * (1.0f - metal) + bc * metal;
        const float F = F0 + (1.0f - F0) * fw;
        f[c] = kd * bc + S * F;
        df[c][c] = kd + S * (1.0f - fw) * metal;
        df[3][c] = -bc * INV_PI_F + S * (1.0f - fw) * (bc - 0.04f);
        df[4][c] = dS * F;
    }
    return mk(f[0], f[1], f[2]);
}

__device__ __forceinline__ float bsdf_pdf(const MatEval& m, v3 n, v3 wo, v3 wi, v3 h) {
    const float co = dot(n, wo), ci = dot(n, wi);
    if (co <= 0.0f || ci <= 0.0f) return 0.0f;
    if (m.type == 0) return ci * INV_PI_F;
    const float a = m.th[4] * m.th[4], a2 = a * a;
    const float ps = 0.5f * (1.0f + m.th[3]);
    const float ch = dot(n, h), oh = dot(wo, h);
    const float pspec = oh > 0.0f ? ggx_d(a2, ch, sin2(n, h)) * ch / (4.0f * oh) : 0.0f;
    return ps * pspec + (1.0f - ps) * ci * INV_PI_F;
}

// returns false if the sampled direction is not above the surface; h: the half vector of
// (wo, wi) (the sampled one for the GGX lobe)
__device__ __forceinline__ bool bsdf_sample(const MatEval& m, v3 n, v3 wo, float ul, float u1, float u2, v3& wi,
                                            v3& hv) {
    if (m.type == 1 && ul < 0.5f * (1.0f + m.th[3])) {
        const float a = m.th[4] * m.th[4], a2 = a * a;
        const float t2 = a2 * u1 / (1.0f - u1);       // tan^2 of the half-vector angle
        const float ct = 1.0f / sqrtf(1.0f + t2);
        const float st = sqrtf(t2) * ct;
        float s, c;
        sincospif(2.0f * u2, &s, &c);
        const v3 h = local_to_world(n, st * c, st * s, ct);
        const float oh = dot(wo, h);
        if (oh <= 0.0f) return false;
        wi = h * (2.0f * oh) - wo;
        hv = h;
    } else {
        wi = cosine_dir(n, u1, u2);
        hv = half_vec(wo, wi);
    }
    return dot(n, wi) > 0.0f;
}

__device__ __forceinline__ float mis2(float a, float b) {
    const float a2 = a * a;
    return a2 / (a2 + b * b);
}

// ray origin offset along the facing normal: 1e-4 * max(1, |p|_inf)
__device__ __forceinline__ v3 offset_origin(v3 p, v3 nf) {
    const float m = fmaxf(1.0f, fmaxf(fabsf(p.x), fmaxf(fabsf(p.y), fabsf(p.z))));
    return p + nf * (1e-4f * m);
}

}  // namespace mer

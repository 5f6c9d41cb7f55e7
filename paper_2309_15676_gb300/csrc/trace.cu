// Wavefront path tracer, path-replay adjoint and finite-difference pairs (sm_103a).
//
// One pass = for depth k = 1..D: extend (closest hit of every queued ray) -> shade
// (emission, next-event estimation, BSDF sampling, gradient records, compaction of the
// surviving paths into the next queue) -> shadow (any-hit of the NEE rays; adds the
// visible NEE radiance and the NEE part of the gradient record). Queues are SoA and the
// compacting appends are warp-aggregated (one atomic per warp).
//
// Passes (Sec. 6 setup: Path Replay Backpropagation; Sec. 3 Eqs. est_def, est_triv):
//   PRIMAL  - radiance per path, resolved into images;
//   ADJ_FWD - radiance per path L_total, kept for the replay;
//   REPLAY  - the same paths again (same counters); at vertex k the texture derivative
//             g_k = adj . [ T_k dF(w_l) Le G w_l / p_l  +  (L_total - L_<=k) dF(w_b) / F(w_b) ]
//             is written as a record {texel footprint, g[C]}; sampling pdfs and MIS weights
//             are treated as constants. Written in two parts so that no path state needs to
//             outlive the kernel: the shade kernel stores adj . (L_total - L_acc) dF(w_b)/F(w_b)
//             with L_acc the radiance before this vertex's NEE, and the NEE shadow ray carries
//             adj . (dN - N dF(w_b)/F(w_b)), added only if the light is visible.
// NB = 2 runs the FD pair of Eq. est_triv: branch A at pi_i, branch B at pi_{i-1}, same
// random numbers, one thread. While both branches follow the same ray ("coincident") they
// share traversal, surface interaction, light sample and shadow ray, and their gradient
// records merge into one record of g_A - g_B.
#include "kernels.cuh"
#include "wavefront.cuh"

namespace mer {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------------
// traversal
// ---------------------------------------------------------------------------------
// near and far slab planes of a node's four children along the ray: with the ray's direction
// signs fixed, the near plane of an axis is the low one for a positive component and the high one
// for a negative one, so the planes are fetched in ray order and need no per-box min/max
struct NodeRay {
    float4 nx, fx, ny, fy, nz, fz;
    int4 child;
};

__device__ __forceinline__ NodeRay load_node(const Node* __restrict__ nodes, const Node* s_nodes, int smem_n, int i,
                                             int sx, int sy, int sz) {
    const float4* p = (i < smem_n) ? reinterpret_cast<const float4*>(s_nodes + i)
                                   : reinterpret_cast<const float4*>(nodes + i);
    NodeRay n;
    if (i < smem_n) {
        n.nx = p[0 + sx]; n.fx = p[1 - sx];
        n.ny = p[2 + sy]; n.fy = p[3 - sy];
        n.nz = p[4 + sz]; n.fz = p[5 - sz];
        n.child = reinterpret_cast<const int4*>(p)[6];
    } else {
        n.nx = __ldg(p + 0 + sx); n.fx = __ldg(p + 1 - sx);
        n.ny = __ldg(p + 2 + sy); n.fy = __ldg(p + 3 - sy);
        n.nz = __ldg(p + 4 + sz); n.fz = __ldg(p + 5 - sz);
        n.child = __ldg(reinterpret_cast<const int4*>(p) + 6);
    }
    return n;
}

__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Moller-Trumbore. The three numerators and the reciprocal are independent and the decision is
// taken once at the end, without branches: lanes of a warp that would reject at different stages
// stay together, and the reciprocal's latency overlaps the other products (same arithmetic, same
// decisions as a test that rejects stage by stage).
__device__ __forceinline__ bool tri_test(const TriGeo& T, v3 o, v3 d, float& t, float& u, float& v) {
    const v3 e1 = mk(T.e1.x, T.e1.y, T.e1.z), e2 = mk(T.e2.x, T.e2.y, T.e2.z);
    const v3 pv = cross(d, e2);
    const float det = dot(e1, pv);
    const v3 tv = o - mk(T.v0.x, T.v0.y, T.v0.z);
    const v3 qv = cross(tv, e1);
    const float un = dot(tv, pv), vn = dot(d, qv), tn = dot(e2, qv);
    const float inv = 1.0f / det;
    u = un * inv;
    v = vn * inv;
    t = tn * inv;
    return det != 0.0f && u >= 0.0f && u <= 1.0f && v >= 0.0f && u + v <= 1.0f && t > 0.0f;
}

__device__ __forceinline__ TriGeo load_tri(const TriGeo* __restrict__ tris, int i) {
    const float4* p = reinterpret_cast<const float4*>(tris + i);
    TriGeo T;
    T.v0 = __ldg(p);
    T.e1 = __ldg(p + 1);
    T.e2 = __ldg(p + 2);
    return T;
}

// robust ray/sphere (Haines et al. 2019, Ray Tracing Gems ch. 7): nearest t > 0
__device__ __forceinline__ bool sphere_test(const Sphere& S, v3 o, v3 d, float& t) {
    const v3 c = mk(S.cr.x, S.cr.y, S.cr.z);
    const float r = S.cr.w;
    const v3 oc = o - c;
    const float b = dot(oc, d);
    const v3 f = oc - d * b;
    const float disc = r * r - dot(f, f);
    if (disc < 0.0f) return false;
    const float cc = dot(oc, oc) - r * r;
    const float q = -(b + copysignf(sqrtf(disc), b));
    if (q == 0.0f) return false;
    float t0 = cc / q, t1 = q;
    if (t0 > t1) { const float s = t0; t0 = t1; t1 = s; }
    if (t0 > 0.0f) { t = t0; return true; }
    if (t1 > 0.0f) { t = t1; return true; }
    return false;
}

struct Hit {
    float t, b1, b2;
    int prim;   // local: triangles [0, n_tris), spheres n_tris + i; -1 = miss
};

// algorithmic work of a traversal (counted only in the counting instantiation)
struct TravCount {
    unsigned nodes = 0;   // four-box node tests
    unsigned prims = 0;   // triangle and sphere tests
};

// One lane's traversal state: closest hit (any = false) or any hit before tmax (any = true) of
// the ray (o, d) against the problem's four-wide BVH and then its spheres. Ties in t go to the
// smaller primitive id, independent of traversal order. Deferred children go on the lane's stack;
// the scene upload refuses trees whose depth could need more than TRAV_STACK entries (three
// deferred children per inner level), and should a push still find the stack full, `complete`
// becomes false and the caller reports MER_ERR_BOUNDS through the error word.
struct TravRay {
    v3 o, d;
    float ix, iy, iz, ox, oy, oz;   // reciprocal direction and origin scaled by it
    int sx, sy, sz;                 // direction signs: which slab plane is near
    float t, b1, b2;                // closest hit so far (t = tmax initially)
    int best;                       // its triangle id (0x7fffffff: none)
    int node, sp;                   // next node (NODE_EMPTY: finished), stack depth
    bool any, hit_any, complete;
};

__device__ __forceinline__ void trav_begin(TravRay& R, v3 o, v3 d, float tmax, bool any, bool has_bvh) {
    R.o = o;
    R.d = d;
    const float dx = fabsf(d.x) < 1e-20f ? copysignf(1e-20f, d.x) : d.x;
    const float dy = fabsf(d.y) < 1e-20f ? copysignf(1e-20f, d.y) : d.y;
    const float dz = fabsf(d.z) < 1e-20f ? copysignf(1e-20f, d.z) : d.z;
    R.ix = 1.0f / dx;
    R.iy = 1.0f / dy;
    R.iz = 1.0f / dz;
    R.ox = o.x * R.ix;
    R.oy = o.y * R.iy;
    R.oz = o.z * R.iz;
    R.sx = R.ix < 0.0f ? 1 : 0;
    R.sy = R.iy < 0.0f ? 1 : 0;
    R.sz = R.iz < 0.0f ? 1 : 0;
    R.t = tmax;
    R.b1 = R.b2 = 0.0f;
    R.best = 0x7fffffff;
    R.node = has_bvh ? 0 : NODE_EMPTY;
    R.sp = 0;
    R.any = any;
    R.hit_any = false;
    R.complete = true;
}

// One step of the BVH walk: descend through inner nodes (nearest child first, the others
// deferred) until a leaf, test its triangles, take the next deferred subtree. Returns true when
// the walk has finished (stack empty, or any-hit found).
// The caller passes the tree's arrays themselves (kept in registers for the whole walk), not the
// problem record in global memory: re-reading them from it would put one more dependent load in
// front of every node fetch.
template <bool STATS>
__device__ __forceinline__ bool trav_step(const Node* __restrict__ nodes, const TriGeo* __restrict__ tris,
                                          const Node* s_nodes, int smem_n, TravRay& R, int* stack, TravCount& tc) {
    const float grow = 1.0f + 4.8e-7f;   // conservative box exit (a few ulp)
    int node = R.node;
    while (node >= 0 && node != NODE_EMPTY) {
        const NodeRay n = load_node(nodes, s_nodes, smem_n, node, R.sx, R.sy, R.sz);
        if (STATS) tc.nodes++;
        const float tfar = R.t * grow;
        // slab test of the four children; a miss (or an unused slot) sorts last
        float tn[4];
        int rf[4];
        const float nxs[4] = {n.nx.x, n.nx.y, n.nx.z, n.nx.w}, fxs[4] = {n.fx.x, n.fx.y, n.fx.z, n.fx.w};
        const float nys[4] = {n.ny.x, n.ny.y, n.ny.z, n.ny.w}, fys[4] = {n.fy.x, n.fy.y, n.fy.z, n.fy.w};
        const float nzs[4] = {n.nz.x, n.nz.y, n.nz.z, n.nz.w}, fzs[4] = {n.fz.x, n.fz.y, n.fz.z, n.fz.w};
        const int cs[4] = {n.child.x, n.child.y, n.child.z, n.child.w};
        int nh = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float t0 = fmax3(fmaf(nxs[k], R.ix, -R.ox), fmaf(nys[k], R.iy, -R.oy), fmaxf(fmaf(nzs[k], R.iz, -R.oz), 0.0f));
            const float t1 = fmin3(fmaf(fxs[k], R.ix, -R.ox), fmaf(fys[k], R.iy, -R.oy), fminf(fmaf(fzs[k], R.iz, -R.oz), tfar));
            const bool hit = t0 <= t1 && cs[k] != NODE_EMPTY;
            tn[k] = hit ? t0 : INFINITY;
            rf[k] = cs[k];
            nh += hit ? 1 : 0;
        }
        if (nh == 0) {
            node = R.sp == 0 ? NODE_EMPTY : stack[--R.sp];
            continue;
        }
        // nearest first: five compare-exchanges sort the four (t, child) pairs
#define MER_CX(i, j)                                   \
    if (tn[j] < tn[i]) {                               \
        const float tt = tn[i]; tn[i] = tn[j]; tn[j] = tt; \
        const int rr = rf[i]; rf[i] = rf[j]; rf[j] = rr;   \
    }
        MER_CX(0, 1) MER_CX(2, 3) MER_CX(0, 2) MER_CX(1, 3) MER_CX(1, 2)
#undef MER_CX
        if (nh > 3) { if (R.sp < TRAV_STACK) stack[R.sp++] = rf[3]; else R.complete = false; }
        if (nh > 2) { if (R.sp < TRAV_STACK) stack[R.sp++] = rf[2]; else R.complete = false; }
        if (nh > 1) { if (R.sp < TRAV_STACK) stack[R.sp++] = rf[1]; else R.complete = false; }
        node = rf[0];
    }
    if (node == NODE_EMPTY) {
        R.node = NODE_EMPTY;
        return true;
    }
    // leaf
    const int x = ~node;
    const int first = x >> 3, count = (x & 7) + 1;
    if (STATS) tc.prims += count;
    // two triangles per round: their loads go out together and their tests are independent; they
    // are taken in leaf order, as one at a time would
    for (int k = 0; k < count; k += 2) {
        const bool two = k + 1 < count;
        const TriGeo T0 = load_tri(tris, first + k);
        const TriGeo T1 = load_tri(tris, first + (two ? k + 1 : k));
        float t0, u0, v0, t1, u1, v1;
        const bool h0 = tri_test(T0, R.o, R.d, t0, u0, v0);
        const bool h1 = two && tri_test(T1, R.o, R.d, t1, u1, v1);
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const bool h = m == 0 ? h0 : h1;
            if (!h) continue;
            const float t = m == 0 ? t0 : t1, u = m == 0 ? u0 : u1, v = m == 0 ? v0 : v1;
            const int pid = __float_as_int(m == 0 ? T0.v0.w : T1.v0.w);
            if (R.any) {
                if (t < R.t) {
                    R.hit_any = true;
                    R.node = NODE_EMPTY;
                    return true;
                }
            } else if (t < R.t || (t == R.t && pid < R.best)) {
                R.t = t; R.b1 = u; R.b2 = v; R.best = pid;
            }
        }
    }
    R.node = R.sp == 0 ? NODE_EMPTY : stack[--R.sp];
    return R.node == NODE_EMPTY;
}

// the walk has finished: the spheres, then the hit (closest: prim -1 if none; any: prim >= 0
// if occluded)
template <bool STATS>
__device__ __forceinline__ Hit trav_end(const ProblemDev& P, TravRay& R, TravCount& tc) {
    Hit h;
    h.t = R.t;
    h.b1 = R.b1;
    h.b2 = R.b2;
    h.prim = R.any ? (R.hit_any ? 0 : -1) : (R.best == 0x7fffffff ? -1 : R.best);
    if (STATS) tc.prims += P.n_sph;
    for (int i = 0; i < P.n_sph && !(R.any && h.prim >= 0); ++i) {
        const Sphere S = P.sph[i];
        float t;
        if (sphere_test(S, R.o, R.d, t)) {
            if (R.any) {
                if (t < R.t) h.prim = P.n_tris + i;
            } else if (t < h.t) {
                h.t = t; h.prim = P.n_tris + i; h.b1 = h.b2 = 0.0f;
            }
        }
    }
    return h;
}

// ---------------------------------------------------------------------------------
// shading helpers
// ---------------------------------------------------------------------------------
struct Surf {
    v3 p, n;
    float u, v;
    int mat, light;
};

__device__ __forceinline__ void surface(const ProblemDev& P, v3 o, v3 d, const Hit& h, Surf& s) {
    s.p = o + d * h.t;
    if (h.prim < P.n_tris) {
        const TriAttr at = P.attr[h.prim];
        s.n = mk(at.n[0], at.n[1], at.n[2]);
        const float w = 1.0f - h.b1 - h.b2;
        s.u = w * at.uv[0] + h.b1 * at.uv[2] + h.b2 * at.uv[4];
        s.v = w * at.uv[1] + h.b1 * at.uv[3] + h.b2 * at.uv[5];
        s.mat = at.mat;
        s.light = at.light;
    } else {
        const Sphere S = P.sph[h.prim - P.n_tris];
        s.n = (s.p - mk(S.cr.x, S.cr.y, S.cr.z)) * (1.0f / S.cr.w);
        float uu = atan2f(s.n.y, s.n.x) * (0.5f * INV_PI_F);
        if (uu < 0.0f) uu += 1.0f;
        const float vv = acosf(fminf(1.0f, fmaxf(-1.0f, s.n.z))) * INV_PI_F;
        s.u = S.uvr.x + uu * (S.uvr.y - S.uvr.x);
        s.v = S.uvr.z + vv * (S.uvr.w - S.uvr.z);
        s.mat = S.mat;
        s.light = -1;
    }
}

struct Foot {
    int x0, y0;
    float fx, fy;
};

// bilinear, clamp-to-edge, texel centres at (x + 1/2) / W
__device__ __forceinline__ void fetch(const float* __restrict__ tex, const ProblemDev& P, float u, float v,
                                      MatEval& m, Foot& f) {
    u = fminf(fmaxf(u, 0.0f), 1.0f);
    v = fminf(fmaxf(v, 0.0f), 1.0f);
    const int W = P.tex_w, H = P.tex_h, C = P.tex_c;
    const float x = u * (float)W - 0.5f, y = v * (float)H - 0.5f;
    const float xf = floorf(x), yf = floorf(y);
    f.x0 = (int)xf;
    f.y0 = (int)yf;
    f.fx = x - xf;
    f.fy = y - yf;
    const int xa = max(f.x0, 0), xb = min(f.x0 + 1, W - 1);
    const int ya = max(f.y0, 0), yb = min(f.y0 + 1, H - 1);
    const float w00 = (1.0f - f.fx) * (1.0f - f.fy), w10 = f.fx * (1.0f - f.fy);
    const float w01 = (1.0f - f.fx) * f.fy, w11 = f.fx * f.fy;
    const float* t00 = tex + ((size_t)ya * W + xa) * C;
    const float* t10 = tex + ((size_t)ya * W + xb) * C;
    const float* t01 = tex + ((size_t)yb * W + xa) * C;
    const float* t11 = tex + ((size_t)yb * W + xb) * C;
#pragma unroll
    for (int j = 0; j < MAXC; ++j) {
        if (j < C)
            m.th[j] = w00 * __ldg(t00 + j) + w10 * __ldg(t10 + j) + w01 * __ldg(t01 + j) + w11 * __ldg(t11 + j);
        else
            m.th[j] = 0.0f;
    }
}

struct LightSample {
    bool ok;
    v3 wi, le;
    float pdf, tmax;
};

// uniform choice among {quads..., env}; quads by area, env by a cosine lobe around nf
__device__ __forceinline__ LightSample sample_light(const ProblemDev& P, v3 po, v3 nf, uint4 r) {
    LightSample L;
    L.ok = false;
    const int nL = P.n_lights;
    if (nL == 0) return L;
    const int l = (int)(((uint64_t)(r.x >> 8) * (uint64_t)nL) >> 24);
    const float u1 = u01(r.y), u2 = u01(r.z);
    if (l < P.n_quads) {
        const QuadLight Q = P.quads[l];
        const v3 y = mk(Q.p0[0], Q.p0[1], Q.p0[2]) + mk(Q.e1[0], Q.e1[1], Q.e1[2]) * u1 +
                     mk(Q.e2[0], Q.e2[1], Q.e2[2]) * u2;
        const v3 w = y - po;
        const float d2 = dot(w, w), dist = sqrtf(d2);
        const v3 wi = w * (1.0f / dist);
        const float cl = -dot(wi, mk(Q.n[0], Q.n[1], Q.n[2]));
        if (cl <= 0.0f || dot(wi, nf) <= 0.0f) return L;
        L.ok = true;
        L.wi = wi;
        L.pdf = d2 / (Q.area * cl * (float)nL);
        L.tmax = dist * (1.0f - 1e-4f);
        L.le = mk(Q.le[0], Q.le[1], Q.le[2]);
    } else {
        const v3 wi = cosine_dir(nf, u1, u2);
        const float cs = dot(wi, nf);
        if (cs <= 0.0f) return L;
        L.ok = true;
        L.wi = wi;
        L.pdf = cs * INV_PI_F / (float)nL;
        L.tmax = INFINITY;
        L.le = mk(P.env[0], P.env[1], P.env[2]);
    }
    return L;
}

__device__ __forceinline__ void camera_ray(const ProblemDev& P, uint32_t pixel, float j0, float j1, v3& o, v3& d) {
    const uint32_t px = pixel % (uint32_t)P.width, py = pixel / (uint32_t)P.width;
    const float sx = 2.0f * ((float)px + j0) / (float)P.width - 1.0f;
    const float sy = 1.0f - 2.0f * ((float)py + j1) / (float)P.height;
    o = mk(P.cam_o[0], P.cam_o[1], P.cam_o[2]);
    d = normalize(mk(P.cam_f[0], P.cam_f[1], P.cam_f[2]) + mk(P.cam_r[0], P.cam_r[1], P.cam_r[2]) * sx +
                  mk(P.cam_u[0], P.cam_u[1], P.cam_u[2]) * sy);
}

// Pixel of a problem's local path index (modulo its pixel count): images whose sides are multiples
// of 16 are walked in 16 x 16 tiles, so that a warp's camera rays are a 16 x 2 patch (coherent
// traversal, and the queue compaction carries some of that order to later depths); others row by
// row. Counters, images and adjoint images are indexed by the pixel itself.
__device__ __forceinline__ uint32_t path_pixel(const ProblemDev& P, uint32_t local) {
    if ((P.width & 15) || (P.height & 15)) return local;
    const uint32_t tiles_x = (uint32_t)P.width >> 4;
    const uint32_t tile = local >> 8, k = local & 255u;
    const uint32_t ty = tile / tiles_x, tx = tile - ty * tiles_x;
    return ((ty << 4) + (k >> 4)) * (uint32_t)P.width + (tx << 4) + (k & 15u);
}

struct PathId {
    int q, e;
    uint32_t pixel, sample, iter;
    int spp;
};

__device__ __forceinline__ PathId decode_path(const PassArgs& A, int64_t g) {
    PathId id;
    int64_t local = g;
    if (A.inl_prob >= 0) {
        id.e = 0;
        id.q = A.inl_prob;
    } else {
        id.e = find_entry(A.path_off, A.n_entries, g);
        id.q = A.entry_prob[id.e];
        local = g - A.path_off[id.e];
    }
    const ProblemDev& P = A.probs[id.q];
    id.pixel = path_pixel(P, (uint32_t)(local % P.n_pix));
    id.sample = (uint32_t)(local / P.n_pix) + (uint32_t)A.sample_base;
    id.iter = A.iter_override >= 0 ? (uint32_t)A.iter_override : (uint32_t)A.pstate[id.q].iteration;
    id.spp = A.spp_override > 0 ? A.spp_override : (A.fd_kind ? P.spp_fd : P.spp_prop);
    return id;
}

__device__ __forceinline__ const float* branch_tex(const PassArgs& A, const ProblemDev& P, int q, int b) {
    if (A.tex_over[b]) return A.tex_over[b];
    const int cur = A.pstate[q].cur;
    return P.pslot[b == 0 ? cur : (cur ^ 1)];
}

// warp-aggregated append: returns this lane's first slot; all 32 lanes must call
__device__ __forceinline__ uint32_t warp_append(uint32_t* ctr, uint32_t cnt) {
    const unsigned lane = threadIdx.x & 31u;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(FULL, incl, o);
        if (lane >= (unsigned)o) incl += v;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    uint32_t base = 0;
    if (lane == 31 && total) base = atomicAdd(ctr, total);
    base = __shfl_sync(FULL, base, 31);
    return base + incl - cnt;
}

__device__ __forceinline__ void set_err(const PassArgs& A, int code) { atomicCAS(&A.cnt[CNT_ERR], 0u, (uint32_t)code); }

// Passes with at least this many paths append their continuation rays grouped by direction
// octant within each block (block_append_grouped); smaller passes append per warp.
constexpr int64_t GROUP_MIN_PATHS = (int64_t)1 << 20;

// Block-aggregated append grouped by key (0..7): the block's entries of each key get contiguous
// slots, keys in ascending order, with one atomic per block. Every thread of the block must call
// it (it synchronises the block); returns this thread's slot if `want`.
__device__ __forceinline__ uint32_t block_append_grouped(uint32_t* ctr, bool want, int key) {
    __shared__ uint32_t s_cnt[8];
    if (threadIdx.x < 8) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    const uint32_t rank = want ? atomicAdd(&s_cnt[key], 1u) : 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t c[8], tot = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            c[k] = s_cnt[k];
            tot += c[k];
        }
        uint32_t off = tot ? atomicAdd(ctr, tot) : 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            s_cnt[k] = off;
            off += c[k];
        }
    }
    __syncthreads();
    const uint32_t slot = s_cnt[key] + rank;
    __syncthreads();   // every thread has read its base before the next call resets them
    return slot;
}

extern __shared__ float4 s_dyn[];

// stages the first nodes of problem smem_prob's BVH (its top levels) in shared memory;
// returns how many were staged
__device__ __forceinline__ int stage_nodes(const PassArgs& A, const Node*& s_nodes) {
    Node* s = reinterpret_cast<Node*>(s_dyn);
    s_nodes = s;
    int cnt = 0;
    if (A.smem_nodes > 0) {
        const ProblemDev& P = A.probs[A.smem_prob];
        cnt = P.nodes ? min(A.smem_nodes, P.n_nodes) : 0;
        const float4* src = reinterpret_cast<const float4*>(P.nodes);
        float4* dst = reinterpret_cast<float4*>(s);
        for (int i = threadIdx.x; i < cnt * 8; i += blockDim.x) dst[i] = __ldg(src + i);
        __syncthreads();
    }
    return cnt;
}

// adds a warp's traversal counts to stats[2*cls], stats[2*cls+1]; all lanes must call
__device__ __forceinline__ void flush_counts(const PassArgs& A, int cls, const TravCount& tc) {
    const unsigned nsum = __reduce_add_sync(FULL, tc.nodes), psum = __reduce_add_sync(FULL, tc.prims);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(A.stats + 2 * cls, (unsigned long long)nsum);
        atomicAdd(A.stats + 2 * cls + 1, (unsigned long long)psum);
    }
}

// ---------------------------------------------------------------------------------
// shade
// ---------------------------------------------------------------------------------
// blocks per SM the register budget keeps: the FD-pair replay is the heaviest, the proportional
// radiance pass the lightest
template <int NB, int MODE>
constexpr int shade_min_blocks() {
    return (NB == 2 && MODE == MODE_REPLAY) ? 1 : (NB == 1 && MODE != MODE_REPLAY) ? 3 : 2;
}

template <int NB, int MODE>
__global__ void __launch_bounds__(256, (shade_min_blocks<NB, MODE>())) k_shade(PassArgs A, int depth) {
    constexpr bool GRAD = MODE == MODE_REPLAY;
    // hit store (PassArgs::hs): the ADJ_FWD pass records what its replay needs, the replay reads
    // it back instead of tracing
    const bool store = MODE != MODE_REPLAY && A.hs != nullptr;
    const bool stored = MODE == MODE_REPLAY && A.hs != nullptr;
    const bool first = depth == 1;
    const int64_t n = first ? A.n_paths : min((int64_t)A.cnt[CNT_Q + depth], A.qcap);
    // whole blocks iterate together (the grouped append synchronises the block)
    const int64_t nb = (n + blockDim.x - 1) / blockDim.x * blockDim.x;
    const bool grouped = A.n_paths >= GROUP_MIN_PATHS;
    const int qi = depth & 1, qo = qi ^ 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x; j0 < nb; j0 += stride) {
        const int64_t j = j0 + threadIdx.x;
        const bool valid = j < n;
        uint32_t flags = 0;
        int64_t g = 0;
        PathId id{};
        v3 o[NB], d[NB], beta[NB];
        float pdfb[NB], pdfenv[NB];
        if (valid) {
            if (first) {
                g = j;
                id = decode_path(A, g);
                flags = (NB == 2) ? (FLAG_A | FLAG_B | FLAG_COINC) : FLAG_A;
                if (A.fd_kind && A.iter_override < 0 && A.pstate[id.q].iteration == 0) flags = 0;
                const ProblemDev& P = A.probs[id.q];
                const uint4 r = draw(P.seed, P.key_id, id.pixel, id.sample, id.iter, A.stream, 0, 0);
                v3 oc, dc;
                camera_ray(P, id.pixel, u01(r.x), u01(r.y), oc, dc);
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    o[b] = oc; d[b] = dc; beta[b] = mk(1, 1, 1); pdfb[b] = 0.0f; pdfenv[b] = 0.0f;
                }
            } else {
                g = A.qu[qi][QU_PATH * A.qcap + j];
                flags = A.qu[qi][QU_FLAGS * A.qcap + j];
                id = decode_path(A, g);
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const float* f = A.qf[qi] + (size_t)(b * QF_PER_BRANCH) * A.qcap + j;
                    o[b] = mk(f[(QF_O + 0) * A.qcap], f[(QF_O + 1) * A.qcap], f[(QF_O + 2) * A.qcap]);
                    d[b] = mk(f[(QF_D + 0) * A.qcap], f[(QF_D + 1) * A.qcap], f[(QF_D + 2) * A.qcap]);
                    beta[b] = mk(f[(QF_BETA + 0) * A.qcap], f[(QF_BETA + 1) * A.qcap], f[(QF_BETA + 2) * A.qcap]);
                    pdfb[b] = f[QF_PDFB * A.qcap];
                    pdfenv[b] = f[QF_PDFENV * A.qcap];
                }
            }
        }
        const int q = id.q;
        const ProblemDev& P = A.probs[q];
        const bool coinc = (NB == 2) && (flags & FLAG_COINC);

        // ---- emission / termination ----
        bool alive[NB];
        Surf s[NB];
        v3 lacc[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            alive[b] = valid && (flags & (1u << b));
            lacc[b] = mk(0, 0, 0);
            if (!alive[b]) continue;
            if (!first) {
                lacc[b] = mk(A.lacc[(size_t)(b * 3 + 0) * A.qcap + g], A.lacc[(size_t)(b * 3 + 1) * A.qcap + g],
                             A.lacc[(size_t)(b * 3 + 2) * A.qcap + g]);
            }
            const int hb = (b == 1 && coinc) ? 0 : b;
            Hit h;
            if (stored) {
                const float4 hv = A.hs[((int64_t)hb * A.hs_depth + depth - 1) * A.hs_cap + g];
                h.t = hv.x;
                h.b1 = hv.y;
                h.b2 = hv.z;
                h.prim = __float_as_int(hv.w);
                if (h.prim < -1 || h.prim >= P.n_tris + P.n_sph) {   // not this pass's path: never used
                    set_err(A, MER_ERR_STATE);
                    h.prim = -1;
                }
            } else {
                h.t = A.hitf[(size_t)(hb * HF_PER_BRANCH + HF_T) * A.qcap + j];
                h.b1 = A.hitf[(size_t)(hb * HF_PER_BRANCH + HF_B1) * A.qcap + j];
                h.b2 = A.hitf[(size_t)(hb * HF_PER_BRANCH + HF_B2) * A.qcap + j];
                h.prim = A.hitp[(size_t)hb * A.qcap + j];
                if (store && hb == b)   // ADJ_FWD: keep the hit for the replay, by path
                    A.hs[((int64_t)b * A.hs_depth + depth - 1) * A.hs_cap + g] =
                        make_float4(h.t, h.b1, h.b2, __int_as_float(h.prim));
            }
            if (h.prim < 0) {
                if (P.has_env) {
                    const float w = first ? 1.0f : mis2(pdfb[b], pdfenv[b]);
                    lacc[b] = lacc[b] + mk(beta[b].x * P.env[0], beta[b].y * P.env[1], beta[b].z * P.env[2]) * w;
                }
                alive[b] = false;
                continue;
            }
            if (b == 1 && coinc) s[1] = s[0]; else surface(P, o[b], d[b], h, s[b]);
            if (s[b].light >= 0) {
                const QuadLight& Q = P.quads[s[b].light];
                const float cl = -dot(d[b], mk(Q.n[0], Q.n[1], Q.n[2]));
                if (cl > 0.0f) {
                    float w = 1.0f;
                    if (!first) {
                        const float pl = h.t * h.t / (Q.area * cl * (float)P.n_lights);
                        w = mis2(pdfb[b], pl);
                    }
                    lacc[b] = lacc[b] + mk(beta[b].x * Q.le[0], beta[b].y * Q.le[1], beta[b].z * Q.le[2]) * w;
                }
            }
            if (depth >= P.max_depth) alive[b] = false;
        }
        // write back the radiance accumulated so far (NEE of this vertex is added by the shadow kernel)
        if (valid) {
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if (first || (flags & (1u << b))) {
                    A.lacc[(size_t)(b * 3 + 0) * A.qcap + g] = lacc[b].x;
                    A.lacc[(size_t)(b * 3 + 1) * A.qcap + g] = lacc[b].y;
                    A.lacc[(size_t)(b * 3 + 2) * A.qcap + g] = lacc[b].z;
                }
            }
        }

        // ---- vertex: NEE + BSDF sample (+ gradient terms) ----
        bool any_alive = false;
#pragma unroll
        for (int b = 0; b < NB; ++b) any_alive |= alive[b];

        bool sh_want[NB], cont[NB], rec_want[NB], textured[NB];
        LightSample ls[NB];
        v3 contrib[NB], wi_b[NB];
        float gbase[NB][MAXC], gnee[NB][MAXC];
        Foot foot[NB];
        v3 po[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            sh_want[b] = cont[b] = rec_want[b] = textured[b] = false;
            ls[b].ok = false;
        }
        // FD pair with a shared path: branch 1 (pi_{i-1}) takes branch 0's light sample, BSDF sample
        // and densities, and evaluates only its own integrand along them
        const bool shared = NB == 2 && P.fd_shared != 0;
        float pbN0 = 0.0f, pbC0 = 0.0f;
        v3 wiC0 = mk(0, 0, 0), hC0 = mk(0, 0, 1);
        bool okC0 = false;
        if (any_alive) {
            const uint4 r0 = draw(P.seed, P.key_id, id.pixel, id.sample, id.iter, A.stream, (uint32_t)depth, 0);
            const uint4 r1 = draw(P.seed, P.key_id, id.pixel, id.sample, id.iter, A.stream, (uint32_t)depth, 1);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if (!alive[b]) continue;
                const v3 wo = -d[b];
                const v3 nf = dot(s[b].n, d[b]) < 0.0f ? s[b].n : -s[b].n;
                po[b] = offset_origin(s[b].p, nf);
                const Material M = P.mats[s[b].mat];
                MatEval m;
                m.type = M.type;
                textured[b] = M.textured != 0;
                if (textured[b]) {
                    fetch(branch_tex(A, P, q, b), P, s[b].u, s[b].v, m, foot[b]);
                } else {
#pragma unroll
                    for (int k = 0; k < MAXC; ++k) m.th[k] = M.c[k];
                }
                const bool wg = GRAD && textured[b];
                v3 adj = mk(0, 0, 0);
                if (wg) {
                    const float* dsrc = A.dimg_over[b] ? A.dimg_over[b] : (A.fd_kind ? (b ? P.dimgB : P.dimgA) : P.dimg);
                    const float* di = dsrc + (size_t)id.pixel * 3;
                    const float inv = 1.0f / (float)id.spp;
                    adj = mk(di[0] * inv, di[1] * inv, di[2] * inv);
                }
                // next-event estimation
                if (b == 1 && coinc) ls[1] = ls[0]; else ls[b] = sample_light(P, po[b], nf, r0);
                float dN[MAXC];
#pragma unroll
                for (int k = 0; k < MAXC; ++k) dN[k] = 0.0f;
                contrib[b] = mk(0, 0, 0);
                if (ls[b].ok) {
                    float df[MAXC][3];
                    const v3 hl = half_vec(wo, ls[b].wi);
                    const v3 f = wg ? bsdf_f_grad(m, nf, wo, ls[b].wi, hl, df) : bsdf_f(m, nf, wo, ls[b].wi, hl);
                    const float pb = (shared && b == 1) ? pbN0 : bsdf_pdf(m, nf, wo, ls[b].wi, hl);
                    if (b == 0) pbN0 = pb;
                    const float qn = dot(ls[b].wi, nf) * mis2(ls[b].pdf, pb) / ls[b].pdf;
                    contrib[b] = mk(beta[b].x * f.x * ls[b].le.x, beta[b].y * f.y * ls[b].le.y,
                                    beta[b].z * f.z * ls[b].le.z) * qn;
                    if (wg) {
                        const v3 k3 = mk(adj.x * beta[b].x * ls[b].le.x, adj.y * beta[b].y * ls[b].le.y,
                                         adj.z * beta[b].z * ls[b].le.z) * qn;
#pragma unroll
                        for (int k = 0; k < MAXC; ++k) dN[k] = k3.x * df[k][0] + k3.y * df[k][1] + k3.z * df[k][2];
                    }
                    // (the storing ADJ_FWD pass tests every shadow ray its replay will need)
                    sh_want[b] = wg || (store && textured[b]) || contrib[b].x != 0.0f || contrib[b].y != 0.0f ||
                                 contrib[b].z != 0.0f;
                }
                // BSDF sample for the continuation
                v3 wi;
                bool ok;
                float df[MAXC][3];
                v3 f = mk(0, 0, 0);
                float pb = 0.0f;
                if (shared && b == 1) {
                    wi = wiC0;
                    ok = okC0;
                    pb = pbC0;
                    if (ok) f = wg ? bsdf_f_grad(m, nf, wo, wi, hC0, df) : bsdf_f(m, nf, wo, wi, hC0);
                } else {
                    v3 hs;
                    ok = bsdf_sample(m, nf, wo, u01(r1.x), u01(r1.y), u01(r1.z), wi, hs);
                    if (ok) {
                        f = wg ? bsdf_f_grad(m, nf, wo, wi, hs, df) : bsdf_f(m, nf, wo, wi, hs);
                        pb = bsdf_pdf(m, nf, wo, wi, hs);
                        ok = pb > 0.0f;
                    }
                    if (b == 0) {
                        okC0 = ok;
                        wiC0 = wi;
                        hC0 = hs;
                        pbC0 = pb;
                    }
                }
                if (wg) {
                    rec_want[b] = true;
                    // ratio dF/F per channel of the continuation (0 where F = 0)
                    v3 lrem = mk(0, 0, 0), nsub = mk(0, 0, 0);
                    if (ok) {
                        const float* lt = A.ltot;
                        const v3 L = mk(lt[(size_t)(b * 3 + 0) * A.qcap + g], lt[(size_t)(b * 3 + 1) * A.qcap + g],
                                        lt[(size_t)(b * 3 + 2) * A.qcap + g]);
                        const v3 ir = mk(f.x != 0.0f ? 1.0f / f.x : 0.0f, f.y != 0.0f ? 1.0f / f.y : 0.0f,
                                         f.z != 0.0f ? 1.0f / f.z : 0.0f);
                        lrem = mk(adj.x * (L.x - lacc[b].x) * ir.x, adj.y * (L.y - lacc[b].y) * ir.y,
                                  adj.z * (L.z - lacc[b].z) * ir.z);
                        nsub = mk(adj.x * contrib[b].x * ir.x, adj.y * contrib[b].y * ir.y, adj.z * contrib[b].z * ir.z);
                    }
#pragma unroll
                    for (int k = 0; k < MAXC; ++k) {
                        gbase[b][k] = ok ? (lrem.x * df[k][0] + lrem.y * df[k][1] + lrem.z * df[k][2]) : 0.0f;
                        gnee[b][k] = dN[k] - (ok ? (nsub.x * df[k][0] + nsub.y * df[k][1] + nsub.z * df[k][2]) : 0.0f);
                    }
                }
                if (ok) {
                    const float cs = dot(wi, nf);
                    const float sc = cs / pb;
                    beta[b] = mk(beta[b].x * f.x * sc, beta[b].y * f.y * sc, beta[b].z * f.z * sc);
                    pdfb[b] = pb;
                    pdfenv[b] = P.has_env ? cs * INV_PI_F / (float)P.n_lights : 0.0f;
                    wi_b[b] = wi;
                    cont[b] = true;
                }
            }
        }

        // ---- stored replay: the NEE shadow rays' visibility from the ADJ_FWD pass ----
        if (stored && valid) {
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if (!sh_want[b]) continue;
                if (!A.hvis[((int64_t)b * A.hs_depth + depth - 1) * A.hs_cap + g]) continue;
                const v3 l = lacc[b] + contrib[b];
                A.lacc[(size_t)(b * 3 + 0) * A.qcap + g] = l.x;
                A.lacc[(size_t)(b * 3 + 1) * A.qcap + g] = l.y;
                A.lacc[(size_t)(b * 3 + 2) * A.qcap + g] = l.z;
                if (rec_want[b]) {
#pragma unroll
                    for (int k = 0; k < MAXC; ++k) gbase[b][k] += gnee[b][k];
                }
            }
        }

        // ---- records (REPLAY) ----
        const bool merged = coinc && rec_want[0] && (NB == 2 && rec_want[NB - 1]);
        uint32_t rec_idx[NB];
        if (GRAD) {
            uint32_t nrec = 0;
            if (merged) nrec = 1;
            else {
#pragma unroll
                for (int b = 0; b < NB; ++b) nrec += rec_want[b] ? 1u : 0u;
            }
            const uint32_t base = warp_append(&A.cnt[CNT_R], nrec);
            uint32_t k = 0;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                rec_idx[b] = 0xffffffffu;
                if (!rec_want[b]) continue;
                if (merged && b == 1) { rec_idx[1] = rec_idx[0]; continue; }
                rec_idx[b] = base + k++;
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if (!rec_want[b] || (merged && b == 1)) continue;
                const uint32_t r = rec_idx[b];
                if (r >= A.rcap) { set_err(A, MER_ERR_BOUNDS); rec_idx[b] = 0xffffffffu; continue; }
                const float sg = (b == 1) ? -1.0f : 1.0f;
                float gv[MAXC];
#pragma unroll
                for (int k2 = 0; k2 < MAXC; ++k2)
                    gv[k2] = merged ? gbase[0][k2] - gbase[NB - 1][k2] : sg * gbase[b][k2];
                const uint32_t pos =
                    ((uint32_t)q << 24) | ((uint32_t)(foot[b].y0 + 1) << 12) | (uint32_t)(foot[b].x0 + 1);
                float4* dst = reinterpret_cast<float4*>(A.rec + r);
                dst[0] = make_float4(__uint_as_float(pos), foot[b].fx, foot[b].fy, gv[0]);
                dst[1] = make_float4(gv[1], gv[2], gv[3], gv[4]);
            }
            if (merged) rec_idx[NB - 1] = rec_idx[0];
        }

        // ---- shadow rays (none in a stored replay) ----
        if (!stored) {
            const bool sh_shared = coinc && ls[0].ok;   // one shadow ray serves both branches
            uint32_t nsh = 0;
            if (sh_shared) nsh = (sh_want[0] || (NB == 2 && sh_want[NB - 1])) ? 1u : 0u;
            else {
#pragma unroll
                for (int b = 0; b < NB; ++b) nsh += sh_want[b] ? 1u : 0u;
            }
            const uint32_t base = warp_append(&A.cnt[CNT_S + depth], nsh);
            uint32_t k = 0;
#pragma unroll
            for (int e = 0; e < NB; ++e) {
                // entry e: shared entry uses e == 0 only; separate entries one per branch
                bool make = sh_shared ? (e == 0 && nsh) : sh_want[e];
                if (!make) continue;
                const uint32_t si = base + k++;
                if (si >= A.shcap) { set_err(A, MER_ERR_BOUNDS); continue; }
                uint32_t mask = 0;
                if (sh_shared) {
#pragma unroll
                    for (int b = 0; b < NB; ++b) mask |= sh_want[b] ? (1u << b) : 0u;
                } else {
                    mask = 1u << e;
                }
                const int bsrc = e;
                float* F = A.shf;
                const size_t C = (size_t)A.shcap;
                F[(SF_O + 0) * C + si] = po[bsrc].x;
                F[(SF_O + 1) * C + si] = po[bsrc].y;
                F[(SF_O + 2) * C + si] = po[bsrc].z;
                F[(SF_D + 0) * C + si] = ls[bsrc].wi.x;
                F[(SF_D + 1) * C + si] = ls[bsrc].wi.y;
                F[(SF_D + 2) * C + si] = ls[bsrc].wi.z;
                F[SF_TMAX * C + si] = ls[bsrc].tmax;
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    if (!(mask & (1u << b))) continue;
                    const size_t base_f = SF_SLOT + (size_t)b * SF_PER_SLOT;
                    F[(base_f + 0) * C + si] = contrib[b].x;
                    F[(base_f + 1) * C + si] = contrib[b].y;
                    F[(base_f + 2) * C + si] = contrib[b].z;
                    if (GRAD) {
                        const float sg = (b == 1) ? -1.0f : 1.0f;
#pragma unroll
                        for (int k2 = 0; k2 < MAXC; ++k2) F[(base_f + 3 + k2) * C + si] = sg * gnee[b][k2];
                        A.shu[(SU_REC + b) * C + si] = rec_want[b] ? rec_idx[b] : 0xffffffffu;
                    }
                }
                A.shu[SU_PATH * C + si] = (uint32_t)g;
                A.shu[SU_META * C + si] = (uint32_t)q | (mask << 8);
            }
        }

        // ---- continuation (compacted) ----
        {
            bool any_cont = false;
#pragma unroll
            for (int b = 0; b < NB; ++b) any_cont |= cont[b];
            // a large pass groups the block's continuation rays by direction octant, so that
            // the next traversal's warps take runs of rays heading the same way
            uint32_t slot;
            if (grouped) {
                const v3 dc = cont[0] ? wi_b[0] : wi_b[NB - 1];
                const int oct = any_cont ? ((dc.x < 0.0f) | ((dc.y < 0.0f) << 1) | ((dc.z < 0.0f) << 2)) : 0;
                slot = block_append_grouped(&A.cnt[CNT_Q + depth + 1], any_cont, oct);
            } else {
                slot = warp_append(&A.cnt[CNT_Q + depth + 1], any_cont ? 1u : 0u);
            }
            if (any_cont) {
                if (slot >= A.qcap) {
                    set_err(A, MER_ERR_BOUNDS);
                } else {
                    uint32_t nf = (uint32_t)q << 8;
#pragma unroll
                    for (int b = 0; b < NB; ++b) nf |= cont[b] ? (1u << b) : 0u;
                    if (NB == 2 && coinc && cont[0] && cont[NB - 1] &&
                        wi_b[0].x == wi_b[NB - 1].x && wi_b[0].y == wi_b[NB - 1].y && wi_b[0].z == wi_b[NB - 1].z)
                        nf |= FLAG_COINC;
                    A.qu[qo][QU_PATH * A.qcap + slot] = (uint32_t)g;
                    A.qu[qo][QU_FLAGS * A.qcap + slot] = nf;
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        if (!cont[b]) continue;
                        float* f = A.qf[qo] + (size_t)(b * QF_PER_BRANCH) * A.qcap + slot;
                        f[(QF_O + 0) * A.qcap] = po[b].x;
                        f[(QF_O + 1) * A.qcap] = po[b].y;
                        f[(QF_O + 2) * A.qcap] = po[b].z;
                        f[(QF_D + 0) * A.qcap] = wi_b[b].x;
                        f[(QF_D + 1) * A.qcap] = wi_b[b].y;
                        f[(QF_D + 2) * A.qcap] = wi_b[b].z;
                        f[(QF_BETA + 0) * A.qcap] = beta[b].x;
                        f[(QF_BETA + 1) * A.qcap] = beta[b].y;
                        f[(QF_BETA + 2) * A.qcap] = beta[b].z;
                        f[QF_PDFB * A.qcap] = pdfb[b];
                        f[QF_PDFENV * A.qcap] = pdfenv[b];
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------
// trace: one launch consumes two independent queues that shade(depth_ext - 1) produced —
// the continuation rays of depth depth_ext (closest hit) and the NEE shadow rays of depth
// depth_sh = depth_ext - 1 (any hit). The first launch of a pass has no shadow rays; the
// last one has no continuation rays.
//
// A work unit is one ray: units [0, n_eu) are continuation rays (NB = 2: entry u >> 1, branch
// u & 1, so an FD pair's two rays take two lanes), units [n_eu, n_eu + n_sh) the shadow rays.
// Units are fetched dynamically (persistent threads with dynamic ray fetching, after Aila and
// Laine 2009): every lane keeps its own walk, and whenever A.refill or more lanes of a warp are
// idle, those lanes take the next units from the launch's fetch counter (one atomic per warp),
// so a warp does not wait for its slowest ray while units remain. Once they are all taken, a
// launch lasts as long as its longest walks, each a chain of dependent node and triangle tests on
// one lane; the idle lanes then split those walks by taking over their deferred subtrees (the
// cooperative tail below).
// ---------------------------------------------------------------------------------
struct Unit {
    int64_t j;   // queue entry
    int b;       // branch of a continuation ray; -1: shadow ray
    int q;       // problem
};

// starts unit u's walk; false if the unit traces nothing (a branch that ended, a problem without
// FD samples at iteration 0, or the second branch of a coincident pair, whose hit the first
// branch's unit writes)
template <int NB>
__device__ __forceinline__ bool unit_setup(const PassArgs& A, int depth_ext, int64_t u, int64_t n_eu, Unit& U,
                                           TravRay& R) {
    v3 o, d;
    if (u < n_eu) {
        U.j = NB == 2 ? (u >> 1) : u;
        U.b = NB == 2 ? (int)(u & 1) : 0;
        if (depth_ext == 1) {
            if (U.b == 1) return false;   // both branches start on the same camera ray
            const PathId id = decode_path(A, U.j);
            U.q = id.q;
            if (A.fd_kind && A.iter_override < 0 && A.pstate[U.q].iteration == 0) return false;
            const ProblemDev& P = A.probs[U.q];
            const uint4 r = draw(P.seed, P.key_id, id.pixel, id.sample, id.iter, A.stream, 0, 0);
            camera_ray(P, id.pixel, u01(r.x), u01(r.y), o, d);
        } else {
            const int qi = depth_ext & 1;
            const uint32_t flags = A.qu[qi][QU_FLAGS * A.qcap + U.j];
            if (!(flags & (1u << U.b)) || (U.b == 1 && (flags & FLAG_COINC))) return false;
            U.q = (flags >> 8) & 0xff;
            const float* f = A.qf[qi] + (size_t)(U.b * QF_PER_BRANCH) * A.qcap + U.j;
            o = mk(f[(QF_O + 0) * A.qcap], f[(QF_O + 1) * A.qcap], f[(QF_O + 2) * A.qcap]);
            d = mk(f[(QF_D + 0) * A.qcap], f[(QF_D + 1) * A.qcap], f[(QF_D + 2) * A.qcap]);
        }
        trav_begin(R, o, d, INFINITY, false, A.probs[U.q].nodes != nullptr);
    } else {
        U.j = u - n_eu;
        U.b = -1;
        const size_t C = (size_t)A.shcap;
        const float* F = A.shf;
        o = mk(F[(SF_O + 0) * C + U.j], F[(SF_O + 1) * C + U.j], F[(SF_O + 2) * C + U.j]);
        d = mk(F[(SF_D + 0) * C + U.j], F[(SF_D + 1) * C + U.j], F[(SF_D + 2) * C + U.j]);
        U.q = A.shu[SU_META * C + U.j] & 0xff;
        trav_begin(R, o, d, F[SF_TMAX * C + U.j], true, A.probs[U.q].nodes != nullptr);
    }
    return true;
}

// the walk of unit U has finished: a continuation ray writes its closest hit; a shadow ray whose
// light is visible adds the NEE radiance to its path's accumulator and (replay) the NEE part of the
// gradient to its record; a radiance pass with a hit store also keeps the visibility for its replay
template <int NB, int MODE, bool STATS>
__device__ __forceinline__ void unit_finish(const PassArgs& A, int depth_sh, const Unit& U, TravRay& R,
                                            TravCount& tc) {
    const Hit h = trav_end<STATS>(A.probs[U.q], R, tc);
    if (!R.complete) set_err(A, MER_ERR_BOUNDS);
    if (U.b >= 0) {
        A.hitf[(size_t)(U.b * HF_PER_BRANCH + HF_T) * A.qcap + U.j] = h.t;
        A.hitf[(size_t)(U.b * HF_PER_BRANCH + HF_B1) * A.qcap + U.j] = h.b1;
        A.hitf[(size_t)(U.b * HF_PER_BRANCH + HF_B2) * A.qcap + U.j] = h.b2;
        A.hitp[(size_t)U.b * A.qcap + U.j] = h.prim;
        return;
    }
    const size_t C = (size_t)A.shcap;
    const float* F = A.shf;
    const int64_t j = U.j;
    const uint32_t g = A.shu[SU_PATH * C + j];
    const uint32_t mask = (A.shu[SU_META * C + j] >> 8) & 3u;
    const bool occluded = h.prim >= 0;
    if (MODE != MODE_REPLAY && A.hs) {   // ADJ_FWD: keep the visibility for the replay, by path
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (mask & (1u << b))
                A.hvis[((int64_t)b * A.hs_depth + depth_sh - 1) * A.hs_cap + g] = occluded ? 0 : 1;
    }
    if (occluded) return;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if (!(mask & (1u << b))) continue;
        const size_t bf = SF_SLOT + (size_t)b * SF_PER_SLOT;
#pragma unroll
        for (int c = 0; c < 3; ++c) A.lacc[(size_t)(b * 3 + c) * A.qcap + g] += F[(bf + c) * C + j];
        if (MODE == MODE_REPLAY) {
            const uint32_t r = A.shu[(SU_REC + b) * C + j];
            if (r == 0xffffffffu) continue;
#pragma unroll
            for (int k = 0; k < MAXC; ++k) A.rec[r].g[k] += F[(bf + 3 + k) * C + j];
        }
    }
}

// Cooperative tail of a traversal launch. Pairs the k-th idle lane with the k-th lane that has
// deferred subtrees (k < the smaller count): that lane pops its top entry and the idle lane walks
// the subtree as a helper of the ray's owner (a helper's own deferred entries can be handed on
// again; the owner stays the one the results go to). The helper copies the ray and its current
// closest distance, which only bounds the search: a hit it finds is compared with the owner's when
// it is merged, under the same rule (nearer, ties to the smaller primitive id), so the owner ends
// with the hit its own walk would have found.
__device__ __forceinline__ void delegate_subtrees(unsigned idle, unsigned donors, unsigned lane, bool& busy,
                                                  bool& helper, int& root, Unit& U, TravRay& R, int* stack) {
    const int m = min(__popc(idle), __popc(donors));
    const unsigned lt = (1u << lane) - 1u;
    const bool take = ((idle >> lane) & 1u) && __popc(idle & lt) < m;
    const bool give = ((donors >> lane) & 1u) && __popc(donors & lt) < m;
    int entry = 0;
    if (give) entry = stack[--R.sp];
    int src = (int)lane;
    if (take) {
        unsigned d = donors;
        for (int i = __popc(idle & lt); i > 0; --i) d &= d - 1u;
        src = __ffs(d) - 1;
    }
    entry = __shfl_sync(FULL, entry, src);
    const float o0 = __shfl_sync(FULL, R.o.x, src), o1 = __shfl_sync(FULL, R.o.y, src), o2 = __shfl_sync(FULL, R.o.z, src);
    const float d0 = __shfl_sync(FULL, R.d.x, src), d1 = __shfl_sync(FULL, R.d.y, src), d2 = __shfl_sync(FULL, R.d.z, src);
    const float ix = __shfl_sync(FULL, R.ix, src), iy = __shfl_sync(FULL, R.iy, src), iz = __shfl_sync(FULL, R.iz, src);
    const float ox = __shfl_sync(FULL, R.ox, src), oy = __shfl_sync(FULL, R.oy, src), oz = __shfl_sync(FULL, R.oz, src);
    const float t = __shfl_sync(FULL, R.t, src);
    const int any = __shfl_sync(FULL, R.any ? 1 : 0, src);
    const int q = __shfl_sync(FULL, U.q, src);
    const int own = __shfl_sync(FULL, helper ? root : (int)lane, src);
    if (take) {
        R.o = mk(o0, o1, o2);
        R.d = mk(d0, d1, d2);
        R.ix = ix; R.iy = iy; R.iz = iz;
        R.ox = ox; R.oy = oy; R.oz = oz;
        R.sx = ix < 0.0f ? 1 : 0;
        R.sy = iy < 0.0f ? 1 : 0;
        R.sz = iz < 0.0f ? 1 : 0;
        R.t = t;
        R.b1 = R.b2 = 0.0f;
        R.best = 0x7fffffff;
        R.node = entry;
        R.sp = 0;
        R.any = any != 0;
        R.hit_any = false;
        R.complete = true;
        U.q = q;
        root = own;
        helper = true;
        busy = true;
    }
}

// Helpers whose subtree walk ended (lanes in `fin`) hand their result to their owner, one at a
// time in lane order: a nearer hit (ties: smaller primitive id), an any-hit (which ends the
// owner's own walk), an overflowed stack.
__device__ __forceinline__ void merge_helpers(unsigned fin, unsigned lane, bool busy, int root, TravRay& R) {
    while (fin) {
        const int src = __ffs(fin) - 1;
        fin &= fin - 1u;
        const float ht = __shfl_sync(FULL, R.t, src), hb1 = __shfl_sync(FULL, R.b1, src),
                    hb2 = __shfl_sync(FULL, R.b2, src);
        const int hbest = __shfl_sync(FULL, R.best, src);
        const int hflags = __shfl_sync(FULL, (R.hit_any ? 1 : 0) | (R.complete ? 0 : 2), src);
        const int hroot = __shfl_sync(FULL, root, src);
        if ((int)lane == hroot) {
            if (hbest != 0x7fffffff && (ht < R.t || (ht == R.t && hbest < R.best))) {
                R.t = ht;
                R.b1 = hb1;
                R.b2 = hb2;
                R.best = hbest;
            }
            if (hflags & 1) {
                R.hit_any = true;
                if (busy) {
                    R.node = NODE_EMPTY;
                    R.sp = 0;
                }
            }
            if (hflags & 2) R.complete = false;
        }
    }
}

template <int NB, int MODE, bool STATS>
__global__ void __launch_bounds__(256, 3) k_trace(PassArgs A, int depth_ext, int depth_sh) {
    const Node* s_nodes;
    const int n_staged = stage_nodes(A, s_nodes);
    const int64_t n_ext = depth_ext == 1 ? A.n_paths : min((int64_t)A.cnt[CNT_Q + depth_ext], A.qcap);
    const int64_t n_sh = depth_sh > 0 ? min((int64_t)A.cnt[CNT_S + depth_sh], A.shcap) : 0;
    const int64_t n_eu = NB == 2 ? 2 * n_ext : n_ext;
    const int64_t n = n_eu + n_sh;
    uint32_t* fetch = A.cnt + CNT_FETCH + depth_ext;   // zeroed with the pass counters
    const unsigned lane = threadIdx.x & 31u;
    int stack[TRAV_STACK];
    TravRay R;
    Unit U{0, 0, 0};
    TravCount tc;
    bool busy = false, more = n > 0;
    // cooperative tail: once the units are all taken, idle lanes take deferred subtrees of the
    // warp's remaining walks (helper lanes), and an owner whose own walk ended waits for its
    // helpers before it finishes its unit
    bool helper = false, waiting = false;
    int root = 0;   // helper: lane of the walk's owner
    const Node* t_nodes = nullptr;     // the walk's tree (problem U.q)
    const TriGeo* t_tris = nullptr;
    const int refill = min(max(A.refill, 1), 32);
    while (true) {
        const unsigned idle = __ballot_sync(FULL, !busy && !waiting);
        if (more && __popc(idle) >= refill) {
            const unsigned cnt = (unsigned)__popc(idle);
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(fetch, cnt);
            base = __shfl_sync(FULL, base, 0);
            if ((int64_t)base + cnt >= n) more = false;
            if (!busy) {
                const int64_t u = (int64_t)base + __popc(idle & ((1u << lane) - 1u));
                if (u < n) busy = unit_setup<NB>(A, depth_ext, u, n_eu, U, R);
                if (busy) {
                    t_nodes = A.probs[U.q].nodes;
                    t_tris = A.probs[U.q].tris;
                }
            }
        }
        if (!more) {
            // lanes still free after this iteration's fetch (which may have taken the last units)
            const unsigned free_now = __ballot_sync(FULL, !busy && !waiting);
            const unsigned donors = __ballot_sync(FULL, busy && R.sp > 0);
            if (free_now && donors) {
                const bool was = busy;
                delegate_subtrees(free_now, donors, lane, busy, helper, root, U, R, stack);
                if (busy && !was) {
                    t_nodes = A.probs[U.q].nodes;
                    t_tris = A.probs[U.q].tris;
                }
            }
        }
        if (!__any_sync(FULL, busy || waiting)) {
            if (!more) break;
            continue;
        }
        bool fin = false;
        if (busy) fin = trav_step<STATS>(t_nodes, t_tris, s_nodes, U.q == A.smem_prob ? n_staged : 0, R, stack, tc);
        if (!__any_sync(FULL, helper || waiting)) {
            if (fin) {
                unit_finish<NB, MODE, STATS>(A, depth_sh, U, R, tc);
                busy = false;
            }
            continue;
        }
        merge_helpers(__ballot_sync(FULL, fin && helper), lane, busy, root, R);
        if (fin) {
            busy = false;
            if (helper) helper = false;
            else waiting = true;
        }
        // an owner's group: itself and the helpers still walking for it
        const unsigned grp = __match_any_sync(FULL, (busy && helper) ? root : (int)lane);
        if (waiting && __popc(grp) == 1) {
            unit_finish<NB, MODE, STATS>(A, depth_sh, U, R, tc);
            waiting = false;
        }
    }
    if (STATS) {
        const int cls = (NB == 1 ? KC_TRACE1_PRIMAL : KC_TRACE2_PRIMAL) + (MODE == MODE_REPLAY ? 1 : 0);
        flush_counts(A, cls, tc);
    }
}

// ---------------------------------------------------------------------------------
// resolve radiance per path into images (mean over samples)
// ---------------------------------------------------------------------------------
template <int NB>
__global__ void k_resolve(PassArgs A, float* img0, float* img1, int accumulate) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < A.n_paths; g += stride) {
        int q = A.inl_prob;
        int64_t local = g;
        if (q < 0) {
            const int e = find_entry(A.path_off, A.n_entries, g);
            q = A.entry_prob[e];
            local = g - A.path_off[e];
        }
        const ProblemDev& P = A.probs[q];
        if (local >= P.n_pix) continue;
        const int spp_here = (int)((A.inl_prob >= 0 ? A.n_paths : 0) / P.n_pix);
        const int nsm = A.inl_prob >= 0 ? spp_here : (A.fd_kind ? P.spp_fd : P.spp_prop);
        const int spp_total = A.spp_override > 0 ? A.spp_override : nsm;
        const float inv = 1.0f / (float)spp_total;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            float* img = A.inl_prob >= 0 ? (b == 0 ? img0 : img1) : (A.fd_kind ? (b ? P.imgB : P.imgA) : P.img);
            if (!img) continue;
            img += (int64_t)path_pixel(P, (uint32_t)local) * 3;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float acc = 0.0f;
                for (int s = 0; s < nsm; ++s) acc += A.lacc[(size_t)(b * 3 + c) * A.qcap + g + (int64_t)s * P.n_pix];
                img[c] = (accumulate ? img[c] : 0.0f) + acc * inv;
            }
        }
    }
}

// per-sample radiance out[(s*n_pix + p)*3 + c] of a single-problem pass
__global__ void k_samples_out(PassArgs A, float* out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const ProblemDev& P = A.probs[A.inl_prob];
    const int64_t base = (int64_t)A.sample_base * P.n_pix;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < A.n_paths; g += stride) {
        const int64_t s = g / P.n_pix, local = g - s * P.n_pix;
        const int64_t o = base + s * P.n_pix + path_pixel(P, (uint32_t)local);
        for (int c = 0; c < 3; ++c) out[o * 3 + c] = A.lacc[(size_t)c * A.qcap + g];
    }
}

// ---------------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------------
// persistent grid: resident blocks per SM from the occupancy calculator (capped by per_sm)
template <class K>
static int persistent_grid(K kernel, const LaunchShape& L, size_t smem) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, L.block, smem) != cudaSuccess || occ < 1) occ = 1;
    if (L.per_sm > 0 && occ > L.per_sm) occ = L.per_sm;
    return occ * L.sms;
}

template <int NB, int MODE>
struct PassLauncher {
    int g_trace = 0, g_shade = 0;
    LaunchShape last{-1, -1, -1, -1};

    void grids(const LaunchShape& L, size_t smem) {
        if (last.block == L.block && last.per_sm == L.per_sm && last.smem_nodes == L.smem_nodes && last.sms == L.sms)
            return;
        g_trace = persistent_grid(k_trace<NB, MODE, false>, L, smem);
        g_shade = persistent_grid(k_shade<NB, MODE>, L, 0);
        last = L;
    }

    void trace(const PassArgs& B, int de, int ds, const LaunchShape& L, size_t smem, cudaStream_t st) {
        const int cls = (NB == 1 ? KC_TRACE1_PRIMAL : KC_TRACE2_PRIMAL) + (MODE == MODE_REPLAY ? 1 : 0);
        if (B.stats) k_trace<NB, MODE, true><<<g_trace, L.block, smem, st>>>(B, de, ds);
        else MER_TIMED(cls, st, k_trace<NB, MODE, false><<<g_trace, L.block, smem, st>>>(B, de, ds));
    }

    void shade(const PassArgs& B, int depth, const LaunchShape& L, cudaStream_t st) {
        const int cls = (NB == 1 ? KC_SHADE1_PRIMAL : KC_SHADE2_PRIMAL) + (MODE == MODE_REPLAY ? 1 : 0);
        if (B.stats) k_shade<NB, MODE><<<g_shade, L.block, 0, st>>>(B, depth);
        else MER_TIMED(cls, st, k_shade<NB, MODE><<<g_shade, L.block, 0, st>>>(B, depth));
    }

    // trace(1) shade(1) trace(2, 1) shade(2) ... shade(D) trace(-, D): 2D + 1 launches; a replay
    // with a hit store: shade(1) ... shade(D)
    int run(const PassArgs& A, int max_depth, const LaunchShape& L, cudaStream_t st) {
        const size_t smem = (size_t)L.smem_nodes * sizeof(Node);
        PassArgs B = A;
        B.smem_nodes = L.smem_nodes;
        B.refill = L.refill;
        grids(L, smem);
        if (MODE == MODE_REPLAY && B.hs) {
            for (int depth = 1; depth <= max_depth; ++depth) shade(B, depth, L, st);
            return max_depth;
        }
        for (int depth = 1; depth <= max_depth; ++depth) {
            trace(B, depth, depth - 1, L, smem, st);
            shade(B, depth, L, st);
        }
        trace(B, max_depth + 1, max_depth, L, smem, st);
        return 2 * max_depth + 1;
    }
};

// enqueues one full pass; returns the number of kernel launches
int run_pass(const PassArgs& A, int nb, int mode, int max_depth, const LaunchShape& L, cudaStream_t st) {
    static PassLauncher<1, MODE_PRIMAL> p1;
    static PassLauncher<1, MODE_REPLAY> r1;
    static PassLauncher<2, MODE_PRIMAL> p2;
    static PassLauncher<2, MODE_REPLAY> r2;
    if (nb == 1) return mode == MODE_REPLAY ? r1.run(A, max_depth, L, st) : p1.run(A, max_depth, L, st);
    return mode == MODE_REPLAY ? r2.run(A, max_depth, L, st) : p2.run(A, max_depth, L, st);
}

int run_resolve(const PassArgs& A, int nb, float* img0, float* img1, int accumulate, int grid, cudaStream_t st) {
    if (nb == 1) MER_TIMED(KC_RESOLVE, st, k_resolve<1><<<grid, 256, 0, st>>>(A, img0, img1, accumulate));
    else MER_TIMED(KC_RESOLVE, st, k_resolve<2><<<grid, 256, 0, st>>>(A, img0, img1, accumulate));
    return 1;
}

int run_samples_out(const PassArgs& A, float* out, int grid, cudaStream_t st) {
    k_samples_out<<<grid, 256, 0, st>>>(A, out);
    return 1;
}

cudaError_t set_trace_smem_limits(int max_nodes) {
    const int bytes = max_nodes * (int)sizeof(Node);
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const void* fns[] = {(const void*)k_trace<1, MODE_PRIMAL, false>, (const void*)k_trace<1, MODE_REPLAY, false>,
                         (const void*)k_trace<2, MODE_PRIMAL, false>, (const void*)k_trace<2, MODE_REPLAY, false>,
                         (const void*)k_trace<1, MODE_PRIMAL, true>,  (const void*)k_trace<1, MODE_REPLAY, true>,
                         (const void*)k_trace<2, MODE_PRIMAL, true>,  (const void*)k_trace<2, MODE_REPLAY, true>};
    for (const void* f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, at, bytes);
        if (e) return e;
    }
    return cudaSuccess;
}

}  // namespace mer

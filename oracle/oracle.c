/*
 * FP64 CPU oracle for meta-estimated inverse path tracing.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests, the smoke check and the CPU-baseline leg of
 * the benchmark load this file's library. The product path never does; it shares no
 * code, header, table or helper with this file.
 *
 * It is deliberately plain: single-threaded, brute-force intersection over every
 * primitive, one path at a time, double precision throughout. It follows:
 *   - Eq. F_def / est_def (Sec. 3): a gradient sample is f/p along one sampled path;
 *   - Eq. est_triv (Sec. 3): the finite-difference sample is the same random numbers
 *     evaluated at two parameter vectors (two separate calls of these functions);
 *   - Sec. 6 setup: gradients by Path Replay Backpropagation (forward pass for the
 *     path's total radiance, then a replay from the same random numbers), with the
 *     sampling densities and MIS weights held constant ("detached").
 * The renderer's conventions the paper leaves to Mitsuba (BSDF model, light selection,
 * MIS heuristic, depth convention, texture filter, ray offsets) are fixed in the
 * project's design notes and restated where they are used below.
 *
 * Parity notes: `trace` in replay mode (bookkeeping with subtraction and division)
 * and `trace_stored` (explicit products over stored vertices, no division) are
 * independent derivations of the same gradient and pin each other.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC 2011). Multipliers and Weyl key increments are the     */
/* published constants; each round multiplies words 0 and 2, xors the high     */
/* halves with words 1/3 and the round key, and permutes.                       */
/* ------------------------------------------------------------------------- */
void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t pa = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t pb = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t a_hi = (uint32_t)(pa >> 32), a_lo = (uint32_t)pa;
        uint32_t b_hi = (uint32_t)(pb >> 32), b_lo = (uint32_t)pb;
        uint32_t y0 = b_hi ^ x1 ^ k0;
        uint32_t y1 = b_lo;
        uint32_t y2 = a_hi ^ x3 ^ k1;
        uint32_t y3 = a_lo;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Stream ids of the counter's fourth word. */
enum { ST_PROP_PRIMAL = 0, ST_PROP_ADJ = 1, ST_FD_PRIMAL = 2, ST_FD_ADJ = 3, ST_TARGET = 4, ST_EVAL = 5 };

/* Four uniforms in [0,1): counter = (pixel, sample, iteration, stream<<16 | vertex<<4 | block),
 * key = (seed, key_id). u = (x >> 8) * 2^-24 is exact in both float and double. */
typedef struct { uint32_t key[2]; uint32_t pixel, sample, iter, stream; } rng_ctx;

static void draw4(const rng_ctx* r, uint32_t vertex, uint32_t block, double u[4], uint32_t raw[4])
{
    uint32_t c[4] = { r->pixel, r->sample, r->iter, (r->stream << 16) | (vertex << 4) | block };
    uint32_t o[4];
    orc_philox(c, r->key, o);
    for (int i = 0; i < 4; ++i) {
        u[i] = (double)(o[i] >> 8) * (1.0 / 16777216.0);
        if (raw) raw[i] = o[i];
    }
}

/* ------------------------------------------------------------------------- */
/* small vector algebra                                                        */
/* ------------------------------------------------------------------------- */
typedef struct { double x, y, z; } v3;
static v3 V(double x, double y, double z) { v3 r = { x, y, z }; return r; }
static v3 vadd(v3 a, v3 b) { return V(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 vsub(v3 a, v3 b) { return V(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 vmul(v3 a, double s) { return V(a.x * s, a.y * s, a.z * s); }
static double vdot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 vcross(v3 a, v3 b) { return V(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static double vlen(v3 a) { return sqrt(vdot(a, a)); }
static v3 vnorm(v3 a) { return vmul(a, 1.0 / vlen(a)); }
static v3 vload(const float* p) { return V(p[0], p[1], p[2]); }

/* ------------------------------------------------------------------------- */
/* scene description (plain arrays; float inputs are widened to double on use)  */
/* ------------------------------------------------------------------------- */
typedef struct orc_scene {
    int32_t n_verts, n_tris;
    const float* pos;          /* n_verts*3 */
    const float* uv;           /* n_verts*2 */
    const int32_t* tris;       /* n_tris*3 */
    const int32_t* tri_mat;    /* n_tris */
    const int32_t* tri_light;  /* n_tris, -1 = not emissive */
    int32_t n_spheres;
    const float* spheres;      /* 8 per sphere: c.xyz, r, u0, u1, v0, v1 */
    const int32_t* sph_mat;
    int32_t n_mats;
    const int32_t* mat_type;   /* 0 Lambert, 1 principled */
    const int32_t* mat_textured;
    const float* mat_const;    /* 5 per material */
    int32_t n_quads;
    const float* quads;        /* 12 per quad light: p0, e1, e2, Le */
    int32_t has_env;
    float env[3];
    float eye[3], target[3], up[3];
    float fov_deg;
    int32_t width, height;
    int32_t tex_c, tex_h, tex_w;
    int32_t max_depth;
    uint32_t seed, key_id;
} orc_scene;

/* ------------------------------------------------------------------------- */
/* intersection: brute force over all primitives, ascending id, strict '<' on t */
/* so equal distances keep the smaller primitive id                             */
/* ------------------------------------------------------------------------- */
typedef struct { double t, b1, b2; int prim; } hit_t;

static int tri_hit(const orc_scene* s, int i, v3 o, v3 d, double* t, double* b1, double* b2)
{
    const int32_t* T = s->tris + 3 * i;
    v3 p0 = vload(s->pos + 3 * T[0]), p1 = vload(s->pos + 3 * T[1]), p2 = vload(s->pos + 3 * T[2]);
    v3 e1 = vsub(p1, p0), e2 = vsub(p2, p0);
    /* Moller-Trumbore */
    v3 pv = vcross(d, e2);
    double det = vdot(e1, pv);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    v3 tv = vsub(o, p0);
    double u = vdot(tv, pv) * inv;
    if (u < 0.0 || u > 1.0) return 0;
    v3 qv = vcross(tv, e1);
    double v = vdot(d, qv) * inv;
    if (v < 0.0 || u + v > 1.0) return 0;
    *t = vdot(e2, qv) * inv;
    *b1 = u; *b2 = v;
    return 1;
}

static int sph_hit(const orc_scene* s, int i, v3 o, v3 d, double* t)
{
    const float* S = s->spheres + 8 * i;
    v3 c = vload(S);
    double r = S[3];
    v3 oc = vsub(o, c);
    double b = vdot(oc, d);                 /* d is unit length */
    double cc = vdot(oc, oc) - r * r;
    double disc = b * b - cc;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    double t0 = -b - sq, t1 = -b + sq;
    if (t0 > 0.0) { *t = t0; return 1; }
    if (t1 > 0.0) { *t = t1; return 1; }
    return 0;
}

static int intersect(const orc_scene* s, v3 o, v3 d, hit_t* h)
{
    h->t = INFINITY; h->prim = -1; h->b1 = h->b2 = 0.0;
    for (int i = 0; i < s->n_tris; ++i) {
        double t, b1, b2;
        if (tri_hit(s, i, o, d, &t, &b1, &b2) && t > 0.0 && t < h->t) {
            h->t = t; h->prim = i; h->b1 = b1; h->b2 = b2;
        }
    }
    for (int i = 0; i < s->n_spheres; ++i) {
        double t;
        if (sph_hit(s, i, o, d, &t) && t < h->t) {
            h->t = t; h->prim = s->n_tris + i; h->b1 = h->b2 = 0.0;
        }
    }
    return h->prim >= 0;
}

static int occluded(const orc_scene* s, v3 o, v3 d, double tmax)
{
    for (int i = 0; i < s->n_tris; ++i) {
        double t, b1, b2;
        if (tri_hit(s, i, o, d, &t, &b1, &b2) && t > 0.0 && t < tmax) return 1;
    }
    for (int i = 0; i < s->n_spheres; ++i) {
        double t;
        if (sph_hit(s, i, o, d, &t) && t < tmax) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* surface interaction                                                          */
/* ------------------------------------------------------------------------- */
typedef struct {
    v3 p, n;          /* position, geometric normal (unit) */
    double u, v;      /* texture coordinates */
    int mat, light;
} surf_t;

static void surface(const orc_scene* s, v3 o, v3 d, const hit_t* h, surf_t* si)
{
    si->p = vadd(o, vmul(d, h->t));
    if (h->prim < s->n_tris) {
        const int32_t* T = s->tris + 3 * h->prim;
        v3 p0 = vload(s->pos + 3 * T[0]), p1 = vload(s->pos + 3 * T[1]), p2 = vload(s->pos + 3 * T[2]);
        si->n = vnorm(vcross(vsub(p1, p0), vsub(p2, p0)));
        double w = 1.0 - h->b1 - h->b2;
        const float *a = s->uv + 2 * T[0], *b = s->uv + 2 * T[1], *c = s->uv + 2 * T[2];
        si->u = w * a[0] + h->b1 * b[0] + h->b2 * c[0];
        si->v = w * a[1] + h->b1 * b[1] + h->b2 * c[1];
        si->mat = s->tri_mat[h->prim];
        si->light = s->tri_light[h->prim];
    } else {
        int i = h->prim - s->n_tris;
        const float* S = s->spheres + 8 * i;
        si->n = vmul(vsub(si->p, vload(S)), 1.0 / S[3]);
        double uu = atan2(si->n.y, si->n.x) / (2.0 * PI);
        if (uu < 0.0) uu += 1.0;
        double zz = si->n.z < -1.0 ? -1.0 : (si->n.z > 1.0 ? 1.0 : si->n.z);
        double vv = acos(zz) / PI;
        si->u = S[4] + uu * (S[5] - S[4]);
        si->v = S[6] + vv * (S[7] - S[6]);
        si->mat = s->sph_mat[i];
        si->light = -1;
    }
}

/* ------------------------------------------------------------------------- */
/* texture: bilinear, clamp-to-edge, texel centres at (x+1/2)/W                */
/* ------------------------------------------------------------------------- */
typedef struct { int x0, y0; double fx, fy; } foot_t;

static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

static void tex_footprint(const orc_scene* s, double u, double v, foot_t* f)
{
    u = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
    v = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
    double x = u * s->tex_w - 0.5, y = v * s->tex_h - 0.5;
    double fx0 = floor(x), fy0 = floor(y);
    f->x0 = (int)fx0; f->y0 = (int)fy0;
    f->fx = x - fx0; f->fy = y - fy0;
}

/* the four texel indices (flattened y*W+x) and bilinear weights of a footprint */
static void tex_taps(const orc_scene* s, const foot_t* f, int idx[4], double w[4])
{
    int W = s->tex_w, H = s->tex_h;
    int xa = clampi(f->x0, 0, W - 1), xb = clampi(f->x0 + 1, 0, W - 1);
    int ya = clampi(f->y0, 0, H - 1), yb = clampi(f->y0 + 1, 0, H - 1);
    idx[0] = ya * W + xa; w[0] = (1.0 - f->fx) * (1.0 - f->fy);
    idx[1] = ya * W + xb; w[1] = f->fx * (1.0 - f->fy);
    idx[2] = yb * W + xa; w[2] = (1.0 - f->fx) * f->fy;
    idx[3] = yb * W + xb; w[3] = f->fx * f->fy;
}

/* ------------------------------------------------------------------------- */
/* materials                                                                    */
/*  Lambert:    f = rho / pi                                                    */
/*  principled: f = (1-m) bc / pi + D F G1(wo) G1(wi) / (4 cos_o cos_i)         */
/*              GGX D with alpha = rough^2, Schlick F with F0 = mix(0.04,bc,m)  */
/*              separable Smith G1; specular lobe picked with P = (1+m)/2       */
/* ------------------------------------------------------------------------- */
typedef struct { int type, textured; double th[5]; foot_t foot; } mat_t;

static void load_material(const orc_scene* s, const double* tex, const surf_t* si, mat_t* m)
{
    m->type = s->mat_type[si->mat];
    m->textured = s->mat_textured[si->mat];
    if (!m->textured) {
        for (int j = 0; j < 5; ++j) m->th[j] = s->mat_const[5 * si->mat + j];
        return;
    }
    tex_footprint(s, si->u, si->v, &m->foot);
    int idx[4]; double w[4];
    tex_taps(s, &m->foot, idx, w);
    int C = s->tex_c;
    for (int j = 0; j < 5; ++j) m->th[j] = 0.0;
    for (int j = 0; j < C; ++j) {
        double acc = 0.0;
        for (int k = 0; k < 4; ++k) acc += w[k] * tex[(size_t)idx[k] * C + j];
        m->th[j] = acc;
    }
}

/* orthonormal basis around a unit normal (Duff et al. 2017, "Building an Orthonormal
 * Basis, Revisited", JCGT 6(1)) */
static void onb(v3 n, v3* t, v3* b)
{
    double sg = copysign(1.0, n.z);
    double a = -1.0 / (sg + n.z);
    double bb = n.x * n.y * a;
    *t = V(1.0 + sg * n.x * n.x * a, sg * bb, -sg * n.x);
    *b = V(bb, sg + n.y * n.y * a, -n.y);
}

static v3 to_world(v3 n, double x, double y, double z)
{
    v3 t, b;
    onb(n, &t, &b);
    return vadd(vadd(vmul(t, x), vmul(b, y)), vmul(n, z));
}

static v3 sample_cosine(v3 n, double u1, double u2)
{
    double r = sqrt(u1), ph = 2.0 * PI * u2;
    double z = 1.0 - u1;
    return to_world(n, r * cos(ph), r * sin(ph), sqrt(z > 0.0 ? z : 0.0));
}

static double ggx_D(double a2, double ch)
{
    double k = ch * ch * (a2 - 1.0) + 1.0;
    return a2 / (PI * k * k);
}

static double smith_G1(double a2, double c)
{
    return 2.0 * c / (c + sqrt(a2 + (1.0 - a2) * c * c));
}

/* value f[c], and (if df) derivatives df[j][c] = d f_c / d theta_j, for unit n facing wo */
static void bsdf_eval(const mat_t* m, v3 n, v3 wo, v3 wi, double f[3], double df[5][3])
{
    for (int c = 0; c < 3; ++c) f[c] = 0.0;
    if (df) memset(df, 0, sizeof(double) * 15);
    double co = vdot(n, wo), ci = vdot(n, wi);
    if (co <= 0.0 || ci <= 0.0) return;
    if (m->type == 0) {
        for (int c = 0; c < 3; ++c) f[c] = m->th[c] / PI;
        if (df) for (int c = 0; c < 3; ++c) df[c][c] = 1.0 / PI;
        return;
    }
    double metal = m->th[3], r = m->th[4];
    double a = r * r, a2 = a * a;
    v3 h = vnorm(vadd(wo, wi));
    double ch = vdot(n, h), vh = vdot(wi, h);
    double D = ggx_D(a2, ch);
    double Go = smith_G1(a2, co), Gi = smith_G1(a2, ci);
    double S = D * Go * Gi / (4.0 * co * ci);
    double Fw = pow(1.0 - vh, 5.0);
    for (int c = 0; c < 3; ++c) {
        double F0 = 0.04 * (1.0 - metal) + m->th[c] * metal;
        double F = F0 + (1.0 - F0) * Fw;
        f[c] = (1.0 - metal) * m->th[c] / PI + S * F;
    }
    if (!df) return;
    /* d/d base colour: diffuse term and Schlick F0 */
    for (int c = 0; c < 3; ++c) df[c][c] = (1.0 - metal) / PI + S * (1.0 - Fw) * metal;
    /* d/d metal */
    for (int c = 0; c < 3; ++c) df[3][c] = -m->th[c] / PI + S * (1.0 - Fw) * (m->th[c] - 0.04);
    /* d/d rough through alpha = r^2 in D, G1(wo), G1(wi) */
    double k = ch * ch * (a2 - 1.0) + 1.0;
    double dD = (2.0 * a / (PI * k * k)) * (1.0 - 2.0 * a2 * ch * ch / k);
    double so = sqrt(a2 + (1.0 - a2) * co * co), si_ = sqrt(a2 + (1.0 - a2) * ci * ci);
    double dGo = -2.0 * co * (a * (1.0 - co * co) / so) / ((co + so) * (co + so));
    double dGi = -2.0 * ci * (a * (1.0 - ci * ci) / si_) / ((ci + si_) * (ci + si_));
    double dS_da = (dD * Go * Gi + D * (dGo * Gi + Go * dGi)) / (4.0 * co * ci);
    double dS_dr = dS_da * 2.0 * r;
    for (int c = 0; c < 3; ++c) {
        double F0 = 0.04 * (1.0 - metal) + m->th[c] * metal;
        double F = F0 + (1.0 - F0) * Fw;
        df[4][c] = dS_dr * F;
    }
}

static double bsdf_pdf(const mat_t* m, v3 n, v3 wo, v3 wi)
{
    double co = vdot(n, wo), ci = vdot(n, wi);
    if (co <= 0.0 || ci <= 0.0) return 0.0;
    if (m->type == 0) return ci / PI;
    double metal = m->th[3], r = m->th[4];
    double a = r * r, a2 = a * a;
    double ps = 0.5 * (1.0 + metal);
    v3 h = vnorm(vadd(wo, wi));
    double ch = vdot(n, h), vh = vdot(wo, h);
    double pspec = vh > 0.0 ? ggx_D(a2, ch) * ch / (4.0 * vh) : 0.0;
    return ps * pspec + (1.0 - ps) * ci / PI;
}

/* returns 1 and the direction if the sample lies above the surface */
static int bsdf_sample(const mat_t* m, v3 n, v3 wo, double ul, double u1, double u2, v3* wi)
{
    if (m->type == 1 && ul < 0.5 * (1.0 + m->th[3])) {
        double a = m->th[4] * m->th[4], a2 = a * a;
        double t2 = a2 * u1 / (1.0 - u1);
        double ct = 1.0 / sqrt(1.0 + t2);
        double st = sqrt(1.0 - ct * ct > 0.0 ? 1.0 - ct * ct : 0.0);
        double ph = 2.0 * PI * u2;
        v3 h = to_world(n, st * cos(ph), st * sin(ph), ct);
        double oh = vdot(wo, h);
        if (oh <= 0.0) return 0;
        *wi = vsub(vmul(h, 2.0 * oh), wo);
    } else {
        *wi = sample_cosine(n, u1, u2);
    }
    return vdot(n, *wi) > 0.0;
}

static double mis2(double a, double b) { return a * a / (a * a + b * b); }

/* ------------------------------------------------------------------------- */
/* camera: pinhole, box-filtered jitter inside the pixel, row 0 at the top      */
/* ------------------------------------------------------------------------- */
static void camera_ray(const orc_scene* s, int px, int py, double j0, double j1, v3* o, v3* d)
{
    v3 eye = vload(s->eye), tg = vload(s->target), up = vload(s->up);
    v3 f = vnorm(vsub(tg, eye));
    v3 r = vnorm(vcross(f, up));
    v3 u = vcross(r, f);
    double th = tan(0.5 * s->fov_deg * PI / 180.0);
    double asp = (double)s->width / (double)s->height;
    double sx = (2.0 * (px + j0) / s->width - 1.0) * th * asp;
    double sy = (1.0 - 2.0 * (py + j1) / s->height) * th;
    *o = eye;
    *d = vnorm(vadd(f, vadd(vmul(r, sx), vmul(u, sy))));
}

static v3 offset_point(v3 p, v3 nf)
{
    double m = fabs(p.x);
    if (fabs(p.y) > m) m = fabs(p.y);
    if (fabs(p.z) > m) m = fabs(p.z);
    double e = 1e-4 * (m > 1.0 ? m : 1.0);
    return vadd(p, vmul(nf, e));
}

/* one light sample for next-event estimation: uniform light choice among
 * {quads..., env}; quads sampled uniformly by area, env by a cosine lobe around nf */
typedef struct { int ok; v3 wi; double pdf, tmax, Le[3]; } nee_t;

static void sample_light(const orc_scene* s, v3 po, v3 nf, const double u[4], const uint32_t raw[4], nee_t* L)
{
    int nL = s->n_quads + (s->has_env ? 1 : 0);
    L->ok = 0;
    if (nL == 0) return;
    int l = (int)(((uint64_t)(raw[0] >> 8) * (uint64_t)nL) >> 24);
    if (l < s->n_quads) {
        const float* Q = s->quads + 12 * l;
        v3 p0 = vload(Q), e1 = vload(Q + 3), e2 = vload(Q + 6);
        v3 y = vadd(p0, vadd(vmul(e1, u[1]), vmul(e2, u[2])));
        v3 w = vsub(y, po);
        double d2 = vdot(w, w), dist = sqrt(d2);
        v3 wi = vmul(w, 1.0 / dist);
        v3 nc = vcross(e1, e2);
        double area = vlen(nc);
        v3 nl = vmul(nc, 1.0 / area);
        double cl = -vdot(wi, nl);
        if (cl <= 0.0 || vdot(wi, nf) <= 0.0) return;
        L->ok = 1; L->wi = wi;
        L->pdf = d2 / (area * cl * nL);
        L->tmax = dist * (1.0 - 1e-4);
        for (int c = 0; c < 3; ++c) L->Le[c] = Q[9 + c];
    } else {
        v3 wi = sample_cosine(nf, u[1], u[2]);
        double cs = vdot(wi, nf);
        if (cs <= 0.0) return;
        L->ok = 1; L->wi = wi;
        L->pdf = cs / (PI * nL);
        L->tmax = INFINITY;
        for (int c = 0; c < 3; ++c) L->Le[c] = s->env[c];
    }
}

/* solid-angle density with which NEE would have picked the quad light hit at distance t */
static double quad_light_pdf(const orc_scene* s, int l, v3 d, double t)
{
    int nL = s->n_quads + (s->has_env ? 1 : 0);
    const float* Q = s->quads + 12 * l;
    v3 nc = vcross(vload(Q + 3), vload(Q + 6));
    double area = vlen(nc);
    double cl = -vdot(d, vmul(nc, 1.0 / area));
    return t * t / (area * cl * nL);
}

static int quad_front(const orc_scene* s, int l, v3 d)
{
    const float* Q = s->quads + 12 * l;
    v3 nc = vcross(vload(Q + 3), vload(Q + 6));
    return vdot(d, nc) < 0.0;
}

/* scatter g[j] (derivative w.r.t. the fetched channel j) to the bilinear taps */
static void splat(const orc_scene* s, const mat_t* m, const double g[5], double* grad)
{
    int idx[4]; double w[4];
    tex_taps(s, &m->foot, idx, w);
    int C = s->tex_c;
    for (int k = 0; k < 4; ++k)
        for (int j = 0; j < C; ++j) grad[(size_t)idx[k] * C + j] += w[k] * g[j];
}

/* ------------------------------------------------------------------------- */
/* one path. Directions, lobe choices, pdfs and MIS weights come from the        */
/* parameters tex_s, the integrand (f and its derivative) from tex_e; tex_s =     */
/* tex_e is the ordinary estimator, tex_s = pi_i with tex_e = pi_{i-1} the FD     */
/* branch that shares the pi_i path and divides by its density (Eq. est_triv).    */
/* mode 0: radiance only. mode 1: PRB replay — needs the path's                   */
/* radiance Ltot from a mode-0 call with the same counters, the adjoint weight  */
/* adj[c] = dLoss/dL_c of this sample, and accumulates into grad.               */
/*                                                                               */
/* Depth convention: vertices 1..D along the path; the camera ray is segment 1. */
/* At vertex k: emission seen (MIS-weighted unless k = 1); if k < D, one NEE     */
/* sample and one BSDF sample. D = 1 shows emitters only, D = 2 direct light.    */
/* ------------------------------------------------------------------------- */
static void trace(const orc_scene* s, const double* tex_s, const double* tex_e, uint32_t pixel, uint32_t sample,
                  uint32_t iter, uint32_t stream, int mode, const double Ltot[3], const double adj[3], double* grad,
                  double Lout[3])
{
    rng_ctx R = { { s->seed, s->key_id }, pixel, sample, iter, stream };
    int nL = s->n_quads + (s->has_env ? 1 : 0);
    double u[4]; uint32_t raw[4];
    draw4(&R, 0, 0, u, raw);
    v3 o, d;
    camera_ray(s, (int)(pixel % (uint32_t)s->width), (int)(pixel / (uint32_t)s->width), u[0], u[1], &o, &d);
    double beta[3] = { 1, 1, 1 }, L[3] = { 0, 0, 0 };
    double pdf_b = 0.0, pdf_env = 0.0;
    for (int k = 1; k <= s->max_depth; ++k) {
        hit_t h;
        if (!intersect(s, o, d, &h)) {
            if (s->has_env) {
                double w = (k == 1) ? 1.0 : mis2(pdf_b, pdf_env);
                for (int c = 0; c < 3; ++c) L[c] += beta[c] * s->env[c] * w;
            }
            break;
        }
        surf_t si;
        surface(s, o, d, &h, &si);
        if (si.light >= 0 && quad_front(s, si.light, d)) {
            double w = (k == 1) ? 1.0 : mis2(pdf_b, quad_light_pdf(s, si.light, d, h.t));
            for (int c = 0; c < 3; ++c) L[c] += beta[c] * s->quads[12 * si.light + 9 + c] * w;
        }
        if (k == s->max_depth) break;
        v3 wo = vmul(d, -1.0);
        v3 nf = vdot(si.n, d) < 0.0 ? si.n : vmul(si.n, -1.0);
        v3 po = offset_point(si.p, nf);
        mat_t m, ms;   /* m: integrand (tex_e); ms: sampling and densities (tex_s) */
        load_material(s, tex_e, &si, &m);
        load_material(s, tex_s, &si, &ms);
        int want_grad = (mode == 1) && m.textured;
        double g[5] = { 0, 0, 0, 0, 0 };

        /* next-event estimation */
        draw4(&R, (uint32_t)k, 0, u, raw);
        nee_t nee;
        sample_light(s, po, nf, u, raw, &nee);
        if (nee.ok) {
            double f[3], df[5][3];
            bsdf_eval(&m, nf, wo, nee.wi, f, want_grad ? df : NULL);
            double pb = bsdf_pdf(&ms, nf, wo, nee.wi);
            double cs = vdot(nee.wi, nf);
            double wl = mis2(nee.pdf, pb);
            double q = cs * wl / nee.pdf;
            if ((f[0] != 0.0 || f[1] != 0.0 || f[2] != 0.0 || want_grad) && !occluded(s, po, nee.wi, nee.tmax)) {
                for (int c = 0; c < 3; ++c) L[c] += beta[c] * f[c] * nee.Le[c] * q;
                if (want_grad)
                    for (int j = 0; j < s->tex_c; ++j)
                        for (int c = 0; c < 3; ++c) g[j] += adj[c] * beta[c] * df[j][c] * nee.Le[c] * q;
            }
        }
        (void)nL;

        /* BSDF sample for the continuation */
        draw4(&R, (uint32_t)k, 1, u, raw);
        v3 wi;
        int ok = bsdf_sample(&ms, nf, wo, u[0], u[1], u[2], &wi);
        double f[3] = { 0, 0, 0 }, df[5][3], pb = 0.0;
        if (ok) {
            bsdf_eval(&m, nf, wo, wi, f, want_grad ? df : NULL);
            pb = bsdf_pdf(&ms, nf, wo, wi);
            if (pb <= 0.0) ok = 0;
        }
        if (want_grad) {
            if (ok) {
                /* radiance still to come along the sampled direction, divided by this vertex's f */
                for (int c = 0; c < 3; ++c) {
                    double Lafter = Ltot[c] - L[c];
                    if (f[c] == 0.0) continue;
                    for (int j = 0; j < s->tex_c; ++j) g[j] += adj[c] * Lafter * df[j][c] / f[c];
                }
            }
            splat(s, &m, g, grad);
        }
        if (!ok) break;
        double cs = vdot(wi, nf);
        for (int c = 0; c < 3; ++c) beta[c] *= f[c] * cs / pb;
        pdf_b = pb;
        pdf_env = s->has_env ? cs / (PI * nL) : 0.0;
        o = po;
        d = wi;
    }
    for (int c = 0; c < 3; ++c) Lout[c] = L[c];
}

/* ------------------------------------------------------------------------- */
/* the same gradient from a stored path: contributions are written as explicit  */
/* products of per-vertex factors and differentiated term by term (no division, */
/* no subtraction); O(D^2) per path                                             */
/* ------------------------------------------------------------------------- */
#define MAXV 64
typedef struct {
    int grad;                 /* textured material at this vertex */
    mat_t m;
    double E[3];              /* emission collected on arrival (MIS-weighted) */
    double N[3];              /* NEE contribution factor f(w_l) * Le * q  (0 if occluded) */
    double dN[5][3];          /* d f(w_l)/d theta * Le * q */
    double fb[3], cb;         /* continuation factor f(w_b) and cos/pdf */
    double dfb[5][3];
    int cont;                 /* a continuation was sampled */
} vtx_t;

static void trace_stored(const orc_scene* s, const double* tex, uint32_t pixel, uint32_t sample, uint32_t iter,
                         uint32_t stream, const double adj[3], double* grad, double Lout[3])
{
    rng_ctx R = { { s->seed, s->key_id }, pixel, sample, iter, stream };
    int nL = s->n_quads + (s->has_env ? 1 : 0);
    static vtx_t vs[MAXV + 2];
    int nv = 0;
    double u[4]; uint32_t raw[4];
    draw4(&R, 0, 0, u, raw);
    v3 o, d;
    camera_ray(s, (int)(pixel % (uint32_t)s->width), (int)(pixel / (uint32_t)s->width), u[0], u[1], &o, &d);
    double pdf_b = 0.0, pdf_env = 0.0;
    for (int k = 1; k <= s->max_depth && k <= MAXV; ++k) {
        vtx_t* V_ = &vs[nv++];
        memset(V_, 0, sizeof(*V_));
        hit_t h;
        if (!intersect(s, o, d, &h)) {
            if (s->has_env) {
                double w = (k == 1) ? 1.0 : mis2(pdf_b, pdf_env);
                for (int c = 0; c < 3; ++c) V_->E[c] = s->env[c] * w;
            }
            break;
        }
        surf_t si;
        surface(s, o, d, &h, &si);
        if (si.light >= 0 && quad_front(s, si.light, d)) {
            double w = (k == 1) ? 1.0 : mis2(pdf_b, quad_light_pdf(s, si.light, d, h.t));
            for (int c = 0; c < 3; ++c) V_->E[c] = s->quads[12 * si.light + 9 + c] * w;
        }
        if (k == s->max_depth) break;
        v3 wo = vmul(d, -1.0);
        v3 nf = vdot(si.n, d) < 0.0 ? si.n : vmul(si.n, -1.0);
        v3 po = offset_point(si.p, nf);
        load_material(s, tex, &si, &V_->m);
        V_->grad = V_->m.textured;
        draw4(&R, (uint32_t)k, 0, u, raw);
        nee_t nee;
        sample_light(s, po, nf, u, raw, &nee);
        if (nee.ok && !occluded(s, po, nee.wi, nee.tmax)) {
            double f[3], df[5][3];
            bsdf_eval(&V_->m, nf, wo, nee.wi, f, df);
            double pb = bsdf_pdf(&V_->m, nf, wo, nee.wi);
            double q = vdot(nee.wi, nf) * mis2(nee.pdf, pb) / nee.pdf;
            for (int c = 0; c < 3; ++c) {
                V_->N[c] = f[c] * nee.Le[c] * q;
                for (int j = 0; j < 5; ++j) V_->dN[j][c] = df[j][c] * nee.Le[c] * q;
            }
        }
        draw4(&R, (uint32_t)k, 1, u, raw);
        v3 wi;
        if (!bsdf_sample(&V_->m, nf, wo, u[0], u[1], u[2], &wi)) break;
        double pb = bsdf_pdf(&V_->m, nf, wo, wi);
        if (pb <= 0.0) break;
        bsdf_eval(&V_->m, nf, wo, wi, V_->fb, V_->dfb);
        double cs = vdot(wi, nf);
        V_->cb = cs / pb;
        V_->cont = 1;
        pdf_b = pb;
        pdf_env = s->has_env ? cs / (PI * nL) : 0.0;
        o = po;
        d = wi;
    }
    /* radiance: L = sum_k beta_k (E_k + N_k), beta_k = prod_{m<k} fb_m cb_m */
    for (int c = 0; c < 3; ++c) {
        double L = 0.0, beta = 1.0;
        for (int k = 0; k < nv; ++k) {
            L += beta * (vs[k].E[c] + vs[k].N[c]);
            beta *= vs[k].cont ? vs[k].fb[c] * vs[k].cb : 0.0;
        }
        Lout[c] = L;
    }
    if (!grad) return;
    for (int k = 0; k < nv; ++k) {
        if (!vs[k].grad) continue;
        double g[5] = { 0, 0, 0, 0, 0 };
        for (int j = 0; j < s->tex_c; ++j) {
            for (int c = 0; c < 3; ++c) {
                double bk = 1.0;
                for (int m = 0; m < k; ++m) bk *= vs[m].fb[c] * vs[m].cb;
                double acc = bk * vs[k].dN[j][c];
                if (vs[k].cont) {
                    for (int jj = k + 1; jj < nv; ++jj) {
                        double prod = 1.0;
                        for (int m = 0; m < jj; ++m)
                            prod *= (m == k) ? vs[k].dfb[j][c] * vs[k].cb : vs[m].fb[c] * vs[m].cb;
                        acc += prod * (vs[jj].E[c] + vs[jj].N[c]);
                    }
                }
                g[j] += adj[c] * acc;
            }
        }
        splat(s, &vs[k].m, g, grad);
    }
}

/* ------------------------------------------------------------------------- */
/* exported entry points                                                        */
/* ------------------------------------------------------------------------- */

/* radiance of n (pixel, sample) pairs */
void orc_render_samples(const orc_scene* s, const double* tex, int64_t n, const uint32_t* pixels,
                        const uint32_t* samples, uint32_t iter, uint32_t stream, double* out)
{
    for (int64_t i = 0; i < n; ++i)
        trace(s, tex, tex, pixels[i], samples[i], iter, stream, 0, NULL, NULL, NULL, out + 3 * i);
}

/* mean over spp samples per pixel; image [H*W*3], sample index s = 0..spp-1 */
void orc_render_image(const orc_scene* s, const double* tex, int spp, uint32_t iter, uint32_t stream, double* img)
{
    int64_t N = (int64_t)s->width * s->height;
    for (int64_t p = 0; p < N; ++p) {
        double acc[3] = { 0, 0, 0 };
        for (int k = 0; k < spp; ++k) {
            double L[3];
            trace(s, tex, tex, (uint32_t)p, (uint32_t)k, iter, stream, 0, NULL, NULL, NULL, L);
            for (int c = 0; c < 3; ++c) acc[c] += L[c];
        }
        for (int c = 0; c < 3; ++c) img[3 * p + c] = acc[c] / spp;
    }
}

/* gradient of sum_p sum_c dimg[p,c] * I_p,c with I_p = (1/spp) sum_s L_s, by PRB:
 * per path a radiance pass and a replay with the same counters; grad [H_t*W_t*C] is
 * accumulated (not cleared) */
void orc_adjoint_image(const orc_scene* s, const double* tex, int spp, uint32_t iter, uint32_t stream,
                       const double* dimg, double* grad)
{
    int64_t N = (int64_t)s->width * s->height;
    for (int64_t p = 0; p < N; ++p) {
        for (int k = 0; k < spp; ++k) {
            double adj[3] = { dimg[3 * p] / spp, dimg[3 * p + 1] / spp, dimg[3 * p + 2] / spp };
            double Lt[3], Lr[3];
            trace(s, tex, tex, (uint32_t)p, (uint32_t)k, iter, stream, 0, NULL, NULL, NULL, Lt);
            trace(s, tex, tex, (uint32_t)p, (uint32_t)k, iter, stream, 1, Lt, adj, grad, Lr);
        }
    }
}

/* The FD branch that shares the pi_i path (Eq. est_triv): image and PRB gradient of the
 * integrand at tex_e along paths sampled, with their densities and MIS weights, at tex_s. */
void orc_render_image_shared(const orc_scene* s, const double* tex_s, const double* tex_e, int spp, uint32_t iter,
                             uint32_t stream, double* img)
{
    int64_t N = (int64_t)s->width * s->height;
    for (int64_t p = 0; p < N; ++p) {
        double acc[3] = { 0, 0, 0 };
        for (int k = 0; k < spp; ++k) {
            double L[3];
            trace(s, tex_s, tex_e, (uint32_t)p, (uint32_t)k, iter, stream, 0, NULL, NULL, NULL, L);
            for (int c = 0; c < 3; ++c) acc[c] += L[c];
        }
        for (int c = 0; c < 3; ++c) img[3 * p + c] = acc[c] / spp;
    }
}

void orc_adjoint_image_shared(const orc_scene* s, const double* tex_s, const double* tex_e, int spp, uint32_t iter,
                              uint32_t stream, const double* dimg, double* grad)
{
    int64_t N = (int64_t)s->width * s->height;
    for (int64_t p = 0; p < N; ++p) {
        for (int k = 0; k < spp; ++k) {
            double adj[3] = { dimg[3 * p] / spp, dimg[3 * p + 1] / spp, dimg[3 * p + 2] / spp };
            double Lt[3], Lr[3];
            trace(s, tex_s, tex_e, (uint32_t)p, (uint32_t)k, iter, stream, 0, NULL, NULL, NULL, Lt);
            trace(s, tex_s, tex_e, (uint32_t)p, (uint32_t)k, iter, stream, 1, Lt, adj, grad, Lr);
        }
    }
}

/* the same gradient through the stored-vertex differentiation */
void orc_adjoint_image_stored(const orc_scene* s, const double* tex, int spp, uint32_t iter, uint32_t stream,
                              const double* dimg, double* grad)
{
    int64_t N = (int64_t)s->width * s->height;
    for (int64_t p = 0; p < N; ++p) {
        for (int k = 0; k < spp; ++k) {
            double adj[3] = { dimg[3 * p] / spp, dimg[3 * p + 1] / spp, dimg[3 * p + 2] / spp };
            double L[3];
            trace_stored(s, tex, (uint32_t)p, (uint32_t)k, iter, stream, adj, grad, L);
        }
    }
}

/* per-path PRB gradient for a list of (pixel, sample) pairs, each with its own adjoint
 * weight adj[3*i..] (already divided by spp); grads land in grad (accumulated) */
void orc_adjoint_samples(const orc_scene* s, const double* tex, int64_t n, const uint32_t* pixels,
                         const uint32_t* samples, uint32_t iter, uint32_t stream, const double* adj,
                         double* grad, int stored)
{
    for (int64_t i = 0; i < n; ++i) {
        double Lt[3], Lr[3];
        if (stored) {
            trace_stored(s, tex, pixels[i], samples[i], iter, stream, adj + 3 * i, grad, Lr);
        } else {
            trace(s, tex, tex, pixels[i], samples[i], iter, stream, 0, NULL, NULL, NULL, Lt);
            trace(s, tex, tex, pixels[i], samples[i], iter, stream, 1, Lt, adj + 3 * i, grad, Lr);
        }
    }
}

/* BSDF access for unit tests of the material model (n, wo, wi unit vectors) */
void orc_bsdf(int type, const double th[5], const double n[3], const double wo[3], const double wi[3],
              double f[3], double df[15], double* pdf)
{
    mat_t m;
    memset(&m, 0, sizeof(m));
    m.type = type;
    for (int j = 0; j < 5; ++j) m.th[j] = th[j];
    double dd[5][3];
    v3 N = V(n[0], n[1], n[2]), O = V(wo[0], wo[1], wo[2]), I = V(wi[0], wi[1], wi[2]);
    bsdf_eval(&m, N, O, I, f, dd);
    for (int j = 0; j < 5; ++j)
        for (int c = 0; c < 3; ++c) df[3 * j + c] = dd[j][c];
    *pdf = bsdf_pdf(&m, N, O, I);
}

int orc_bsdf_sample(int type, const double th[5], const double n[3], const double wo[3], double ul, double u1,
                    double u2, double wi[3])
{
    mat_t m;
    memset(&m, 0, sizeof(m));
    m.type = type;
    for (int j = 0; j < 5; ++j) m.th[j] = th[j];
    v3 w;
    int ok = bsdf_sample(&m, V(n[0], n[1], n[2]), V(wo[0], wo[1], wo[2]), ul, u1, u2, &w);
    wi[0] = w.x; wi[1] = w.y; wi[2] = w.z;
    return ok;
}

/* textbook L2 image loss and its derivative: L = 1/(3N) sum (I-T)^2, dL/dI = 2(I-T)/(3N) */
double orc_l2_loss(int64_t n_pix, const double* img, const double* target, double* dimg)
{
    double acc = 0.0;
    double inv = 1.0 / (3.0 * (double)n_pix);
    for (int64_t i = 0; i < 3 * n_pix; ++i) {
        double r = img[i] - target[i];
        acc += r * r;
        if (dimg) dimg[i] = 2.0 * r * inv;
    }
    return acc * inv;
}

/* Relative squared error of the experiments' setup (Sec. 6), normalised by the target alone:
 * L = 1/(3N) sum (I - T)^2 / (T^2 + 0.01), dL/dI = 2 (I - T) / ((T^2 + 0.01) 3N). */
double orc_mrse_loss(int64_t n_pix, const double* img, const double* target, double* dimg)
{
    double acc = 0.0;
    double inv = 1.0 / (3.0 * (double)n_pix);
    for (int64_t i = 0; i < 3 * n_pix; ++i) {
        double r = img[i] - target[i];
        double w = 1.0 / (target[i] * target[i] + 0.01);
        acc += r * r * w;
        if (dimg) dimg[i] = 2.0 * r * w * inv;
    }
    return acc * inv;
}

/* n Philox evaluations: ctr [n][4], out [n][4] */
void orc_philox_batch(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i) orc_philox(ctr + 4 * i, key, out + 4 * i);
}

/* ========================================================================= */
/* Emissive-absorptive volume (the high-dimensional experiment of Sec. 6):    */
/* a voxel grid of emission (RGB) and density over an axis-aligned box, seen  */
/* from several pinhole views and rendered by a jittered ray march:           */
/*   L = sum_k T_k (1 - exp(-sigma_k delta)) e_k + T_end * background,        */
/*   T_{k+1} = T_k exp(-sigma_k delta),                                       */
/* sample k at t0 + (k + u) delta for one uniform u per ray (Philox vertex 1), */
/* samples past the exit skipped. Parameters: ((z ny + y) nx + x) * 4 + c,     */
/* c = 0..2 emission, 3 density; trilinear, clamp-to-edge, voxel centres at    */
/* (i + 1/2) / n across the box. Gradients by replay: d L / d e_k = T_k a_k,   */
/* d L / d sigma_k = delta ((1 - a_k) T_k e_k - L_after_k).                    */
/* ========================================================================= */
typedef struct {
    int32_t nx, ny, nz;
    float lo[3], hi[3];
    int32_t n_views, width, height;
    const float* cameras;   /* [n_views][10]: eye, target, up, fov_deg */
    float step;             /* march step (world units) */
    float bg[3];
    uint32_t seed, key_id;
} orc_volume;

static void vol_camera_ray(const orc_volume* v, int view, int px, int py, double j0, double j1, v3* o, v3* d)
{
    const float* c = v->cameras + 10 * view;
    v3 eye = vload(c), tg = vload(c + 3), up = vload(c + 6);
    v3 f = vnorm(vsub(tg, eye));
    v3 r = vnorm(vcross(f, up));
    v3 u = vcross(r, f);
    double th = tan(0.5 * c[9] * PI / 180.0);
    double asp = (double)v->width / (double)v->height;
    double sx = (2.0 * (px + j0) / v->width - 1.0) * th * asp;
    double sy = (1.0 - 2.0 * (py + j1) / v->height) * th;
    *o = eye;
    *d = vnorm(vadd(f, vadd(vmul(r, sx), vmul(u, sy))));
}

/* entry and exit of the box along the ray (t0 clamped to 0); 0 if the ray misses */
static int vol_box(const orc_volume* v, v3 o, v3 d, double* t0, double* t1)
{
    double a = 0.0, b = INFINITY;
    double oo[3] = { o.x, o.y, o.z }, dd[3] = { d.x, d.y, d.z };
    for (int k = 0; k < 3; ++k) {
        double lo = v->lo[k], hi = v->hi[k];
        if (dd[k] == 0.0) {
            if (oo[k] < lo || oo[k] > hi) return 0;
            continue;
        }
        double ta = (lo - oo[k]) / dd[k], tb = (hi - oo[k]) / dd[k];
        if (ta > tb) { double t = ta; ta = tb; tb = t; }
        if (ta > a) a = ta;
        if (tb < b) b = tb;
    }
    *t0 = a;
    *t1 = b;
    return b > a;
}

/* trilinear taps of point p: voxel indices and weights (clamp-to-edge) */
static void vol_taps(const orc_volume* v, v3 p, int idx[8], double w[8])
{
    int n[3] = { v->nx, v->ny, v->nz };
    double pp[3] = { p.x, p.y, p.z };
    int i0[3], i1[3];
    double f[3];
    for (int k = 0; k < 3; ++k) {
        double g = (pp[k] - v->lo[k]) / (v->hi[k] - v->lo[k]) * n[k] - 0.5;
        double fl = floor(g);
        f[k] = g - fl;
        int a = (int)fl, b = a + 1;
        if (a < 0) a = 0;
        if (a > n[k] - 1) a = n[k] - 1;
        if (b < 0) b = 0;
        if (b > n[k] - 1) b = n[k] - 1;
        i0[k] = a;
        i1[k] = b;
    }
    for (int c = 0; c < 8; ++c) {
        int x = (c & 1) ? i1[0] : i0[0], y = (c & 2) ? i1[1] : i0[1], z = (c & 4) ? i1[2] : i0[2];
        double wx = (c & 1) ? f[0] : 1.0 - f[0], wy = (c & 2) ? f[1] : 1.0 - f[1], wz = (c & 4) ? f[2] : 1.0 - f[2];
        idx[c] = (z * v->ny + y) * v->nx + x;
        w[c] = wx * wy * wz;
    }
}

/* one sample of pixel `pixel` (= view * W * H + py * W + px). mode 0: radiance into Lout. mode 1:
 * replay with the sample's total radiance Ltot and adjoint weight adj, gradients into grad. */
static void vol_march(const orc_volume* v, const double* par, uint32_t pixel, uint32_t sample, uint32_t iter,
                      uint32_t stream, int mode, const double Ltot[3], const double adj[3], double* grad,
                      double Lout[3])
{
    rng_ctx R = { { v->seed, v->key_id }, pixel, sample, iter, stream };
    uint32_t per_view = (uint32_t)v->width * (uint32_t)v->height;
    int view = (int)(pixel / per_view);
    uint32_t local = pixel % per_view;
    double u[4];
    draw4(&R, 0, 0, u, NULL);
    v3 o, d;
    vol_camera_ray(v, view, (int)(local % (uint32_t)v->width), (int)(local / (uint32_t)v->width), u[0], u[1], &o, &d);
    double L[3] = { 0, 0, 0 }, T = 1.0;
    double t0, t1;
    if (vol_box(v, o, d, &t0, &t1)) {
        draw4(&R, 1, 0, u, NULL);
        const double dl = v->step;
        for (int k = 0;; ++k) {
            double t = t0 + (k + u[0]) * dl;
            if (!(t < t1)) break;
            v3 p = vadd(o, vmul(d, t));
            int idx[8];
            double w[8], e[3] = { 0, 0, 0 }, sg = 0.0;
            vol_taps(v, p, idx, w);
            for (int c = 0; c < 8; ++c) {
                for (int j = 0; j < 3; ++j) e[j] += w[c] * par[4 * (size_t)idx[c] + j];
                sg += w[c] * par[4 * (size_t)idx[c] + 3];
            }
            double tr = exp(-sg * dl), a = 1.0 - tr;
            for (int j = 0; j < 3; ++j) L[j] += T * a * e[j];
            if (mode == 1) {
                double ge[3], gs = 0.0;
                for (int j = 0; j < 3; ++j) {
                    double after = Ltot[j] - L[j];
                    ge[j] = adj[j] * T * a;
                    gs += adj[j] * (tr * T * e[j] - after);
                }
                gs *= dl;
                for (int c = 0; c < 8; ++c) {
                    for (int j = 0; j < 3; ++j) grad[4 * (size_t)idx[c] + j] += w[c] * ge[j];
                    grad[4 * (size_t)idx[c] + 3] += w[c] * gs;
                }
            }
            T *= tr;
        }
    }
    for (int j = 0; j < 3; ++j) L[j] += T * v->bg[j];
    for (int j = 0; j < 3; ++j) Lout[j] = L[j];
}

void orc_vol_render_samples(const orc_volume* v, const double* par, int64_t n, const uint32_t* pixels,
                            const uint32_t* samples, uint32_t iter, uint32_t stream, double* out)
{
    for (int64_t i = 0; i < n; ++i) vol_march(v, par, pixels[i], samples[i], iter, stream, 0, NULL, NULL, NULL, out + 3 * i);
}

/* mean over spp samples per pixel; image [n_views * H * W * 3] */
void orc_vol_render_image(const orc_volume* v, const double* par, int spp, uint32_t iter, uint32_t stream, double* img)
{
    int64_t N = (int64_t)v->n_views * v->width * v->height;
    for (int64_t p = 0; p < N; ++p) {
        double acc[3] = { 0, 0, 0 };
        for (int k = 0; k < spp; ++k) {
            double L[3];
            vol_march(v, par, (uint32_t)p, (uint32_t)k, iter, stream, 0, NULL, NULL, NULL, L);
            for (int c = 0; c < 3; ++c) acc[c] += L[c];
        }
        for (int c = 0; c < 3; ++c) img[3 * p + c] = acc[c] / spp;
    }
}

/* gradient of sum_p dimg[p] . I_p (I_p the spp-sample mean), accumulated into grad [nvox * 4] */
void orc_vol_adjoint_image(const orc_volume* v, const double* par, int spp, uint32_t iter, uint32_t stream,
                           const double* dimg, double* grad)
{
    int64_t N = (int64_t)v->n_views * v->width * v->height;
    for (int64_t p = 0; p < N; ++p) {
        for (int k = 0; k < spp; ++k) {
            double adj[3] = { dimg[3 * p] / spp, dimg[3 * p + 1] / spp, dimg[3 * p + 2] / spp };
            double Lt[3], Lr[3];
            vol_march(v, par, (uint32_t)p, (uint32_t)k, iter, stream, 0, NULL, NULL, NULL, Lt);
            vol_march(v, par, (uint32_t)p, (uint32_t)k, iter, stream, 1, Lt, adj, grad, Lr);
        }
    }
}

"""ctypes binding of the FP64 oracle (oracle.c) plus image-level helpers.

TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the benchmark's
CPU-baseline leg; never by the product path.

The FD estimator is computed here exactly as Eq. est_triv defines it: the same
random numbers (same counters) evaluated at pi_i and at pi_{i-1} in two separate
renders / adjoint passes, then subtracted.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import build as _build

ST_PROP_PRIMAL, ST_PROP_ADJ, ST_FD_PRIMAL, ST_FD_ADJ, ST_TARGET, ST_EVAL = range(6)

_f32p = ct.POINTER(ct.c_float)
_f64p = ct.POINTER(ct.c_double)
_i32p = ct.POINTER(ct.c_int32)
_u32p = ct.POINTER(ct.c_uint32)


class OrcScene(ct.Structure):
    _fields_ = [
        ("n_verts", ct.c_int32), ("n_tris", ct.c_int32),
        ("pos", _f32p), ("uv", _f32p), ("tris", _i32p), ("tri_mat", _i32p), ("tri_light", _i32p),
        ("n_spheres", ct.c_int32), ("spheres", _f32p), ("sph_mat", _i32p),
        ("n_mats", ct.c_int32), ("mat_type", _i32p), ("mat_textured", _i32p), ("mat_const", _f32p),
        ("n_quads", ct.c_int32), ("quads", _f32p),
        ("has_env", ct.c_int32), ("env", ct.c_float * 3),
        ("eye", ct.c_float * 3), ("target", ct.c_float * 3), ("up", ct.c_float * 3),
        ("fov_deg", ct.c_float),
        ("width", ct.c_int32), ("height", ct.c_int32),
        ("tex_c", ct.c_int32), ("tex_h", ct.c_int32), ("tex_w", ct.c_int32),
        ("max_depth", ct.c_int32),
        ("seed", ct.c_uint32), ("key_id", ct.c_uint32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ct.CDLL(_build.build())
        L.orc_philox.argtypes = [_u32p, _u32p, _u32p]
        L.orc_philox_batch.argtypes = [ct.c_int64, _u32p, _u32p, _u32p]
        L.orc_render_samples.argtypes = [ct.POINTER(OrcScene), _f64p, ct.c_int64, _u32p, _u32p,
                                         ct.c_uint32, ct.c_uint32, _f64p]
        L.orc_render_image.argtypes = [ct.POINTER(OrcScene), _f64p, ct.c_int, ct.c_uint32, ct.c_uint32, _f64p]
        L.orc_render_image_shared.argtypes = [ct.POINTER(OrcScene), _f64p, _f64p, ct.c_int, ct.c_uint32,
                                              ct.c_uint32, _f64p]
        L.orc_adjoint_image_shared.argtypes = [ct.POINTER(OrcScene), _f64p, _f64p, ct.c_int, ct.c_uint32,
                                               ct.c_uint32, _f64p, _f64p]
        for name in ("orc_adjoint_image", "orc_adjoint_image_stored"):
            getattr(L, name).argtypes = [ct.POINTER(OrcScene), _f64p, ct.c_int, ct.c_uint32, ct.c_uint32,
                                         _f64p, _f64p]
        L.orc_adjoint_samples.argtypes = [ct.POINTER(OrcScene), _f64p, ct.c_int64, _u32p, _u32p,
                                          ct.c_uint32, ct.c_uint32, _f64p, _f64p, ct.c_int]
        L.orc_bsdf.argtypes = [ct.c_int, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
        L.orc_bsdf_sample.argtypes = [ct.c_int, _f64p, _f64p, _f64p, ct.c_double, ct.c_double, ct.c_double, _f64p]
        L.orc_bsdf_sample.restype = ct.c_int
        L.orc_l2_loss.argtypes = [ct.c_int64, _f64p, _f64p, _f64p]
        L.orc_l2_loss.restype = ct.c_double
        L.orc_mrse_loss.argtypes = [ct.c_int64, _f64p, _f64p, _f64p]
        L.orc_vol_render_samples.argtypes = [ct.POINTER(OrcVolume), _f64p, ct.c_int64, _u32p, _u32p, ct.c_uint32,
                                             ct.c_uint32, _f64p]
        L.orc_vol_render_image.argtypes = [ct.POINTER(OrcVolume), _f64p, ct.c_int, ct.c_uint32, ct.c_uint32, _f64p]
        L.orc_vol_adjoint_image.argtypes = [ct.POINTER(OrcVolume), _f64p, ct.c_int, ct.c_uint32, ct.c_uint32,
                                            _f64p, _f64p]
        L.orc_mrse_loss.restype = ct.c_double
        _lib = L
    return _lib


_lib32 = None


def lib32():
    """The oracle's source built in single precision (oracle_f32.c): only the per-sample radiance,
    for telling paths that FP32 arithmetic cannot resolve to the parity tolerance."""
    global _lib32
    if _lib32 is None:
        L = ct.CDLL(_build.build_f32())
        f32p = ct.POINTER(ct.c_float)
        L.orc_render_samples.argtypes = [ct.POINTER(OrcScene), f32p, ct.c_int64, _u32p, _u32p, ct.c_uint32,
                                         ct.c_uint32, f32p]
        _lib32 = L
    return _lib32


def _p(a, t):
    return a.ctypes.data_as(t)


class Scene:
    """Holds contiguous copies of the scene arrays and the ctypes struct pointing at them."""

    def __init__(self, s: dict):
        self.d = s
        self._keep = {}

        def arr(name, dt, shape=None):
            a = np.ascontiguousarray(np.asarray(s[name], dt))
            if a.size == 0:
                a = np.zeros(1, dt)
            self._keep[name] = a
            return a

        st = OrcScene()
        pos = arr("positions", np.float32)
        tris = arr("tris", np.int32)
        st.n_verts = int(np.asarray(s["positions"]).reshape(-1, 3).shape[0])
        st.n_tris = int(np.asarray(s["tris"]).reshape(-1, 3).shape[0])
        st.pos = _p(pos, _f32p)
        st.uv = _p(arr("uvs", np.float32), _f32p)
        st.tris = _p(tris, _i32p)
        st.tri_mat = _p(arr("tri_mat", np.int32), _i32p)
        st.tri_light = _p(arr("tri_light", np.int32), _i32p)
        st.n_spheres = int(np.asarray(s["spheres"]).reshape(-1, 8).shape[0])
        st.spheres = _p(arr("spheres", np.float32), _f32p)
        st.sph_mat = _p(arr("sph_mat", np.int32), _i32p)
        st.n_mats = int(len(s["mat_type"]))
        st.mat_type = _p(arr("mat_type", np.int32), _i32p)
        st.mat_textured = _p(arr("mat_textured", np.int32), _i32p)
        st.mat_const = _p(arr("mat_const", np.float32), _f32p)
        st.n_quads = int(np.asarray(s["quads"]).reshape(-1, 12).shape[0])
        st.quads = _p(arr("quads", np.float32), _f32p)
        st.has_env = int(s["has_env"])
        for k in ("env", "eye", "target", "up"):
            getattr(st, k)[:] = [float(x) for x in np.asarray(s[k], np.float32)]
        st.fov_deg = float(s["fov_deg"])
        st.width, st.height = int(s["width"]), int(s["height"])
        st.tex_c, st.tex_h, st.tex_w = int(s["tex_c"]), int(s["tex_h"]), int(s["tex_w"])
        st.max_depth = int(s["max_depth"])
        st.seed, st.key_id = int(s["seed"]) & 0xFFFFFFFF, int(s["key_id"]) & 0xFFFFFFFF
        self.st = st

    @property
    def n_pix(self):
        return self.st.width * self.st.height

    @property
    def tex_shape(self):
        return (self.st.tex_h, self.st.tex_w, self.st.tex_c)

    def ref(self):
        return ct.byref(self.st)


def philox(ctr, key):
    """Philox4x32-10 of one counter (4 x u32) under one key (2 x u32)."""
    c = np.asarray(ctr, np.uint32).copy()
    k = np.asarray(key, np.uint32).copy()
    o = np.zeros(4, np.uint32)
    lib().orc_philox(_p(c, _u32p), _p(k, _u32p), _p(o, _u32p))
    return o


def philox_batch(ctr, key):
    """Philox4x32-10 of counters ctr [n, 4] under one key."""
    c = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros_like(c)
    lib().orc_philox_batch(c.shape[0], _p(c, _u32p), _p(k, _u32p), _p(o, _u32p))
    return o


def _tex(tex):
    return np.ascontiguousarray(np.asarray(tex, np.float64))


def render_samples(sc: Scene, tex, pixels, samples, iteration, stream):
    pixels = np.ascontiguousarray(pixels, np.uint32)
    samples = np.ascontiguousarray(samples, np.uint32)
    out = np.zeros((len(pixels), 3), np.float64)
    t = _tex(tex)
    lib().orc_render_samples(sc.ref(), _p(t, _f64p), len(pixels), _p(pixels, _u32p), _p(samples, _u32p),
                             iteration, stream, _p(out, _f64p))
    return out


def render_samples_f32(sc: Scene, tex, pixels, samples, iteration, stream):
    """render_samples evaluated by the single-precision build (never a reference value)."""
    pixels = np.ascontiguousarray(pixels, np.uint32)
    samples = np.ascontiguousarray(samples, np.uint32)
    out = np.zeros((len(pixels), 3), np.float32)
    t = np.ascontiguousarray(np.asarray(tex, np.float32))
    f32p = ct.POINTER(ct.c_float)
    lib32().orc_render_samples(sc.ref(), t.ctypes.data_as(f32p), len(pixels), _p(pixels, _u32p), _p(samples, _u32p),
                               iteration, stream, out.ctypes.data_as(f32p))
    return out.astype(np.float64)


def render_image(sc: Scene, tex, spp, iteration, stream):
    out = np.zeros((sc.st.height, sc.st.width, 3), np.float64)
    t = _tex(tex)
    lib().orc_render_image(sc.ref(), _p(t, _f64p), spp, iteration, stream, _p(out, _f64p))
    return out


def adjoint_image(sc: Scene, tex, spp, iteration, stream, dimg, stored=False):
    """d/dtex of sum(dimg * I) with I the spp-sample image of (iteration, stream)."""
    grad = np.zeros(sc.tex_shape, np.float64)
    t = _tex(tex)
    d = np.ascontiguousarray(dimg, np.float64)
    fn = lib().orc_adjoint_image_stored if stored else lib().orc_adjoint_image
    fn(sc.ref(), _p(t, _f64p), spp, iteration, stream, _p(d, _f64p), _p(grad, _f64p))
    return grad


def render_image_shared(sc: Scene, tex_s, tex_e, spp, iteration, stream):
    """Image of the integrand at tex_e along paths sampled (directions, densities, MIS) at tex_s."""
    out = np.zeros((sc.st.height, sc.st.width, 3), np.float64)
    ts, te = _tex(tex_s), _tex(tex_e)
    lib().orc_render_image_shared(sc.ref(), _p(ts, _f64p), _p(te, _f64p), spp, iteration, stream, _p(out, _f64p))
    return out


def adjoint_image_shared(sc: Scene, tex_s, tex_e, spp, iteration, stream, dimg):
    """PRB gradient (w.r.t. tex_e) of sum(dimg * I) for the paths sampled at tex_s."""
    grad = np.zeros(sc.tex_shape, np.float64)
    ts, te = _tex(tex_s), _tex(tex_e)
    d = np.ascontiguousarray(dimg, np.float64)
    lib().orc_adjoint_image_shared(sc.ref(), _p(ts, _f64p), _p(te, _f64p), spp, iteration, stream, _p(d, _f64p),
                                   _p(grad, _f64p))
    return grad


def adjoint_samples(sc: Scene, tex, pixels, samples, iteration, stream, adj, stored=False):
    pixels = np.ascontiguousarray(pixels, np.uint32)
    samples = np.ascontiguousarray(samples, np.uint32)
    adj = np.ascontiguousarray(adj, np.float64).reshape(-1, 3)
    grad = np.zeros(sc.tex_shape, np.float64)
    t = _tex(tex)
    lib().orc_adjoint_samples(sc.ref(), _p(t, _f64p), len(pixels), _p(pixels, _u32p), _p(samples, _u32p),
                              iteration, stream, _p(adj, _f64p), _p(grad, _f64p), int(stored))
    return grad


def l2_loss(img, target):
    img = np.ascontiguousarray(img, np.float64)
    target = np.ascontiguousarray(target, np.float64)
    d = np.zeros_like(img)
    loss = lib().orc_l2_loss(img.size // 3, _p(img, _f64p), _p(target, _f64p), _p(d, _f64p))
    return loss, d


LOSS_L2, LOSS_MRSE = 0, 1


def mrse_loss(img, target):
    """Relative squared error (Sec. 6 setup) and its adjoint image; see orc_mrse_loss."""
    img = np.ascontiguousarray(img, np.float64)
    target = np.ascontiguousarray(target, np.float64)
    d = np.zeros_like(img)
    loss = lib().orc_mrse_loss(img.size // 3, _p(img, _f64p), _p(target, _f64p), _p(d, _f64p))
    return loss, d


def image_loss(img, target, kind=LOSS_L2):
    return mrse_loss(img, target) if kind == LOSS_MRSE else l2_loss(img, target)


def bsdf(mtype, th, n, wo, wi):
    th = np.ascontiguousarray(th, np.float64)
    n, wo, wi = (np.ascontiguousarray(x, np.float64) for x in (n, wo, wi))
    f = np.zeros(3)
    df = np.zeros(15)
    pdf = np.zeros(1)
    lib().orc_bsdf(mtype, _p(th, _f64p), _p(n, _f64p), _p(wo, _f64p), _p(wi, _f64p),
                   _p(f, _f64p), _p(df, _f64p), _p(pdf, _f64p))
    return f, df.reshape(5, 3), float(pdf[0])


def bsdf_sample(mtype, th, n, wo, ul, u1, u2):
    th = np.ascontiguousarray(th, np.float64)
    n, wo = (np.ascontiguousarray(x, np.float64) for x in (n, wo))
    wi = np.zeros(3)
    ok = lib().orc_bsdf_sample(mtype, _p(th, _f64p), _p(n, _f64p), _p(wo, _f64p), ul, u1, u2, _p(wi, _f64p))
    return bool(ok), wi


# ---------------------------------------------------------------------------
# one iteration's gradient estimates (Sec. 3, Eq. est_def and est_triv)
# ---------------------------------------------------------------------------

def prop_gradient(sc: Scene, tex, target, spp, iteration, stream_offset=0, loss_kind=0):
    """<F_i>: image-loss gradient (L2, or MRSE with loss_kind 1) with an independent primal image (stream PROP_PRIMAL) for the
    adjoint weights and the PRB adjoint on stream PROP_ADJ. Returns (grad, loss, image).
    stream_offset shifts both streams (the independent variance samples of the uncorrelated
    variant use offset 8)."""
    img = render_image(sc, tex, spp, iteration, ST_PROP_PRIMAL + stream_offset)
    loss, dimg = image_loss(img, target, loss_kind)
    g = adjoint_image(sc, tex, spp, iteration, ST_PROP_ADJ + stream_offset, dimg)
    return g, loss, img


def fd_gradient(sc: Scene, tex_cur, tex_prev, target, spp, iteration, stream_offset=0, loss_kind=0,
                shared=False):
    """<dF_i> = <F_i>(u) - <F_{i-1}>(u): both terms use the same counters (streams FD_PRIMAL
    for the adjoint weights and FD_ADJ for the adjoint) at pi_i and pi_{i-1}; stream_offset
    shifts both streams as in prop_gradient. shared: the pi_{i-1} term follows the pi_i paths
    and divides by their density (Eq. est_triv read literally) instead of replaying the same
    random numbers with its own sampling."""
    img_c = render_image(sc, tex_cur, spp, iteration, ST_FD_PRIMAL + stream_offset)
    if shared:
        img_p = render_image_shared(sc, tex_cur, tex_prev, spp, iteration, ST_FD_PRIMAL + stream_offset)
    else:
        img_p = render_image(sc, tex_prev, spp, iteration, ST_FD_PRIMAL + stream_offset)
    _, d_c = image_loss(img_c, target, loss_kind)
    _, d_p = image_loss(img_p, target, loss_kind)
    g_c = adjoint_image(sc, tex_cur, spp, iteration, ST_FD_ADJ + stream_offset, d_c)
    if shared:
        g_p = adjoint_image_shared(sc, tex_cur, tex_prev, spp, iteration, ST_FD_ADJ + stream_offset, d_p)
    else:
        g_p = adjoint_image(sc, tex_prev, spp, iteration, ST_FD_ADJ + stream_offset, d_p)
    return g_c - g_p


# ---------------------------------------------------------------------------------------
# emissive-absorptive volume (see orc_vol_* in oracle.c)
# ---------------------------------------------------------------------------------------
class OrcVolume(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32), ("lo", ct.c_float * 3),
                ("hi", ct.c_float * 3), ("n_views", ct.c_int32), ("width", ct.c_int32), ("height", ct.c_int32),
                ("cameras", ct.POINTER(ct.c_float)), ("step", ct.c_float), ("bg", ct.c_float * 3),
                ("seed", ct.c_uint32), ("key_id", ct.c_uint32)]


class Volume:
    """A volume scene dict (synth.volume_scene) held for the oracle."""

    def __init__(self, scene: dict):
        self.cams = np.ascontiguousarray(scene["cameras"], np.float32)
        v = OrcVolume()
        v.nx, v.ny, v.nz = scene["nx"], scene["ny"], scene["nz"]
        v.lo = (ct.c_float * 3)(*scene["lo"])
        v.hi = (ct.c_float * 3)(*scene["hi"])
        v.n_views, v.width, v.height = scene["n_views"], scene["width"], scene["height"]
        v.cameras = self.cams.ctypes.data_as(ct.POINTER(ct.c_float))
        v.step = scene["step"]
        v.bg = (ct.c_float * 3)(*scene["bg"])
        v.seed, v.key_id = scene["seed"], scene["key_id"]
        self.v = v
        self.shape = (scene["nz"], scene["ny"], scene["nx"], 4)
        self.image_shape = (scene["n_views"], scene["height"], scene["width"], 3)

    def ref(self):
        return ct.byref(self.v)


def vol_render_image(vol: Volume, params, spp, iteration, stream):
    out = np.zeros(vol.image_shape, np.float64)
    par = np.ascontiguousarray(params, np.float64)
    lib().orc_vol_render_image(vol.ref(), _p(par, _f64p), spp, iteration, stream, _p(out, _f64p))
    return out


def vol_render_samples(vol: Volume, params, pixels, samples, iteration, stream):
    pixels = np.ascontiguousarray(pixels, np.uint32)
    samples = np.ascontiguousarray(samples, np.uint32)
    out = np.zeros((len(pixels), 3), np.float64)
    par = np.ascontiguousarray(params, np.float64)
    lib().orc_vol_render_samples(vol.ref(), _p(par, _f64p), len(pixels), _p(pixels, _u32p), _p(samples, _u32p),
                                 iteration, stream, _p(out, _f64p))
    return out


def vol_adjoint_image(vol: Volume, params, spp, iteration, stream, dimg):
    grad = np.zeros(vol.shape, np.float64)
    par = np.ascontiguousarray(params, np.float64)
    d = np.ascontiguousarray(dimg, np.float64)
    lib().orc_vol_adjoint_image(vol.ref(), _p(par, _f64p), spp, iteration, stream, _p(d, _f64p), _p(grad, _f64p))
    return grad


"""Thin Python binding over the C ABI (include/mer.h): argument marshalling only.

Every computation runs in the CUDA library; PyTorch only provides device memory and the
current stream. Tensors passed in must live on the context's device.
"""
from __future__ import annotations

import ctypes as ct
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import check

STREAM_PROP_PRIMAL = _lib.STREAM_PROP_PRIMAL
STREAM_PROP_ADJ = _lib.STREAM_PROP_ADJ
STREAM_FD_PRIMAL = _lib.STREAM_FD_PRIMAL
STREAM_FD_ADJ = _lib.STREAM_FD_ADJ
STREAM_TARGET = _lib.STREAM_TARGET
STREAM_EVAL = _lib.STREAM_EVAL
MODE_META, MODE_ADAM = _lib.MODE_META, _lib.MODE_ADAM


@dataclass
class HyperParams:
    mode: int = MODE_META
    lr: float = 0.01
    beta_f: float = 0.99
    beta_d: float = 0.9
    eps: float = 1e-8
    eps_alpha: float = 1e-30
    beta1: float = 0.9
    beta2: float = 0.999
    flags: int = 0            # MER_META_* variant bits (META_* constants below)
    precond_lambda: float = 0.0   # > 0: (I + lambda L)^{-1} gradient preconditioning per texture channel

    def to_c(self) -> _lib.Hyper:
        return _lib.Hyper(self.mode, self.lr, self.beta_f, self.beta_d, self.eps, self.eps_alpha, self.beta1,
                          self.beta2, self.flags, self.precond_lambda)


# image losses (scene key "loss"; the header's MER_LOSS_* values)
LOSS_L2 = 0
LOSS_MRSE = 1

# variant bits of HyperParams.flags (the header's MER_META_* values)
META_PER_ELEMENT = 1
META_NO_CLIP = 2
META_CENTRED = 4
META_GROWING_BETA = 8
META_NAIVE_ADAM = 16
META_UNCORRELATED = 32
META_FD_SHARED_PATH = 64


def _ptr(t):
    return ct.c_void_p(0 if t is None else t.data_ptr())


def _cur_stream(device):
    return ct.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _numel(x) -> int:
    return x.numel() if isinstance(x, torch.Tensor) else int(np.asarray(x).size)


def _need(x, numel, what):
    """Refuses an array whose element count is not `numel` (the library receives bare pointers: a
    short array would be read past its end)."""
    if _numel(x) != numel:
        raise ValueError(f"{what}: {numel} values expected, got {_numel(x)}")
    return x


def _dev_f32(x, device, numel=None, what="array"):
    """x as a contiguous float32 tensor on `device`, its element count checked before any copy."""
    if numel is not None:
        _need(x, numel, what)
    if isinstance(x, torch.Tensor):
        t = x.to(device=device, dtype=torch.float32)
    else:
        t = torch.as_tensor(np.asarray(x, np.float32), device=device)
    return t.contiguous()


def _out_f32(t, device, numel, what="output"):
    """A caller-supplied output buffer: float32, contiguous, on `device`, with `numel` elements."""
    if not (isinstance(t, torch.Tensor) and t.dtype == torch.float32 and t.device == torch.device(device)
            and t.is_contiguous() and t.numel() == numel):
        raise ValueError(f"{what}: a contiguous float32 tensor of {numel} elements on {device} expected")
    return t


def _dev_buf(t, dtype, numel, what, device=None):
    """A caller-supplied device tensor handed to the library as is: contiguous, `dtype`, `numel`
    values (at least `-numel` if negative), on a CUDA device (`device` if given)."""
    ok = (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
          and (t.numel() == numel if numel >= 0 else t.numel() >= -numel)
          and (device is None or t.device == device))
    if not ok:
        raise ValueError(f"{what}: a contiguous CUDA {dtype} tensor of {abs(numel)} elements expected")
    return t


def _host_buf(t, dtype, numel, what):
    """A caller-supplied host tensor for the asynchronous copies: contiguous, `dtype`, `numel` values."""
    if not (isinstance(t, torch.Tensor) and t.device.type == "cpu" and t.dtype == dtype and t.is_contiguous()
            and t.numel() == numel):
        raise ValueError(f"{what}: a contiguous host {dtype} tensor of {numel} elements expected")
    return t


class _Arr:
    """Keeps numpy arrays alive while their pointers sit in a SceneDesc."""

    def __init__(self):
        self.keep = []

    def __call__(self, a, dt, cty):
        a = np.ascontiguousarray(np.asarray(a, dt))
        if a.size == 0:
            a = np.zeros(1, dt)
        self.keep.append(a)
        return a.ctypes.data_as(ct.POINTER(cty))


def scene_desc(scene: dict, hyper: HyperParams) -> tuple[_lib.SceneDesc, _Arr]:
    A = _Arr()
    d = _lib.SceneDesc()
    pos = np.asarray(scene["positions"], np.float32).reshape(-1, 3)
    tris = np.asarray(scene["tris"], np.int32).reshape(-1, 3)
    d.n_verts, d.n_tris = pos.shape[0], tris.shape[0]
    d.positions = A(pos, np.float32, ct.c_float)
    d.uvs = A(scene["uvs"], np.float32, ct.c_float)
    d.tris = A(tris, np.int32, ct.c_int32)
    d.tri_mat = A(scene["tri_mat"], np.int32, ct.c_int32)
    d.tri_light = A(scene["tri_light"], np.int32, ct.c_int32)
    sph = np.asarray(scene["spheres"], np.float32).reshape(-1, 8)
    d.n_spheres = sph.shape[0]
    d.spheres = A(sph, np.float32, ct.c_float)
    d.sph_mat = A(scene["sph_mat"], np.int32, ct.c_int32)
    d.n_mats = len(scene["mat_type"])
    d.mat_type = A(scene["mat_type"], np.int32, ct.c_int32)
    d.mat_textured = A(scene["mat_textured"], np.int32, ct.c_int32)
    d.mat_const = A(scene["mat_const"], np.float32, ct.c_float)
    q = np.asarray(scene["quads"], np.float32).reshape(-1, 12)
    d.n_quads = q.shape[0]
    d.quads = A(q, np.float32, ct.c_float)
    d.has_env = int(scene["has_env"])
    for k in ("env", "eye", "target", "up"):
        getattr(d, k)[:] = [float(v) for v in np.asarray(scene[k], np.float32)]
    d.fov_deg = float(scene["fov_deg"])
    d.width, d.height = int(scene["width"]), int(scene["height"])
    d.tex_c, d.tex_h, d.tex_w = int(scene["tex_c"]), int(scene["tex_h"]), int(scene["tex_w"])
    lo = np.zeros(8, np.float32)
    hi = np.zeros(8, np.float32)
    lo[:d.tex_c] = scene["clamp_lo"]
    hi[:d.tex_c] = scene["clamp_hi"]
    d.clamp_lo[:] = lo.tolist()
    d.clamp_hi[:] = hi.tolist()
    d.max_depth = int(scene["max_depth"])
    d.spp_prop, d.spp_fd = int(scene["spp_prop"]), int(scene["spp_fd"])
    d.seed, d.key_id = int(scene["seed"]) & 0xFFFFFFFF, int(scene["key_id"]) & 0xFFFFFFFF
    d.loss = int(scene.get("loss", LOSS_L2))
    d.hyper = hyper.to_c()
    return d, A


class Context:
    """A set of inverse-rendering problems on one GPU (mer_ctx)."""

    def __init__(self, device: int = 0, block_size: int = 0, blocks_per_sm: int = 0, smem_nodes: int = 0,
                 max_paths: int = 0, replay_hit_store: bool = False, trace_refill: int = 0):
        self.L = _lib.load()
        self.device = torch.device("cuda", device)
        cfg = _lib.Config(device, block_size, blocks_per_sm, smem_nodes, max_paths, int(replay_hit_store),
                          int(trace_refill))
        h = ct.c_void_p()
        check(self.L.mer_create(ct.byref(cfg), _cur_stream(self.device), ct.byref(h)))
        self.h = h
        self.shapes = []   # (H, W, C) texture shape per problem
        self.images = []   # (height, width) per problem

    def close(self):
        if getattr(self, "h", None):
            self.L.mer_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, s):
        check(s, self.h)

    # ---- problems ----
    def add_scene(self, scene: dict, hyper: HyperParams | None = None) -> int:
        d, keep = scene_desc(scene, hyper or HyperParams())
        pid = ct.c_int32()
        self._ck(self.L.mer_scene_add(self.h, ct.byref(d), ct.byref(pid)))
        del keep
        self.shapes.append((int(scene["tex_h"]), int(scene["tex_w"]), int(scene["tex_c"])))
        self.images.append((int(scene["height"]), int(scene["width"])))
        return pid.value

    def _ntex(self, pid: int) -> int:
        h, w, c = self.shapes[pid]
        return h * w * c

    def _nimg(self, pid: int) -> int:
        h, w = self.images[pid]
        return h * w * 3

    def set_params(self, pid: int, tex):
        t = _dev_f32(tex, self.device, self._ntex(pid), "texture")
        self._ck(self.L.mer_params_set(self.h, pid, _ptr(t), 1))
        torch.cuda.current_stream(self.device).synchronize()

    def force_params(self, pid: int, tex):
        """Replace the parameters the last update produced by `tex` (prescribed trajectory)."""
        t = _dev_f32(tex, self.device, self._ntex(pid), "texture")
        torch.cuda.current_stream(self.device).synchronize()
        self._ck(self.L.mer_params_force(self.h, pid, _ptr(t), 1))

    def get_params(self, pid: int) -> torch.Tensor:
        out = torch.empty(self.shapes[pid], device=self.device, dtype=torch.float32)
        self._ck(self.L.mer_params_get(self.h, pid, _ptr(out), 1))
        return out

    def set_target(self, pid: int, img):
        t = _dev_f32(img, self.device, self._nimg(pid), "target image")
        self._ck(self.L.mer_target_set(self.h, pid, _ptr(t), 1))
        torch.cuda.current_stream(self.device).synchronize()

    def set_target_host(self, pid: int, img_pinned: torch.Tensor):
        """Target upload from a (pinned) host tensor."""
        _host_buf(img_pinned, torch.float32, self._nimg(pid), "target image")
        self._ck(self.L.mer_target_set(self.h, pid, _ptr(img_pinned), 0))

    def set_target_async(self, pid: int, img_pinned: torch.Tensor):
        """Target upload from a pinned host tensor without waiting; the tensor must stay unchanged
        until the work enqueued so far has completed."""
        _host_buf(img_pinned, torch.float32, self._nimg(pid), "target image")
        self._ck(self.L.mer_target_set_async(self.h, pid, _ptr(img_pinned)))

    def loss_async(self, pid: int, out_pinned: torch.Tensor):
        """Enqueue a copy of the problem's last loss into a pinned float64 host tensor (one element);
        valid once the caller's stream has reached this point (e.g. after an event recorded next)."""
        _host_buf(out_pinned, torch.float64, 1, "loss")
        self._ck(self.L.mer_loss_async(self.h, pid, _ptr(out_pinned)))

    def render_target(self, pid: int, tex, spp: int):
        t = _dev_f32(tex, self.device, self._ntex(pid), "texture")
        self._ck(self.L.mer_target_render(self.h, pid, _ptr(t), spp))
        torch.cuda.current_stream(self.device).synchronize()

    # ---- renders and adjoints ----
    def render(self, pid, tex=None, spp=1, stream=STREAM_EVAL, iteration=0, out=None) -> torch.Tensor:
        H, W = self.images[pid]
        if out is not None:
            _out_f32(out, self.device, H * W * 3, "image")
        t = None if tex is None else _dev_f32(tex, self.device, self._ntex(pid), "texture")
        out = out if out is not None else torch.empty((H, W, 3), device=self.device, dtype=torch.float32)
        self._ck(self.L.mer_render(self.h, pid, _ptr(t), spp, stream, iteration, _ptr(out)))
        return out

    def render_samples(self, pid, tex=None, spp=1, stream=STREAM_EVAL, iteration=0) -> torch.Tensor:
        H, W = self.images[pid]
        t = None if tex is None else _dev_f32(tex, self.device, self._ntex(pid), "texture")
        out = torch.empty((spp, H * W, 3), device=self.device, dtype=torch.float32)
        self._ck(self.L.mer_render_samples(self.h, pid, _ptr(t), spp, stream, iteration, _ptr(out)))
        return out

    def render_pair(self, pid, texA, texB, spp=1, stream=STREAM_FD_PRIMAL, iteration=0):
        H, W = self.images[pid]
        n = self._ntex(pid)
        _need(texA, n, "texture A"), _need(texB, n, "texture B")
        ta, tb = _dev_f32(texA, self.device), _dev_f32(texB, self.device)
        a = torch.empty((H, W, 3), device=self.device, dtype=torch.float32)
        b = torch.empty_like(a)
        self._ck(self.L.mer_render_pair(self.h, pid, _ptr(ta), _ptr(tb), spp, stream, iteration, _ptr(a), _ptr(b)))
        return a, b

    def adjoint(self, pid, tex, dimg, spp=1, stream=STREAM_EVAL, iteration=0) -> torch.Tensor:
        if tex is not None:
            _need(tex, self._ntex(pid), "texture")
        _need(dimg, self._nimg(pid), "adjoint image")
        t = None if tex is None else _dev_f32(tex, self.device)
        d = _dev_f32(dimg, self.device)
        g = torch.empty(self.shapes[pid], device=self.device, dtype=torch.float32)
        self._ck(self.L.mer_adjoint(self.h, pid, _ptr(t), _ptr(d), spp, stream, iteration, _ptr(g)))
        return g

    def adjoint_pair(self, pid, texA, texB, dimgA, dimgB, spp=1, stream=STREAM_FD_ADJ, iteration=0):
        n, m = self._ntex(pid), self._nimg(pid)
        _need(texA, n, "texture A"), _need(texB, n, "texture B")
        _need(dimgA, m, "adjoint image A"), _need(dimgB, m, "adjoint image B")
        ta, tb = _dev_f32(texA, self.device), _dev_f32(texB, self.device)
        da, db = _dev_f32(dimgA, self.device), _dev_f32(dimgB, self.device)
        g = torch.empty(self.shapes[pid], device=self.device, dtype=torch.float32)
        self._ck(self.L.mer_adjoint_pair(self.h, pid, _ptr(ta), _ptr(tb), _ptr(da), _ptr(db), spp, stream, iteration,
                                         _ptr(g)))
        return g

    # ---- optimisation ----
    def gradient_step(self):
        self._ck(self.L.mer_gradient_step(self.h))

    def update_step(self):
        self._ck(self.L.mer_update_step(self.h))

    def iterate(self, n: int = 1, use_graph: bool = True):
        self._ck(self.L.mer_iterate(self.h, n, int(use_graph)))

    def grads(self, pid):
        F = torch.empty(self.shapes[pid], device=self.device, dtype=torch.float32)
        dF = torch.empty_like(F)
        self._ck(self.L.mer_grads_get(self.h, pid, _ptr(F), _ptr(dF), 1))
        return F, dF

    def stats(self, pid) -> dict:
        s = _lib.IterStats()
        self._ck(self.L.mer_stats(self.h, pid, ct.byref(s)))
        return dict(iteration=s.iteration, loss=s.loss, dpi_norm2=s.dpi_norm2, count_f=s.count_f,
                    count_d=s.count_d, paths_per_iter=s.paths_per_iter)

    def state(self, pid) -> dict:
        """Copies of the optimiser state arrays (parameter-shaped)."""
        v = _lib.StateView()
        self._ck(self.L.mer_state_get(self.h, pid, ct.byref(v)))
        out = {}
        for name in ("pi_cur", "pi_prev", "F", "dF", "m2f", "m2d", "mean", "var", "alpha_prev",
                     "mu_f", "mu_d", "adam_m", "adam_v", "F_var", "dF_var"):
            addr = ct.cast(getattr(v, name), ct.c_void_p).value
            if not addr:
                continue            # variant state the problem's flags do not allocate
            t = torch.empty(self.shapes[pid], device=self.device, dtype=torch.float32)
            _memcpy_d2d(t, addr, v.n * 4)
            out[name] = t
        return out

    def profile(self, mode: int = 1):
        """0 off, 1 event timing of every launch, 2 counting of traversal tests."""
        self._ck(self.L.mer_profile_enable(self.h, int(mode)))

    def profile_read(self) -> dict:
        arr = (_lib.KernelTime * 32)()
        n = ct.c_int32()
        self._ck(self.L.mer_profile_read(self.h, arr, 32, ct.byref(n)))
        return {arr[i].name.decode(): dict(launches=arr[i].launches, units=arr[i].units, ms=arr[i].total_ms,
                                           node_tests=arr[i].node_tests, prim_tests=arr[i].prim_tests)
                for i in range(n.value)}

    def launch_count(self) -> int:
        n = ct.c_int64()
        self._ck(self.L.mer_launch_count(self.h, ct.byref(n)))
        return n.value

    def checkpoint_save(self) -> bytes:
        n = ct.c_size_t()
        self._ck(self.L.mer_checkpoint_save(self.h, None, ct.byref(n)))
        buf = ct.create_string_buffer(n.value)
        self._ck(self.L.mer_checkpoint_save(self.h, buf, ct.byref(n)))
        return buf.raw[:n.value]

    def checkpoint_load(self, blob: bytes):
        buf = ct.create_string_buffer(blob, len(blob))
        self._ck(self.L.mer_checkpoint_load(self.h, buf, len(blob)))

    def autotune(self, trial_iters: int = 2) -> str:
        desc = ct.create_string_buffer(256)
        self._ck(self.L.mer_autotune(self.h, trial_iters, desc, 256))
        return desc.value.decode()


def _memcpy_d2d(dst: torch.Tensor, src_addr: int, nbytes: int):
    class _View:
        __cuda_array_interface__ = {"shape": (nbytes // 4,), "typestr": "<f4", "data": (src_addr, False),
                                    "version": 3, "strides": None}
    src = torch.as_tensor(_View(), device=dst.device)
    dst.view(-1).copy_(src)


def meta_step_raw(hyper: HyperParams, pi, pi_next, F, dF, m2f, m2d, mean, var, alpha_prev, C, lo, hi,
                  iteration, count_f, count_d, dpi_norm2, zero_grads=True, out=None):
    """mer_meta_step_raw on torch device tensors; returns the device tensor holding ||dpi||^2."""
    L = _lib.load()
    n = _dev_buf(pi, torch.float32, -1, "pi").numel()
    dev = pi.device
    for name, t in (("pi_next", pi_next), ("F", F), ("dF", dF), ("m2f", m2f), ("m2d", m2d), ("mean", mean),
                    ("var", var), ("alpha_prev", alpha_prev)):
        _dev_buf(t, torch.float32, n, name, dev)
    out = (_dev_buf(out, torch.float64, -1, "out", dev) if out is not None
           else torch.zeros(1, device=dev, dtype=torch.float64))
    lo_a = (ct.c_float * 8)(*([float(x) for x in lo] + [0.0] * (8 - len(lo))))
    hi_a = (ct.c_float * 8)(*([float(x) for x in hi] + [0.0] * (8 - len(hi))))
    h = hyper.to_c()
    check(L.mer_meta_step_raw(ct.byref(h), pi.numel(), C, lo_a, hi_a, _ptr(pi), _ptr(pi_next), _ptr(F), _ptr(dF),
                              _ptr(m2f), _ptr(m2d), _ptr(mean), _ptr(var), _ptr(alpha_prev), iteration, count_f,
                              count_d, float(dpi_norm2), int(zero_grads), _ptr(out), _cur_stream(dev)))
    return out


class Volume:
    """Emissive-absorptive volume (mer_volume_*): render, replay adjoints and FD pairs of voxel
    parameters (torch float32 (nz, ny, nx, 4) on the device: emission RGB, density)."""

    def __init__(self, scene: dict, device: int = 0):
        self.L = _lib.load()
        self.device = torch.device("cuda", device)
        self.cams = np.ascontiguousarray(scene["cameras"], np.float32)
        d = _lib.VolumeDesc()
        d.nx, d.ny, d.nz = scene["nx"], scene["ny"], scene["nz"]
        d.lo = (ct.c_float * 3)(*scene["lo"])
        d.hi = (ct.c_float * 3)(*scene["hi"])
        d.n_views, d.width, d.height = scene["n_views"], scene["width"], scene["height"]
        d.cameras = self.cams.ctypes.data_as(ct.POINTER(ct.c_float))
        d.step = scene["step"]
        d.background = (ct.c_float * 3)(*scene["bg"])
        d.seed, d.key_id = scene["seed"], scene["key_id"]
        h = ct.c_void_p()
        check(self.L.mer_volume_create(ct.byref(d), device, ct.byref(h)))
        self.h = h
        self.shape = (scene["nz"], scene["ny"], scene["nx"], 4)
        self.image_shape = (scene["n_views"], scene["height"], scene["width"], 3)

    def close(self):
        if getattr(self, "h", None):
            self.L.mer_volume_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _nvox(self) -> int:
        return int(np.prod(self.shape))

    def _nimg(self) -> int:
        return int(np.prod(self.image_shape))

    def render(self, params, spp=1, stream=STREAM_EVAL, iteration=0) -> torch.Tensor:
        p = _dev_f32(params, self.device, self._nvox(), "voxel parameters")
        img = torch.empty(self.image_shape, device=self.device, dtype=torch.float32)
        check(self.L.mer_volume_render(self.h, _ptr(p), spp, stream, iteration, _ptr(img), _cur_stream(self.device)))
        return img

    def adjoint(self, params, dimg, spp=1, stream=STREAM_EVAL, iteration=0, grad=None) -> torch.Tensor:
        _need(params, self._nvox(), "voxel parameters"), _need(dimg, self._nimg(), "adjoint images")
        if grad is not None:
            _out_f32(grad, self.device, self._nvox(), "gradient")
        p, d = _dev_f32(params, self.device), _dev_f32(dimg, self.device)
        g = torch.zeros(self.shape, device=self.device, dtype=torch.float32) if grad is None else grad
        check(self.L.mer_volume_adjoint(self.h, _ptr(p), _ptr(d), spp, stream, iteration, _ptr(g),
                                        _cur_stream(self.device)))
        return g

    def adjoint_pair(self, pA, pB, dA, dB, spp=1, stream=STREAM_FD_ADJ, iteration=0, grad=None) -> torch.Tensor:
        nv, ni = self._nvox(), self._nimg()
        _need(pA, nv, "voxel parameters A"), _need(pB, nv, "voxel parameters B")
        _need(dA, ni, "adjoint images A"), _need(dB, ni, "adjoint images B")
        if grad is not None:
            _out_f32(grad, self.device, nv, "gradient")
        a, b = _dev_f32(pA, self.device), _dev_f32(pB, self.device)
        da, db = _dev_f32(dA, self.device), _dev_f32(dB, self.device)
        g = torch.zeros(self.shape, device=self.device, dtype=torch.float32) if grad is None else grad
        check(self.L.mer_volume_adjoint_pair(self.h, _ptr(a), _ptr(b), _ptr(da), _ptr(db), spp, stream, iteration,
                                             _ptr(g), _cur_stream(self.device)))
        return g


class VolumeOptimizer:
    """mer_volume_opt_*: the meta-estimator (or Adam) fitting a Volume's voxels to target images,
    every iteration on the device (one captured graph with use_graph=True)."""

    def __init__(self, vol: Volume, target, init, hyper: HyperParams = None, loss: int = LOSS_L2, spp_f: int = 1,
                 spp_d: int = 1, lo=(0.0, 0.0, 0.0, 0.0), hi=(4.0, 4.0, 4.0, 60.0)):
        self.L = vol.L
        self.vol = vol                          # kept alive: the optimiser borrows its description
        self.device = vol.device
        hyper = hyper or HyperParams()
        _need(target, vol._nimg(), "target images"), _need(init, vol._nvox(), "voxel parameters")
        t, p = _dev_f32(target, self.device), _dev_f32(init, self.device)
        lo_a = (ct.c_float * 4)(*[float(x) for x in lo])
        hi_a = (ct.c_float * 4)(*[float(x) for x in hi])
        h = hyper.to_c()
        out = ct.c_void_p()
        check(self.L.mer_volume_opt_create(vol.h, ct.byref(h), loss, spp_f, spp_d, lo_a, hi_a, _ptr(t), _ptr(p),
                                           ct.byref(out)))
        self.h = out
        self.shape = vol.shape

    def close(self):
        if getattr(self, "h", None):
            self.L.mer_volume_opt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = _dev_f32(params, self.device, int(np.prod(self.shape)), "voxel parameters")
        check(self.L.mer_volume_opt_set_params(self.h, _ptr(p)))

    def iterate(self, n: int = 1, use_graph: bool = True):
        check(self.L.mer_volume_opt_iterate(self.h, n, int(use_graph), _cur_stream(self.device)))

    def stats(self) -> dict:
        s = _lib.IterStats()
        check(self.L.mer_volume_opt_stats(self.h, ct.byref(s)))
        return dict(iteration=s.iteration, loss=s.loss, dpi_norm2=s.dpi_norm2, count_f=s.count_f,
                    count_d=s.count_d, marches_per_iter=s.paths_per_iter)

    def launches(self) -> int:
        n = ct.c_int32()
        check(self.L.mer_volume_opt_launches(self.h, ct.byref(n)))
        return n.value

    def state(self) -> dict:
        """Copies of the optimiser's arrays (voxel-shaped)."""
        v = _lib.StateView()
        check(self.L.mer_volume_opt_state(self.h, ct.byref(v)))
        out = {}
        for name in ("pi_cur", "pi_prev", "F", "dF", "m2f", "m2d", "mean", "var", "alpha_prev",
                     "mu_f", "mu_d", "adam_m", "adam_v", "F_var", "dF_var"):
            addr = ct.cast(getattr(v, name), ct.c_void_p).value
            if not addr:
                continue
            t = torch.empty(self.shape, device=self.device, dtype=torch.float32)
            _memcpy_d2d(t, addr, v.n * 4)
            out[name] = t
        return out

    def params(self) -> torch.Tensor:
        return self.state()["pi_cur"]

def image_loss(img: torch.Tensor, target: torch.Tensor, kind: int = 0):
    """(loss device double tensor, dLoss/dimg) of an RGB image (mer_image_loss)."""
    L = _lib.load()
    img = _dev_buf(img.contiguous(), torch.float32, -3, "image")
    target = _dev_buf(target.contiguous(), torch.float32, img.numel(), "target", img.device)
    if img.numel() % 3:
        raise ValueError("image: RGB values expected (a multiple of 3)")
    dimg = torch.empty_like(img)
    loss = torch.zeros(1, device=img.device, dtype=torch.float64)
    check(L.mer_image_loss(kind, img.numel() // 3, _ptr(img), _ptr(target), _ptr(dimg), _ptr(loss),
                           _cur_stream(img.device)))
    return loss, dimg


def meta_step_raw_ex(hyper: HyperParams, arrays: dict, C, lo, hi, iteration, count_f, count_d, dpi_norm2,
                     zero_grads=True, out=None):
    """mer_meta_step_raw_ex on torch device tensors (dict keys as in mer_update_arrays; absent keys
    are NULL); returns the device tensor holding ||dpi||^2."""
    L = _lib.load()
    n = _dev_buf(arrays["pi"], torch.float32, -1, "pi").numel()
    dev = arrays["pi"].device
    for name, t in arrays.items():
        if name not in {f for f, _ in _lib.UpdateArrays._fields_}:
            raise ValueError(f"unknown update array {name!r}")
        if t is not None:
            _dev_buf(t, torch.float32, n, name, dev)
    out = (_dev_buf(out, torch.float64, -1, "out", dev) if out is not None
           else torch.zeros(1, device=dev, dtype=torch.float64))
    lo_a = (ct.c_float * 8)(*([float(x) for x in lo] + [0.0] * (8 - len(lo))))
    hi_a = (ct.c_float * 8)(*([float(x) for x in hi] + [0.0] * (8 - len(hi))))
    A = _lib.UpdateArrays()
    for name, _ in _lib.UpdateArrays._fields_:
        setattr(A, name, _ptr(arrays.get(name)))
    h = hyper.to_c()
    check(L.mer_meta_step_raw_ex(ct.byref(h), arrays["pi"].numel(), C, lo_a, hi_a, ct.byref(A), iteration, count_f,
                                 count_d, float(dpi_norm2), int(zero_grads), _ptr(out), _cur_stream(dev)))
    return out


def precondition(g: torch.Tensor, lam: float) -> torch.Tensor:
    """(I + lam L)^{-1} applied in place to each channel of an (H, W, C) float32 CUDA gradient
    (mer_precondition); returns g."""
    if g.dim() != 3:
        raise ValueError("precondition: an (H, W, C) tensor expected")
    H, W, C = g.shape
    _dev_buf(g, torch.float32, H * W * C, "precondition: g")
    L = _lib.load()
    check(L.mer_precondition(C, H, W, float(lam), _ptr(g), _cur_stream(g.device)))
    return g


def philox(k0: int, k1: int, ctr: torch.Tensor) -> torch.Tensor:
    """Philox4x32-10 of int32/uint32-bit counters [n, 4] (device) under key (k0, k1)."""
    L = _lib.load()
    ctr = ctr.contiguous()
    if not (ctr.is_cuda and ctr.dim() == 2 and ctr.shape[1] == 4 and ctr.element_size() == 4
            and not ctr.is_floating_point()):
        raise ValueError("ctr: a CUDA tensor of 32-bit integer counters [n, 4] expected")
    out = torch.empty_like(ctr)
    check(L.mer_philox(k0 & 0xFFFFFFFF, k1 & 0xFFFFFFFF, _ptr(ctr), ctr.shape[0], _ptr(out), _cur_stream(ctr.device)))
    return out

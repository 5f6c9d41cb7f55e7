"""ctypes declarations of the C ABI in include/mer.h (argument marshalling only).

Loads paper_2309_15676_gb300/_build/libmer.so and fails loudly if it is missing:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as ct
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmer.so")

MER_OK = 0
ERRORS = {1: "MER_ERR_INVALID_ARG", 2: "MER_ERR_CUDA", 3: "MER_ERR_OOM", 4: "MER_ERR_TIMEOUT",
          5: "MER_ERR_BOUNDS", 6: "MER_ERR_STATE", 7: "MER_ERR_NAN"}
MODE_META, MODE_ADAM = 0, 1
STREAM_PROP_PRIMAL, STREAM_PROP_ADJ, STREAM_FD_PRIMAL, STREAM_FD_ADJ, STREAM_TARGET, STREAM_EVAL = range(6)

_f = ct.c_float
_fp = ct.POINTER(ct.c_float)
_ip = ct.POINTER(ct.c_int32)
_u32p = ct.POINTER(ct.c_uint32)
_vp = ct.c_void_p


class Hyper(ct.Structure):
    _fields_ = [("mode", ct.c_int32), ("lr", _f), ("beta_f", _f), ("beta_d", _f), ("eps", _f),
                ("eps_alpha", _f), ("beta1", _f), ("beta2", _f), ("flags", ct.c_int32), ("precond_lambda", _f)]


class SceneDesc(ct.Structure):
    _fields_ = [
        ("n_verts", ct.c_int32), ("n_tris", ct.c_int32),
        ("positions", _fp), ("uvs", _fp), ("tris", _ip), ("tri_mat", _ip), ("tri_light", _ip),
        ("n_spheres", ct.c_int32), ("spheres", _fp), ("sph_mat", _ip),
        ("n_mats", ct.c_int32), ("mat_type", _ip), ("mat_textured", _ip), ("mat_const", _fp),
        ("n_quads", ct.c_int32), ("quads", _fp),
        ("has_env", ct.c_int32), ("env", _f * 3),
        ("eye", _f * 3), ("target", _f * 3), ("up", _f * 3), ("fov_deg", _f),
        ("width", ct.c_int32), ("height", ct.c_int32),
        ("tex_c", ct.c_int32), ("tex_h", ct.c_int32), ("tex_w", ct.c_int32),
        ("clamp_lo", _f * 8), ("clamp_hi", _f * 8),
        ("max_depth", ct.c_int32), ("spp_prop", ct.c_int32), ("spp_fd", ct.c_int32),
        ("seed", ct.c_uint32), ("key_id", ct.c_uint32),
        ("loss", ct.c_int32),
        ("hyper", Hyper),
    ]


class Config(ct.Structure):
    _fields_ = [("device", ct.c_int32), ("block_size", ct.c_int32), ("blocks_per_sm", ct.c_int32),
                ("smem_nodes", ct.c_int32), ("max_paths", ct.c_int64), ("replay_hit_store", ct.c_int32), ("trace_refill", ct.c_int32)]


class IterStats(ct.Structure):
    _fields_ = [("iteration", ct.c_int64), ("loss", ct.c_double), ("dpi_norm2", ct.c_double),
                ("count_f", ct.c_int32), ("count_d", ct.c_int32), ("paths_per_iter", ct.c_int64)]


class StateView(ct.Structure):
    _fields_ = [(n, _fp) for n in ("pi_cur", "pi_prev", "F", "dF", "m2f", "m2d", "mean", "var", "alpha_prev",
                                   "mu_f", "mu_d", "adam_m", "adam_v", "F_var", "dF_var")] + \
               [("n", ct.c_int64)]


class VolumeDesc(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32), ("lo", _f * 3), ("hi", _f * 3),
                ("n_views", ct.c_int32), ("width", ct.c_int32), ("height", ct.c_int32), ("cameras", _fp),
                ("step", _f), ("background", _f * 3), ("seed", ct.c_uint32), ("key_id", ct.c_uint32)]


class UpdateArrays(ct.Structure):
    _fields_ = [(n, _vp) for n in ("pi", "pi_next", "F", "dF", "m2f", "m2d", "mean", "var", "alpha_prev",
                                   "mu_f", "mu_d", "adam_m", "adam_v", "F_var", "dF_var")]


class KernelTime(ct.Structure):
    _fields_ = [("name", ct.c_char * 32), ("launches", ct.c_int64), ("units", ct.c_int64), ("total_ms", ct.c_double),
                ("node_tests", ct.c_int64), ("prim_tests", ct.c_int64)]


# name -> (restype, argtypes); every symbol mer.h declares
SIGNATURES = {
    "mer_hyper_default": (ct.c_int, [ct.POINTER(Hyper)]),
    "mer_create": (ct.c_int, [ct.POINTER(Config), _vp, ct.POINTER(_vp)]),
    "mer_destroy": (None, [_vp]),
    "mer_last_error": (ct.c_char_p, [_vp]),
    "mer_scene_add": (ct.c_int, [_vp, ct.POINTER(SceneDesc), _ip]),
    "mer_params_set": (ct.c_int, [_vp, ct.c_int32, _vp, ct.c_int32]),
    "mer_params_get": (ct.c_int, [_vp, ct.c_int32, _vp, ct.c_int32]),
    "mer_params_force": (ct.c_int, [_vp, ct.c_int32, _vp, ct.c_int32]),
    "mer_wait_selftest": (ct.c_int, [ct.c_double, ct.POINTER(ct.c_double)]),
    "mer_volume_create": (ct.c_int, [ct.POINTER(VolumeDesc), ct.c_int32, ct.POINTER(_vp)]),
    "mer_volume_destroy": (None, [_vp]),
    "mer_volume_render": (ct.c_int, [_vp, _vp, ct.c_int32, ct.c_uint32, ct.c_uint32, _vp, _vp]),
    "mer_volume_adjoint": (ct.c_int, [_vp, _vp, _vp, ct.c_int32, ct.c_uint32, ct.c_uint32, _vp, _vp]),
    "mer_volume_adjoint_pair": (ct.c_int, [_vp, _vp, _vp, _vp, _vp, ct.c_int32, ct.c_uint32, ct.c_uint32, _vp, _vp]),
    "mer_image_loss": (ct.c_int, [ct.c_int32, ct.c_int64, _vp, _vp, _vp, _vp, _vp]),
    "mer_volume_opt_create": (ct.c_int, [_vp, ct.POINTER(Hyper), ct.c_int32, ct.c_int32, ct.c_int32, _fp, _fp, _vp,
                                         _vp, ct.POINTER(_vp)]),
    "mer_volume_opt_destroy": (None, [_vp]),
    "mer_volume_opt_set_params": (ct.c_int, [_vp, _vp]),
    "mer_volume_opt_iterate": (ct.c_int, [_vp, ct.c_int32, ct.c_int32, _vp]),
    "mer_volume_opt_stats": (ct.c_int, [_vp, ct.POINTER(IterStats)]),
    "mer_volume_opt_state": (ct.c_int, [_vp, ct.POINTER(StateView)]),
    "mer_volume_opt_launches": (ct.c_int, [_vp, ct.POINTER(ct.c_int32)]),
    "mer_target_set": (ct.c_int, [_vp, ct.c_int32, _vp, ct.c_int32]),
    "mer_target_set_async": (ct.c_int, [_vp, ct.c_int32, _vp]),
    "mer_loss_async": (ct.c_int, [_vp, ct.c_int32, _vp]),
    "mer_target_render": (ct.c_int, [_vp, ct.c_int32, _vp, ct.c_int32]),
    "mer_render": (ct.c_int, [_vp, ct.c_int32, _vp, ct.c_int32, ct.c_uint32, ct.c_uint32, _vp]),
    "mer_render_samples": (ct.c_int, [_vp, ct.c_int32, _vp, ct.c_int32, ct.c_uint32, ct.c_uint32, _vp]),
    "mer_adjoint": (ct.c_int, [_vp, ct.c_int32, _vp, _vp, ct.c_int32, ct.c_uint32, ct.c_uint32, _vp]),
    "mer_adjoint_pair": (ct.c_int, [_vp, ct.c_int32, _vp, _vp, _vp, _vp, ct.c_int32, ct.c_uint32, ct.c_uint32, _vp]),
    "mer_render_pair": (ct.c_int, [_vp, ct.c_int32, _vp, _vp, ct.c_int32, ct.c_uint32, ct.c_uint32, _vp, _vp]),
    "mer_gradient_step": (ct.c_int, [_vp]),
    "mer_grads_get": (ct.c_int, [_vp, ct.c_int32, _vp, _vp, ct.c_int32]),
    "mer_update_step": (ct.c_int, [_vp]),
    "mer_iterate": (ct.c_int, [_vp, ct.c_int32, ct.c_int32]),
    "mer_stats": (ct.c_int, [_vp, ct.c_int32, ct.POINTER(IterStats)]),
    "mer_state_get": (ct.c_int, [_vp, ct.c_int32, ct.POINTER(StateView)]),
    "mer_meta_step_raw": (ct.c_int, [ct.POINTER(Hyper), ct.c_int64, ct.c_int32, _fp, _fp, _vp, _vp, _vp, _vp, _vp,
                                     _vp, _vp, _vp, _vp, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_double,
                                     ct.c_int32, _vp, _vp]),
    "mer_meta_step_raw_ex": (ct.c_int, [ct.POINTER(Hyper), ct.c_int64, ct.c_int32, _fp, _fp, ct.POINTER(UpdateArrays),
                                        ct.c_int32, ct.c_int32, ct.c_int32, ct.c_double, ct.c_int32, _vp, _vp]),
    "mer_meta_step_raw_noalloc": (ct.c_int, [ct.POINTER(Hyper), ct.c_int64, ct.c_int32, _fp, _fp, _vp, _vp, _vp,
                                             _vp, _vp, _vp, _vp, _vp, _vp, ct.c_int32, ct.c_int32, ct.c_int32,
                                             ct.c_double, ct.c_int32, _vp, _vp]),
    "mer_philox": (ct.c_int, [ct.c_uint32, ct.c_uint32, _vp, ct.c_int64, _vp, _vp]),
    "mer_precondition": (ct.c_int, [ct.c_int32, ct.c_int32, ct.c_int32, ct.c_float, _vp, _vp]),
    "mer_checkpoint_save": (ct.c_int, [_vp, _vp, ct.POINTER(ct.c_size_t)]),
    "mer_checkpoint_load": (ct.c_int, [_vp, _vp, ct.c_size_t]),
    "mer_autotune": (ct.c_int, [_vp, ct.c_int32, ct.c_char_p, ct.c_size_t]),
    "mer_launch_count": (ct.c_int, [_vp, ct.POINTER(ct.c_int64)]),
    "mer_profile_enable": (ct.c_int, [_vp, ct.c_int32]),
    "mer_profile_read": (ct.c_int, [_vp, ct.POINTER(KernelTime), ct.c_int32, ct.POINTER(ct.c_int32)]),
}

_lib = None


class MerError(RuntimeError):
    pass


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                              "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        L = ct.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status, ctx=None):
    if status != MER_OK:
        msg = load().mer_last_error(ctx).decode(errors="replace")
        raise MerError(f"{ERRORS.get(status, status)}: {msg}")

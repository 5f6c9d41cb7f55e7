"""The C-ABI library loads and exports every entry point include/mer.h declares (no GPU calls)."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mer.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mer_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2309_15676_gb300 import _lib
    return _lib.load()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("mer_create", "mer_scene_add", "mer_render", "mer_adjoint", "mer_gradient_step",
                 "mer_update_step", "mer_meta_step_raw", "mer_iterate", "mer_philox"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(lib):
    from paper_2309_15676_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared()


def test_context_free_errors_without_gpu(lib):
    """Argument validation happens before any device work: bad calls fail with a status and a message."""
    from paper_2309_15676_gb300 import _lib
    h = _lib.Hyper()
    assert lib.mer_hyper_default(ct.byref(h)) == 0 and abs(h.lr - 0.01) < 1e-9 and abs(h.eps_alpha - 1e-30) < 1e-36
    assert lib.mer_meta_step_raw(None, 0, 3, None, None, None, None, None, None, None, None, None, None, None,
                                 0, 0, 0, 0.0, 1, None, None) == 1
    st = lib.mer_philox(0, 0, None, 5, None, None)
    assert st == 1
    assert b"bad arguments" in lib.mer_last_error(None)
    for args in ((0, 4, 4, 1.0), (6, 4, 4, 1.0), (3, 0, 4, 1.0), (3, 4, 4095, 1.0), (3, 4, 4, -1.0),
                 (3, 4, 4, float("nan")), (3, 4, 4, float("inf"))):
        assert lib.mer_precondition(*args, ct.c_void_p(16), None) == 1, args
        assert b"bad arguments to mer_precondition" in lib.mer_last_error(None)


def test_struct_sizes_match_header():
    """ctypes layouts against the C compiler's sizeof (compiled on the host with gcc)."""
    import subprocess
    import tempfile
    from paper_2309_15676_gb300 import _lib
    prog = r'''
#include <stdio.h>
#include "mer.h"
int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(mer_hyper), sizeof(mer_scene_desc),
 sizeof(mer_config), sizeof(mer_iter_stats), sizeof(mer_state_view), sizeof(mer_volume_desc),
 sizeof(mer_update_arrays), sizeof(mer_kernel_time));return 0;}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert sizes == [ct.sizeof(_lib.Hyper), ct.sizeof(_lib.SceneDesc), ct.sizeof(_lib.Config),
                     ct.sizeof(_lib.IterStats), ct.sizeof(_lib.StateView), ct.sizeof(_lib.VolumeDesc),
                     ct.sizeof(_lib.UpdateArrays), ct.sizeof(_lib.KernelTime)]


def test_volume_create_refuses_degenerate_cameras_before_device_work(lib):
    """mer_volume_create validates every camera (eye != target, up not parallel to the view
    direction, field of view in (0, 180) degrees) before any CUDA call, on any machine."""
    from paper_2309_15676_gb300 import _lib
    good = [3.0, 1.0, 2.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 40.0]
    bad = [[0.0, 0.0, 0.0] + good[3:],                              # eye == target
           good[:6] + [-3.0, -1.0, -2.0] + [40.0],                  # up parallel to the view
           good[:9] + [0.0], good[:9] + [180.0], good[:9] + [float("nan")]]
    for cam in bad:
        cams = (ct.c_float * 20)(*(good + cam))                     # the second view is the bad one
        d = _lib.VolumeDesc(nx=4, ny=4, nz=4, n_views=2, width=8, height=8, step=0.5)
        for k in range(3):
            d.lo[k], d.hi[k] = -1.0, 1.0
        d.cameras = ct.cast(cams, _lib._fp)
        out = ct.c_void_p()
        assert lib.mer_volume_create(ct.byref(d), 0, ct.byref(out)) == 1, cam
        assert out.value is None
        assert b"degenerate volume camera" in lib.mer_last_error(None)


def test_a_c99_program_links_and_calls_the_library(lib):
    """The header is plain C: a strict C99 program includes it, links against the built library and
    calls context-free entry points whose argument checks come before any device work."""
    import subprocess
    import tempfile
    from paper_2309_15676_gb300 import _lib
    prog = r'''
#include <stdio.h>
#include <string.h>
#include "mer.h"
int main(void) {
    mer_hyper h;
    memset(&h, 0, sizeof h);
    if (mer_hyper_default(&h) != MER_OK || h.mode != MER_MODE_META) return 1;
    if (mer_hyper_default(NULL) != MER_ERR_INVALID_ARG) return 2;
    if (mer_philox(0u, 0u, NULL, 5, NULL, NULL) != MER_ERR_INVALID_ARG) return 3;
    mer_volume* v = NULL;
    if (mer_volume_create(NULL, 0, &v) != MER_ERR_INVALID_ARG || v != NULL) return 4;
    if (mer_last_error(NULL) == NULL) return 5;
    mer_destroy(NULL);
    printf("ok %s\n", mer_last_error(NULL));
    return 0;
}'''
    libdir = os.path.dirname(_lib.LIB_PATH)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "consumer.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "consumer")
        r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                            os.path.join(ROOT, "include"), c, "-o", exe, "-L", libdir, "-lmer",
                            "-Wl,-rpath," + libdir], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True)
        assert r.returncode == 0 and r.stdout.startswith("ok"), (r.returncode, r.stdout, r.stderr)


def test_binding_constants_match_the_header():
    """Every constant the header defines and the binding (or the oracle's stream ids) repeats has
    the header's value: error codes, modes, stream ids, loss kinds, variant flags, limits."""
    from oracle import orc
    from paper_2309_15676_gb300 import _lib, api
    src = open(os.path.join(ROOT, "include", "mer.h")).read()
    defs = {m.group(1): int(m.group(2), 0) for m in re.finditer(r"#define MER_(\w+)\s+(0x[0-9A-Fa-f]+|\d+)u?\b", src)}
    assert len(defs) >= 30
    checked = 0
    for name, v in defs.items():
        for mod in (api, _lib):
            if hasattr(mod, name):
                assert getattr(mod, name) == v, (name, getattr(mod, name), v)
                checked += 1
    assert checked >= 20
    assert {k: n for k, n in _lib.ERRORS.items()} == {v: "MER_" + k for k, v in defs.items() if k.startswith("ERR_")}
    for s in ("PROP_PRIMAL", "PROP_ADJ", "FD_PRIMAL", "FD_ADJ", "TARGET", "EVAL"):
        assert getattr(orc, "ST_" + s) == defs["STREAM_" + s], s


@pytest.mark.parametrize("field,value,why", [
    ("beta_f", 1.0, b"decays"), ("beta_d", -0.1, b"decays"), ("beta2", 1.5, b"decays"), ("beta1", float("nan"), b"decays"),
    ("lr", -1.0, b"finite"), ("lr", float("nan"), b"finite"), ("eps", float("inf"), b"finite"),
    ("precond_lambda", -2.0, b"finite"), ("mode", 7, b"mode"), ("flags", 1 << 10, b"flag")])
def test_update_refuses_hyper_parameters_it_cannot_run(lib, field, value, why):
    """A decay of 1 would divide the start-up correction by zero; negative or non-finite rates and
    epsilons, unknown modes and flag bits are refused before any device work, by both standalone
    update entry points (and by the scene and volume-optimiser constructors, which share the check)."""
    from paper_2309_15676_gb300 import _lib
    h = _lib.Hyper()
    assert lib.mer_hyper_default(ct.byref(h)) == 0
    setattr(h, field, value)
    lo, hi = (ct.c_float * 8)(), (ct.c_float * 8)(*([1.0] * 8))
    out = ct.c_double()
    st = lib.mer_meta_step_raw(ct.byref(h), 0, 3, lo, hi, None, None, None, None, None, None, None, None, None,
                               0, 0, 0, 0.0, 1, ct.byref(out), None)
    assert st == 1 and why in lib.mer_last_error(None), (st, lib.mer_last_error(None))
    st = lib.mer_meta_step_raw_noalloc(ct.byref(h), 0, 3, lo, hi, None, None, None, None, None, None, None, None,
                                       None, 0, 0, 0, 0.0, 1, ct.byref(out), None)
    assert st == 1 and why in lib.mer_last_error(None), (st, lib.mer_last_error(None))

"""FD pairs with a shared path (MER_META_FD_SHARED_PATH, Eq. est_triv read literally): the
pi_{i-1} branch follows the pi_i path and divides by its densities. The GPU pair (images and
adjoints) and the whole gradient step against the oracle's shared-path branch on the same counters
(per-sample radiance tolerance on the images, image-summed gradient tolerance 1e-3)."""
import numpy as np
import pytest

from oracle import orc
from paper_2309_15676_gb300 import synth

from .gpu_common import frac_within, need_gpu
from .test_gpu_parity import _grad_check

pytestmark = pytest.mark.gpu

SHARED = 64


def test_shared_pair_matches_oracle():
    torch = need_gpu()
    from paper_2309_15676_gb300.api import Context, HyperParams
    w = synth.workload_spiral(40, 32, 64, 16, 32, max_depth=4)
    sc = w.scene
    ctx = Context(0)
    pid = ctx.add_scene(sc, HyperParams(flags=SHARED))
    tA = w.init_tex
    tB = np.clip(w.init_tex + np.random.default_rng(2).normal(0, 0.05, w.init_tex.shape), 0.05, 0.95
                 ).astype(np.float32)
    iA, iB = ctx.render_pair(pid, tA, tB, spp=2, stream=2, iteration=3)
    s = orc.Scene(sc)
    rA = orc.render_image(s, tA, 2, 3, 2)
    rB = orc.render_image_shared(s, tA, tB, 2, 3, 2)
    assert frac_within(iA.cpu().numpy(), rA, 1e-4, 1e-6) > 0.999
    assert frac_within(iB.cpu().numpy(), rB, 1e-4, 1e-6) > 0.999
    rng = np.random.default_rng(3)
    dA = rng.normal(size=rA.shape).astype(np.float32)
    dB = rng.normal(size=rA.shape).astype(np.float32)
    got = ctx.adjoint_pair(pid, tA, tB, dA, dB, spp=2, stream=3, iteration=3).cpu().numpy()
    ref = orc.adjoint_image(s, tA, 2, 3, 3, dA) - orc.adjoint_image_shared(s, tA, tB, 2, 3, 3, dB)
    e, f = _grad_check(got, ref)
    assert e < 1e-3 and f >= 0.999, (e, f)
    ctx.close()


def test_shared_fd_gradient_step_matches_oracle():
    torch = need_gpu()
    from paper_2309_15676_gb300.api import Context, HyperParams
    w = synth.workload_spiral(32, 24, 32, 8, 16, max_depth=3, spp_prop=2, spp_fd=1)
    sc = w.scene
    target = np.random.default_rng(5).uniform(0, 1, (24, 32, 3)).astype(np.float32)
    ctx = Context(0)
    pid = ctx.add_scene(sc, HyperParams(lr=0.03, flags=SHARED))
    ctx.set_target(pid, target)
    ctx.set_params(pid, w.init_tex)
    s = orc.Scene(sc)
    for it in range(3):
        pre = {k: v.cpu().numpy().astype(np.float64) for k, v in ctx.state(pid).items()}
        ctx.gradient_step()
        F, dF = (x.cpu().numpy().astype(np.float64) for x in ctx.grads(pid))
        if it >= 1:
            ref = orc.fd_gradient(s, pre["pi_cur"], pre["pi_prev"], target, 1, it, shared=True)
            e, f = _grad_check(dF, ref)
            assert e < 1e-3 and f > 0.999, (it, e, f)
        ctx.update_step()
    ctx.close()

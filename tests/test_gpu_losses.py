"""The MRSE image loss (step a7 with MER_LOSS_MRSE) through a whole gradient step: loss value,
proportional gradient <F_i> and FD gradient <dF_i> of the GPU against the oracle on the same
counters (image-summed gradient tolerance 1e-3 relative, loss 1e-4)."""
import numpy as np
import pytest

from oracle import orc
from paper_2309_15676_gb300 import synth

from .gpu_common import need_gpu
from .test_gpu_parity import _grad_check

pytestmark = pytest.mark.gpu


def test_mrse_gradient_step_matches_oracle():
    torch = need_gpu()
    from paper_2309_15676_gb300.api import LOSS_MRSE, Context, HyperParams
    w = synth.workload_spiral(32, 24, 32, 8, 16, max_depth=3, spp_prop=2, spp_fd=1)
    sc = dict(w.scene, loss=LOSS_MRSE)
    target = np.random.default_rng(12).uniform(0, 1.5, (24, 32, 3)).astype(np.float32)
    ctx = Context(0)
    pid = ctx.add_scene(sc, HyperParams(lr=0.02))
    ctx.set_target(pid, target)
    ctx.set_params(pid, w.init_tex)
    s = orc.Scene(sc)
    for it in range(2):
        pre = {k: v.cpu().numpy().astype(np.float64) for k, v in ctx.state(pid).items()}
        ctx.gradient_step()
        F, dF = (x.cpu().numpy().astype(np.float64) for x in ctx.grads(pid))
        Fo, loss_o, _ = orc.prop_gradient(s, pre["pi_cur"], target, 2, it, loss_kind=orc.LOSS_MRSE)
        e, f = _grad_check(F, Fo)
        assert e < 1e-3 and f > 0.999, ("F", it, e, f)
        assert abs(ctx.stats(pid)["loss"] - loss_o) <= 1e-4 * loss_o
        if it >= 1:
            dFo = orc.fd_gradient(s, pre["pi_cur"], pre["pi_prev"], target, 1, it, loss_kind=orc.LOSS_MRSE)
            e, f = _grad_check(dF, dFo)
            assert e < 1e-3 and f > 0.999, ("dF", it, e, f)
        ctx.update_step()
    ctx.close()

"""Gradient preconditioning on the GPU (precond_lambda > 0): after a gradient step, F and dF of a
preconditioned problem equal the oracle's (I + lambda L)^{-1} applied to the unpreconditioned
gradients of the same problem on the same counters (relative L2 below 1e-4); and the solve on its
own (mer_precondition) equals the oracle's on random gradients of power-of-two sides (the FFT route,
up to 2048), other sides (the direct route) and mixed shapes, for weak and strong smoothing."""
import numpy as np
import pytest

from oracle import precond
from paper_2309_15676_gb300 import synth

from .gpu_common import need_gpu, params_match, rel_l2

pytestmark = pytest.mark.gpu


def test_preconditioned_gradients_match_oracle():
    torch = need_gpu()
    from paper_2309_15676_gb300.api import Context, HyperParams
    lam = 5.0
    w = synth.workload_spiral(48, 40, 64, 16, 64, max_depth=4, spp_prop=2, spp_fd=1)
    target = np.random.default_rng(3).uniform(0, 1, (40, 48, 3)).astype(np.float32)
    ctxs = []
    for l in (0.0, lam):
        c = Context(0)
        p = c.add_scene(w.scene, HyperParams(lr=0.02, precond_lambda=l))
        c.set_target(p, target)
        c.set_params(p, w.init_tex)
        ctxs.append((c, p))
    pi1 = np.clip(w.init_tex + np.random.default_rng(4).normal(0, 0.01, w.init_tex.shape), 0.05, 0.95).astype(np.float32)
    for it in range(2):
        grads = []
        for c, p in ctxs:
            c.gradient_step()
            grads.append([x.cpu().numpy().astype(np.float64) for x in c.grads(p)])
        (F0, dF0), (Fl, dFl) = grads
        assert np.abs(F0).max() > 0
        assert rel_l2(Fl, precond.precondition(F0, lam)) < 1e-4, it
        if it == 1:
            assert np.abs(dF0).max() > 0
            assert rel_l2(dFl, precond.precondition(dF0, lam)) < 1e-4
        for c, p in ctxs:
            c.update_step()
            c.force_params(p, pi1)      # both problems continue from the same pi_1
    for c, _ in ctxs:
        c.close()


def test_preconditioned_iterations_in_a_graph():
    """The preconditioner's kernels are captured in the iteration graph: graph-launched iterations
    equal plain ones."""
    torch = need_gpu()
    from paper_2309_15676_gb300.api import Context, HyperParams
    w = synth.workload_box(32, 32, 16, max_depth=3)
    target = np.random.default_rng(5).uniform(0, 1, (32, 32, 3)).astype(np.float32)
    out = []
    for graph in (False, True):
        c = Context(0)
        p = c.add_scene(w.scene, HyperParams(lr=0.02, precond_lambda=2.0))
        c.set_target(p, target)
        c.set_params(p, w.init_tex)
        c.iterate(3, use_graph=graph)
        out.append(c.get_params(p).cpu().numpy())
        c.close()
    assert params_match(out[0], out[1])


@pytest.mark.parametrize("C,H,W", [(5, 64, 64), (3, 1024, 1024), (5, 2048, 64), (5, 64, 2048), (3, 5, 7),
                                   (5, 100, 36), (3, 1, 33), (5, 33, 1), (3, 1, 1), (5, 48, 2), (4, 4, 4),
                                   (3, 256, 100)])
@pytest.mark.parametrize("lam", [0.5, 4.0, 100.0])
def test_precondition_standalone_matches_oracle(C, H, W, lam):
    """FP32 transforms of a texture of unit-variance noise: relative L2 error below 1e-5 (a few
    FP32 ulp times the log of the side for the FFT route, the sum length for the direct route)."""
    torch = need_gpu()
    from paper_2309_15676_gb300.api import precondition
    g = np.random.default_rng(C * 7919 + H * 31 + W).normal(size=(H, W, C)).astype(np.float32)
    got = precondition(torch.from_numpy(g).cuda(), lam).cpu().numpy()
    ref = precond.precondition(g.astype(np.float64), lam)
    assert rel_l2(got, ref) < 1e-5, rel_l2(got, ref)

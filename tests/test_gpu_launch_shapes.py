"""Launch shapes change speed, not results: the autotuner leaves the optimisation state as it was
(parameters bit for bit, iteration count), a tuned context continues like an untuned one, and
contexts with other shapes (BVH top levels staged in shared memory, 256-thread blocks, a per-SM
block cap, the traversal refilling its lanes after every finished ray or only when a whole warp is
idle) give the same iterations up to the order of float reductions."""
import numpy as np
import pytest

from paper_2309_15676_gb300 import synth

from .gpu_common import need_gpu, params_match, rel_l2

pytestmark = pytest.mark.gpu


def _setup(ctx, w, target):
    from paper_2309_15676_gb300.api import HyperParams
    pid = ctx.add_scene(w.scene, HyperParams(lr=0.02))
    ctx.set_target(pid, target)
    ctx.set_params(pid, w.init_tex)
    return pid


def test_autotune_keeps_state_and_results():
    need_gpu()
    from paper_2309_15676_gb300.api import Context
    w = synth.workload_spiral(48, 40, 64, 16, 32, max_depth=4)
    target = np.random.default_rng(5).uniform(0.1, 0.8, (40, 48, 3)).astype(np.float32)
    a, b = Context(0), Context(0)
    pa, pb = _setup(a, w, target), _setup(b, w, target)
    a.iterate(2, use_graph=True)
    b.iterate(2, use_graph=True)
    before = a.get_params(pa).cpu().numpy().copy()
    it = a.stats(pa)["iteration"]
    desc = a.autotune(2)
    assert isinstance(desc, str) and desc
    assert np.array_equal(a.get_params(pa).cpu().numpy(), before) and a.stats(pa)["iteration"] == it
    a.iterate(2, use_graph=True)
    b.iterate(2, use_graph=True)
    assert params_match(a.get_params(pa).cpu().numpy(), b.get_params(pb).cpu().numpy())
    a.close()
    b.close()


@pytest.mark.parametrize("shape", [dict(smem_nodes=128), dict(block_size=256), dict(blocks_per_sm=2),
                                   dict(trace_refill=1), dict(trace_refill=32)])
def test_launch_shapes_give_the_same_iterations(shape):
    need_gpu()
    from paper_2309_15676_gb300.api import Context
    w = synth.workload_spiral(48, 40, 64, 16, 32, max_depth=4)
    target = np.random.default_rng(6).uniform(0.1, 0.8, (40, 48, 3)).astype(np.float32)
    out = []
    for kw in ({}, shape):
        ctx = Context(0, **kw)
        pid = _setup(ctx, w, target)
        ctx.iterate(2, use_graph=True)
        ctx.gradient_step()
        F, dF = (x.cpu().numpy().astype(np.float64) for x in ctx.grads(pid))
        out.append((F, dF, ctx.get_params(pid).cpu().numpy()))
        ctx.close()
    (Fa, dFa, pa), (Fb, dFb, pb) = out
    assert np.abs(Fa).max() > 0
    assert rel_l2(Fb, Fa) < 1e-5 and rel_l2(dFb, dFa) < 1e-5, (rel_l2(Fb, Fa), rel_l2(dFb, dFa))
    assert params_match(pa, pb)


@pytest.mark.parametrize("shape", [dict(block_size=256, blocks_per_sm=1), dict(blocks_per_sm=2), dict(trace_refill=32)])
def test_per_sample_radiance_is_bit_identical_across_launch_shapes(shape):
    """Each path's radiance is accumulated by one thread per depth, so only the hits could make
    it depend on the launch shape. The shape decides which lanes take which rays and, once the
    rays of a launch are all taken, which idle lanes walk which deferred subtrees for which owner;
    the nearest hit (ties to the smaller primitive id) and the any-hit answer must not change, so
    every sample of a render (closest hits and shadow rays) and of an FD render pair is the same
    bit for bit."""
    torch = need_gpu()
    from paper_2309_15676_gb300.api import Context
    w = synth.workload_spiral(64, 48, 64, 16, 32, max_depth=5)
    tex = torch.from_numpy(w.init_tex).cuda()
    tex_b = torch.from_numpy(np.clip(w.init_tex + 0.05, 0.0, 1.0).astype(np.float32)).cuda()
    out = []
    for kw in ({}, shape):
        ctx = Context(0, **kw)
        pid = ctx.add_scene(w.scene)
        s = ctx.render_samples(pid, tex, spp=6, stream=5, iteration=3).cpu().numpy()
        a, b = ctx.render_pair(pid, tex, tex_b, spp=3, iteration=3)
        out.append((s, a.cpu().numpy(), b.cpu().numpy()))
        ctx.close()
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)


def test_tiny_launches_match_the_oracle():
    """A 6 x 5 image: every traversal launch holds fewer rays than a block has lanes, so nearly
    every walk is shared among helper lanes; the samples still match the oracle."""
    torch = need_gpu()
    from oracle import orc
    from paper_2309_15676_gb300.api import Context
    w = synth.workload_spiral(6, 5, 64, 16, 32, max_depth=5)
    ctx = Context(0)
    pid = ctx.add_scene(w.scene)
    spp = 8
    got = ctx.render_samples(pid, torch.from_numpy(w.init_tex).cuda(), spp=spp, stream=5, iteration=1).cpu().numpy()
    ctx.close()
    npix = 30
    idx = np.arange(spp * npix)
    ref = orc.render_samples(orc.Scene(w.scene), w.init_tex, idx % npix, idx // npix, 1, 5)
    got = got.reshape(spp * npix, 3)
    ok = np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + 1e-6, axis=1)
    assert ok.all(), np.argwhere(~ok)

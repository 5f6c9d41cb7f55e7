"""Edge cases of the path tracer and the iteration against the oracle: the depth extremes (1:
emitters only, so every texture gradient is exactly zero; 2: direct light only; 16: the largest
depth the library accepts, deep queues, re-tracing replays and the hit-store variant), a ragged image far from the 16x16 tiling
(7 x 5 pixels) with a 2 x 2 texture (bilinear clamp-to-edge on every fetch), and one-pixel images.
Tolerances as elsewhere: >= 99.99% of per-sample radiances within 1e-4 relative (floor 1e-6),
image-summed gradients within 1e-3 relative L2."""
import numpy as np
import pytest

from oracle import orc
from paper_2309_15676_gb300 import synth

from .gpu_common import need_gpu
from .test_gpu_parity import _grad_check, _sample_parity

pytestmark = pytest.mark.gpu


def _ctx(scene):
    from paper_2309_15676_gb300.api import Context, HyperParams
    ctx = Context(0)
    return ctx, ctx.add_scene(scene, HyperParams(lr=0.02))


@pytest.mark.parametrize("depth", [1, 2, 16])
def test_depth_extremes(depth):
    need_gpu()
    w = synth.workload_box(16, 16, 8, max_depth=depth)
    sc = w.scene
    ctx, pid = _ctx(sc)
    frac, n = _sample_parity(ctx, pid, sc, w.init_tex, 4, 0, 3)
    assert frac >= 0.9999, (depth, frac, n)
    dimg = np.random.default_rng(4).normal(size=(16, 16, 3)).astype(np.float32)
    got = ctx.adjoint(pid, w.init_tex, dimg, spp=2, stream=1, iteration=2).cpu().numpy()
    if depth == 1:          # emitters only: the albedo never enters the radiance
        assert np.all(got == 0.0)
    else:
        ref = orc.adjoint_image(orc.Scene(sc), w.init_tex, 2, 2, 1, dimg)
        e, f = _grad_check(got, ref)
        assert e < 1e-3 and f >= 0.999, (depth, e, f)
    ctx.close()
    # whole iterations (re-tracing replays, and the hit-store variant; FD pairs) run and stay finite
    from paper_2309_15676_gb300.api import Context, HyperParams
    for hit_store in (False, True):
        ctx = Context(0, replay_hit_store=hit_store)
        pid = ctx.add_scene(sc, HyperParams(lr=0.02))
        ctx.set_target(pid, np.full((16, 16, 3), 0.3, np.float32))
        ctx.set_params(pid, w.init_tex)
        ctx.iterate(3, use_graph=True)
        st = ctx.stats(pid)
        assert st["iteration"] == 3 and np.isfinite(st["loss"])
        assert np.all(np.isfinite(ctx.get_params(pid).cpu().numpy()))
        ctx.close()


@pytest.mark.parametrize("size", [(7, 5), (1, 1)])
def test_ragged_image_and_two_texel_texture(size):
    need_gpu()
    wdt, hgt = size
    w = synth.workload_spiral(wdt, hgt, 32, 8, 2, max_depth=4)
    sc = w.scene
    ctx, pid = _ctx(sc)
    frac, n = _sample_parity(ctx, pid, sc, w.init_tex, 16, 0, 5)
    assert frac >= 0.9999, (size, frac, n)
    dimg = np.random.default_rng(6).normal(size=(hgt, wdt, 3)).astype(np.float32)
    got = ctx.adjoint(pid, w.init_tex, dimg, spp=8, stream=1, iteration=5).cpu().numpy()
    ref = orc.adjoint_image(orc.Scene(sc), w.init_tex, 8, 5, 1, dimg)
    if np.abs(ref).max() > 0:
        e, f = _grad_check(got, ref)
        assert e < 1e-3 and f >= 0.999, (size, e, f)
    else:
        assert np.abs(got).max() == 0.0
    ctx.close()


def test_context_at_its_problem_limit():
    """MER_MAX_PROBLEMS (256) tiny problems in one context: a 257th is refused, and the first and the
    last problem's gradients in the full batch equal the same problem's alone."""
    torch = need_gpu()
    from paper_2309_15676_gb300._lib import MerError
    from paper_2309_15676_gb300.api import Context, HyperParams
    ws = [synth.workload_box(8, 8, 4, max_depth=2, key_id=k) for k in range(256)]
    tgt = np.full((8, 8, 3), 0.3, np.float32)
    ctx = Context(0)
    ids = []
    for w in ws:
        p = ctx.add_scene(w.scene, HyperParams())
        ctx.set_target(p, tgt)
        ctx.set_params(p, w.init_tex)
        ids.append(p)
    with pytest.raises(MerError):
        ctx.add_scene(ws[0].scene, HyperParams())
    ctx.iterate(1, use_graph=True)
    ctx.gradient_step()
    batched = {q: ctx.grads(ids[q])[0].cpu().numpy().astype(np.float64) for q in (0, 255)}
    ctx.close()
    for q, F in batched.items():
        c1 = Context(0)
        p1 = c1.add_scene(ws[q].scene, HyperParams())
        c1.set_target(p1, tgt)
        c1.set_params(p1, ws[q].init_tex)
        c1.iterate(1, use_graph=True)
        c1.gradient_step()
        F1 = c1.grads(p1)[0].cpu().numpy().astype(np.float64)
        c1.close()
        assert np.abs(F1).max() > 0
        assert np.linalg.norm(F - F1) <= 1e-5 * np.linalg.norm(F1), q

"""Parity at the full sizes of the third, fourth and fifth configurations, in the launch
configuration the benchmark uses, on outputs the oracle computes one by one:
- per-sample radiance of randomly chosen paths of the 512^2 / 32,768-triangle spiral (depth 8) and
  of the 1024^2 / 204,800-triangle displaced sphere (depth 8, 2048^2 x 5 textures);
- full-size adjoints whose loss adjoint is non-zero only at a few hundred randomly chosen pixels,
  against the oracle's per-path replay of exactly those samples (image-summed gradient tolerance);
- the 64-problem batch (images, meshes, textures and depths of uneven sizes, images shrunk 4x):
  sampled radiance of several problems inside the batched context, and their gradient step in the
  batch against each problem alone.
Tolerances as elsewhere: >= 99.9% of sampled radiances within 1e-4 relative (floor 1e-6), relative
L2 of image-summed gradients below 1e-3."""
import numpy as np
import pytest

from oracle import orc
from paper_2309_15676_gb300 import synth

from .gpu_common import need_gpu, rel_l2
from .test_gpu_parity import _grad_check, _sample_parity

pytestmark = pytest.mark.gpu


def _ctx(scene):
    from paper_2309_15676_gb300.api import Context, HyperParams
    ctx = Context(0, max_paths=1 << 20)
    return ctx, ctx.add_scene(scene, HyperParams())


@pytest.mark.parametrize("which", ["spiral512", "dsphere1024"])
def test_full_size_radiance_sampled(which):
    need_gpu()
    w = synth.workload_spiral(512, 512, 512, 32, 1024, max_depth=8) if which == "spiral512" else synth.workload_sphere()
    ctx, pid = _ctx(w.scene)
    frac, n = _sample_parity(ctx, pid, w.scene, w.init_tex, 1, 0, 11, max_ref=1500 if which == "dsphere1024" else 2000,
                             seed=5)
    ctx.close()
    assert frac >= 0.999, (which, frac, n)


@pytest.mark.parametrize("which,npix,spp", [("spiral256", 300, 2), ("dsphere1024", 100, 1)])
def test_full_size_adjoint_sparse_loss(which, npix, spp):
    need_gpu()
    w = synth.workload_spiral() if which == "spiral256" else synth.workload_sphere()
    sc = w.scene
    H, W = sc["height"], sc["width"]
    rng = np.random.default_rng(17)
    pix = np.sort(rng.choice(H * W, npix, replace=False))
    dimg = np.zeros((H * W, 3), np.float32)
    dimg[pix] = rng.normal(size=(npix, 3)).astype(np.float32)
    ctx, pid = _ctx(sc)
    got = ctx.adjoint(pid, w.init_tex, dimg.reshape(H, W, 3), spp=spp, stream=1, iteration=9).cpu().numpy()
    ctx.close()
    pixels = np.repeat(pix, spp).astype(np.uint32)
    samples = np.tile(np.arange(spp), npix).astype(np.uint32)
    adj = dimg[pixels].astype(np.float64) / spp
    ref = orc.adjoint_samples(orc.Scene(sc), w.init_tex, pixels, samples, 9, 1, adj)
    assert np.abs(ref).max() > 0
    e, f = _grad_check(got, ref)
    assert e < 1e-3 and f > 0.999, (which, e, f)


def test_batch_of_64_problems():
    need_gpu()
    from paper_2309_15676_gb300.api import Context, HyperParams
    ws = synth.workload_batch(64, seed=4, scale=0.25)
    ctx = Context(0, max_paths=1 << 20)
    ids = []
    rng = np.random.default_rng(23)
    targets = []
    for w in ws:
        p = ctx.add_scene(w.scene, HyperParams())
        t = rng.uniform(0, 1, (w.scene["height"], w.scene["width"], 3)).astype(np.float32)
        ctx.set_target(p, t)
        ctx.set_params(p, w.init_tex)
        ids.append(p)
        targets.append(t)
    # sampled radiance of a few problems of different kinds inside the batched context
    for q in (0, 17, 40, 63):
        frac, n = _sample_parity(ctx, ids[q], ws[q].scene, ws[q].init_tex, 1, 0, 5, max_ref=300, seed=q)
        assert frac >= 0.999, (q, frac, n)
    # the batched gradient step equals each problem alone
    ctx.iterate(1, use_graph=True)
    ctx.gradient_step()
    batched = {q: [x.cpu().numpy().astype(np.float64) for x in ctx.grads(ids[q])] for q in (3, 29, 51)}
    ctx.close()
    for q, (F, dF) in batched.items():
        c1 = Context(0, max_paths=1 << 20)
        p1 = c1.add_scene(ws[q].scene, HyperParams())
        c1.set_target(p1, targets[q])
        c1.set_params(p1, ws[q].init_tex)
        c1.iterate(1, use_graph=True)
        c1.gradient_step()
        F1, dF1 = (x.cpu().numpy().astype(np.float64) for x in c1.grads(p1))
        c1.close()
        assert np.abs(F1).max() > 0
        assert rel_l2(F, F1) < 1e-4 and rel_l2(dF, dF1) < 1e-3, (q, rel_l2(F, F1), rel_l2(dF, dF1))

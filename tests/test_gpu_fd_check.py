"""Differentiation check on the 512x512 / 32,768-triangle / 1024^2 x 5 spiral at depth 8: the
path-replay adjoint against central finite differences of the GPU's own render with common random
numbers (the third configuration's check).

Base colour does not steer the sampling (the diffuse weight and Schlick F0 are linear in it; the
lobe choice, the GGX sample and every pdf are independent of it), so per seed the adjoint equals the
finite difference of the same-seed render: checked on 64 random texels, h = 1e-3.

Metalness sets the lobe-selection probability (1 + m) / 2 and roughness shapes the GGX sample, so
both enter the sample directions, the mixture pdf and the MIS weights. The detached-sampling
adjoint then equals the derivative of the expected image only in expectation, while the same-seed
finite difference also picks up the samples that cross a lobe boundary or a visibility edge. For
those two channels the mean over 64 seeds of the paired difference (adjoint minus same-seed finite
difference, h = 5e-3) is checked to be zero within 5 standard errors at the texels with the largest
gradient.
"""
import numpy as np
import pytest

from paper_2309_15676_gb300 import synth

from .gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def _setup(torch):
    from paper_2309_15676_gb300.api import Context, HyperParams
    w = synth.workload_spiral(512, 512, 512, 32, 1024, max_depth=8)
    ctx = Context(0)
    pid = ctx.add_scene(w.scene, HyperParams())
    tex = torch.from_numpy(w.init_tex).cuda()
    rng = np.random.default_rng(8)
    dimg = torch.from_numpy(rng.normal(size=(512, 512, 3)).astype(np.float32)).cuda()
    return ctx, pid, tex, dimg, rng


def _central_fd(ctx, pid, tex, dimg, spp, stream, it, y, x, c, h):
    def J(t):
        img = ctx.render(pid, t, spp=spp, stream=stream, iteration=it)
        return float((img.double() * dimg.double()).sum())
    tp, tm = tex.clone(), tex.clone()
    tp[y, x, c] += h
    tm[y, x, c] -= h
    return (J(tp) - J(tm)) / (2 * h)


def test_adjoint_vs_central_fd_base_colour_per_seed():
    torch = need_gpu()
    ctx, pid, tex, dimg, rng = _setup(torch)
    spp, stream, it = 1, 5, 2
    g = ctx.adjoint(pid, tex, dimg, spp=spp, stream=stream, iteration=it).cpu().numpy()
    # 64 random texels among those that receive gradient
    mag = np.abs(g[..., :3]).sum(-1)
    cand = np.argwhere(mag > np.quantile(mag[mag > 0], 0.5))
    pick = cand[rng.choice(len(cand), 64, replace=False)]
    rows = []
    for (y, x) in pick:
        for c in range(3):
            rows.append((g[y, x, c], _central_fd(ctx, pid, tex, dimg, spp, stream, it, y, x, c, 1e-3)))
    ctx.close()
    rows = np.array(rows)
    scale = np.abs(rows[:, 1]).max()
    ok = np.abs(rows[:, 0] - rows[:, 1]) <= 1e-2 * np.abs(rows[:, 1]) + 1e-4 * scale
    assert ok.mean() >= 0.95, ok.mean()


def test_adjoint_vs_central_fd_metal_rough_in_expectation():
    torch = need_gpu()
    ctx, pid, tex, dimg, _ = _setup(torch)
    stream, n, h = 5, 64, 5e-3
    g16 = ctx.adjoint(pid, tex, dimg, spp=16, stream=stream, iteration=1).cpu().numpy()
    cases = []
    for c in (3, 4):
        top = np.argsort(-np.abs(g16[..., c]).ravel())[:4]
        ys, xs = np.unravel_index(top, g16.shape[:2])
        cases += [(int(y), int(x), c) for y, x in zip(ys, xs)]
    a = np.zeros((n, len(cases)))
    b = np.zeros((n, len(cases)))
    for s in range(n):
        it = 100 + s
        g = ctx.adjoint(pid, tex, dimg, spp=1, stream=stream, iteration=it).cpu().numpy()
        for k, (y, x, c) in enumerate(cases):
            a[s, k] = g[y, x, c]
            b[s, k] = _central_fd(ctx, pid, tex, dimg, 1, stream, it, y, x, c, h)
    ctx.close()
    # same seeds on both sides: the paired difference has the smaller spread
    d = a - b
    se = d.std(0, ddof=1) / np.sqrt(n)
    z = d.mean(0) / np.maximum(se, 1e-12)
    assert np.all(np.abs(z) < 5), (cases, a.mean(0), b.mean(0), se)
    # the pooled statistic stays near its chi-square mean of 1 per case
    assert np.mean(z * z) < 4, z

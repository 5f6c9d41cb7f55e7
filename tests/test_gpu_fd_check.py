"""Differentiation check on the 512x512 / 32,768-triangle / 1024^2 x 5 spiral at depth 8: the
path-replay adjoint against central finite differences of the GPU's own render with common random
numbers (the third configuration's check).

Base colour does not steer the sampling (the diffuse weight and Schlick F0 are linear in it; the
lobe choice, the GGX sample and every pdf are independent of it), so per seed the adjoint equals the
finite difference of the same-seed render. Checked against the FP64 oracle's central differences
(h = 1e-5) of the same-seed objective J = sum of dimg . I over 200 sampled pixels, at the 16 texels
with the largest gradient and all three colour channels, within 1e-3 relative (the image-summed
gradient tolerance), every value; and against the GPU's own render with common random numbers on the
full image, where the FP32 rounding of the two renders bounds the finite difference (see that
test).

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


def test_adjoint_vs_oracle_central_fd_base_colour_per_seed():
    torch = need_gpu()
    from .oracle_pool import OraclePool
    w = synth.workload_spiral(512, 512, 512, 32, 1024, max_depth=8)
    from paper_2309_15676_gb300.api import Context, HyperParams
    ctx = Context(0)
    pid = ctx.add_scene(w.scene, HyperParams())
    rng = np.random.default_rng(8)
    H, W = 512, 512
    pix = np.sort(rng.choice(H * W, 200, replace=False)).astype(np.uint32)
    dimg = np.zeros((H * W, 3), np.float32)
    dimg[pix] = rng.normal(size=(len(pix), 3)).astype(np.float32)
    stream, it = 5, 2
    g = ctx.adjoint(pid, w.init_tex, dimg.reshape(H, W, 3), spp=1, stream=stream, iteration=it).cpu().numpy()
    ctx.close()
    g = g.astype(np.float64)
    mag = np.abs(g[..., :3]).sum(-1)
    top = np.argsort(-mag.ravel())[:16]
    ys, xs = np.unravel_index(top, mag.shape)
    d64 = dimg[pix].astype(np.float64)
    zeros = np.zeros(len(pix), np.uint32)
    h = 1e-5
    rows = []
    with OraclePool(w.scene, w.init_tex) as op:
        J = lambda pert: float((op.render_samples(pix, zeros, it, stream, pert) * d64).sum())
        for y, x in zip(ys, xs):
            for c in range(3):
                fd = (J((int(y), int(x), c, h)) - J((int(y), int(x), c, -h))) / (2 * h)
                rows.append((g[y, x, c], fd))
    rows = np.array(rows)
    scale = np.abs(rows[:, 1]).max()
    assert scale > 0
    err = np.abs(rows[:, 0] - rows[:, 1])
    ok = err <= 1e-3 * np.abs(rows[:, 1]) + 1e-5 * scale
    assert ok.all(), rows[~ok]


def test_adjoint_vs_gpu_central_fd_base_colour_per_seed():
    """The same check against the GPU's own full-image render with common random numbers (h = 1e-2;
    base colour enters a path's radiance as a polynomial, so central differences carry no
    truncation error for the paths that touch the texel once). The two renders round every touched
    pixel's radiance in FP32: with at most 2^-20 |I_p| of error per pixel (a few ulp through the
    path's arithmetic), the finite difference is off by at most sum_p |dimg_p| 2^-20 |I_p| / h over
    the pixels whose radiance moved; the adjoint must be within that bound plus 1e-3 relative."""
    torch = need_gpu()
    ctx, pid, tex, dimg, rng = _setup(torch)
    spp, stream, it = 1, 5, 2
    g = ctx.adjoint(pid, tex, dimg, spp=spp, stream=stream, iteration=it).cpu().numpy()
    mag = np.abs(g[..., :3]).sum(-1)
    cand = np.argwhere(mag > np.quantile(mag[mag > 0], 0.5))
    pick = cand[rng.choice(len(cand), 32, replace=False)]
    h = 1e-2
    dd = dimg.double()
    for (y, x) in pick:
        for c in range(3):
            tp, tm = tex.clone(), tex.clone()
            tp[y, x, c] += h
            tm[y, x, c] -= h
            ip = ctx.render(pid, tp, spp=spp, stream=stream, iteration=it).double()
            im = ctx.render(pid, tm, spp=spp, stream=stream, iteration=it).double()
            fd = float(((ip - im) * dd).sum()) / (2 * h)
            moved = (ip != im).any(-1)
            bound = float((dd.abs() * 2.0 ** -20 * (ip.abs() + im.abs()) / 2)[moved].sum()) / h
            assert abs(g[y, x, c] - fd) <= 1e-3 * abs(fd) + bound, (y, x, c, g[y, x, c], fd, bound)
    ctx.close()


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

"""The validation experiments of Sec. 3 and Sec. 6 against the oracle, step by step.

- Prescribed trajectory ("variance reduction without lag", "approximation accuracy"): eight
  independent runs of a small box scene (8x8 image, 8x8 RGB albedo, depth 3, 1 FD + 1 proportional
  spp), the parameters moved along a fixed schedule by mer_params_force after every update. At every
  iteration the GPU's F and dF equal the oracle's gradients of the same run at the same parameters
  (image-summed tolerance, 1e-3 relative L2); the GPU's update (Moment2s, meta-estimate, alpha,
  variance, step) equals the oracle's on identical inputs (1e-5 of the magnitude of its terms); and
  the norm of the forced step that the device recomputes equals the schedule's.
- The exposition toy (Sec. 3, the exponential-rate figure): the rate lambda of an exponential
  distribution is optimised so that the mean of its samples matches 2 (optimum 0.5), one toy run per
  parameter element (per-element step norms keep the runs independent), through the standalone
  fused update with seeded sample gradients computed from the GPU's current rates. Every step equals
  the oracle's on identical inputs; the GPU trajectory follows the oracle's own FP64 trajectory of
  the same samples; both converge to 0.5 - for the meta-estimator and for Adam.
"""
import numpy as np
import pytest

from oracle import meta, orc
from paper_2309_15676_gb300 import synth

from .gpu_common import need_gpu, rel_l2

pytestmark = pytest.mark.gpu


def _update_close(pre, post, F, dF, H, n2, it, lo, hi, flags=0, pi_prev=None):
    """The GPU's update outputs `post` against the oracle's meta_update on the GPU's own inputs."""
    ost = meta.MetaState(pre["m2f"].copy(), pre["m2d"].copy(), pre["mean"].copy(), pre["var"].copy(),
                         pre["alpha_prev"].copy(), pre["count_f"], pre["count_d"], it)
    ref_pi, ref_n2, alpha = meta.meta_update(pre["pi"], F, dF, ost, H, n2, lo, hi, flags=flags, pi_prev=pi_prev)
    assert np.allclose(post["m2f"], ost.m2f, rtol=1e-5, atol=0)
    assert np.allclose(post["m2d"], ost.m2d, rtol=1e-5, atol=0)
    assert np.allclose(post["var"], ost.var, rtol=1e-5, atol=0)
    have_fd = it >= 1 and n2 > 0
    scale_mean = np.abs(pre["mean"] + (dF if have_fd else 0.0)) + np.abs(F)
    assert np.all(np.abs(post["mean"] - ost.mean) <= 1e-5 * scale_mean + 1e-30)
    assert np.all(np.abs(post["alpha_prev"] - alpha) <= 1e-5 * np.abs(alpha) + 1e-7)
    step_scale = H.lr * scale_mean / (np.sqrt(ost.var) + H.eps)
    assert np.all(np.abs(post["pi"] - ref_pi) <= 1e-5 * step_scale + 2 ** -23 * np.abs(pre["pi"]) + 1e-12)
    return ref_pi, ref_n2, alpha


def test_prescribed_trajectory_matches_oracle_step_by_step():
    torch = need_gpu()
    from paper_2309_15676_gb300.api import Context, HyperParams
    runs, iters = 8, 10
    w = synth.workload_box(8, 8, 8, max_depth=3)
    sc0 = w.scene
    init, tgt = w.init_tex.astype(np.float32), w.target_tex.astype(np.float32)
    path = [init + (tgt - init) * np.float32(k / iters) for k in range(iters + 1)]
    target = orc.render_image(orc.Scene(sc0), tgt, 64, 0, orc.ST_TARGET).astype(np.float32)
    H = meta.Hyper(lr=float(np.float32(0.01)), beta_f=float(np.float32(0.99)), beta_d=float(np.float32(0.9)))
    lo = np.asarray(sc0["clamp_lo"], np.float64)[None, None, :]
    hi = np.asarray(sc0["clamp_hi"], np.float64)[None, None, :]
    ctx = Context(0)
    ids, scenes = [], []
    for r in range(runs):
        sc = dict(sc0)
        sc["key_id"] = 1 + r
        p = ctx.add_scene(sc, HyperParams(lr=0.01))
        ctx.set_target(p, target)
        ctx.set_params(p, path[0])
        ids.append(p)
        scenes.append(orc.Scene(sc))
    for k in range(iters):
        pre = {}
        for p in ids:
            s = {n: v.cpu().numpy().astype(np.float64) for n, v in ctx.state(p).items()}
            st = ctx.stats(p)
            pre[p] = dict(s, pi=s["pi_cur"], count_f=st["count_f"], count_d=st["count_d"], n2=st["dpi_norm2"])
        ctx.gradient_step()
        grads = {p: [x.cpu().numpy().astype(np.float64) for x in ctx.grads(p)] for p in ids}
        ctx.update_step()
        for p, sco in zip(ids, scenes):
            F, dF = grads[p]
            Fo, _, _ = orc.prop_gradient(sco, pre[p]["pi"], target, 1, k)
            assert np.abs(Fo).max() > 0
            assert rel_l2(F, Fo) < 1e-3, (k, p, rel_l2(F, Fo))
            if k >= 1:
                dFo = orc.fd_gradient(sco, pre[p]["pi"], pre[p]["pi_prev"], target, 1, k)
                assert rel_l2(dF, dFo) < 1e-3, (k, p, rel_l2(dF, dFo))
            else:
                assert np.all(dF == 0)
            s = {n: v.cpu().numpy().astype(np.float64) for n, v in ctx.state(p).items()}
            post = dict(s, pi=s["pi_cur"])
            _update_close(pre[p], post, F, dF, H, pre[p]["n2"], k, lo, hi)
        if k < iters - 1:
            for p in ids:
                ctx.force_params(p, path[k + 1])
            want = float(((path[k + 1].astype(np.float64) - path[k].astype(np.float64)) ** 2).sum())
            for p in ids:
                got = ctx.stats(p)["dpi_norm2"]
                assert abs(got - want) <= 1e-6 * want, (k, got, want)
    ctx.close()


def _toy_grad(lam, u, v):
    """Per run: 2 (mean(y) - 2) mean(d x / d lambda), y = -ln(1 - v) / lambda the residual's
    independent samples, x = -ln(1 - u) / lambda the samples the gradient is taken of."""
    y = -np.log1p(-v) / lam[:, None]
    return 2.0 * (y.mean(1) - 2.0) * np.mean(np.log1p(-u) / (lam[:, None] ** 2), axis=1)


@pytest.mark.parametrize("mode", ["meta", "adam"])
def test_exposition_toy_gpu_matches_oracle(mode):
    torch = need_gpu()
    from paper_2309_15676_gb300.api import HyperParams, MODE_ADAM, MODE_META, META_PER_ELEMENT, meta_step_raw
    R, iters, S = 2048, 300, 32
    rng = np.random.default_rng(6)
    hp = HyperParams(mode=MODE_META if mode == "meta" else MODE_ADAM, lr=0.02, beta_f=0.99, beta_d=0.9,
                     flags=META_PER_ELEMENT if mode == "meta" else 0)
    H = meta.Hyper(lr=float(np.float32(0.02)), beta_f=float(np.float32(0.99)), beta_d=float(np.float32(0.9)),
                   eps=float(np.float32(1e-8)), eps_alpha=float(np.float32(1e-30)),
                   beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)))
    lo_e, hi_e = np.full(R, 0.05), np.full(R, 10.0)
    lam0 = rng.uniform(1.0, 3.0, R).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    cur, prev = dev(lam0), dev(lam0)
    z = np.zeros(R, np.float32)
    m2f, m2d, mean, var = dev(z), dev(z), dev(z), dev(z)
    ap = dev(np.full(R, -np.inf, np.float32))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # the oracle's own FP64 trajectory on the same samples
    o_lam, o_prev = lam0.astype(np.float64), lam0.astype(np.float64)
    o_st, o_ad = meta.MetaState.zeros((R,)), meta.AdamState.zeros((R,))
    o_n2 = 0.0
    n2 = 0.0
    count_f = count_d = 0
    gap = 0.0
    for i in range(iters):
        u, v = rng.random((R, S)), rng.random((R, S))
        u2, v2 = rng.random((R, S)), rng.random((R, S))
        lam_g = cur.cpu().numpy().astype(np.float64)
        lam_p = prev.cpu().numpy().astype(np.float64)
        F = _toy_grad(lam_g, u, v).astype(np.float32)
        dF = (_toy_grad(lam_g, u2, v2) - _toy_grad(lam_p, u2, v2)).astype(np.float32) if i else np.zeros(R, np.float32)
        pre = {"pi": lam_g, "m2f": m2f.cpu().numpy().astype(np.float64), "m2d": m2d.cpu().numpy().astype(np.float64),
               "mean": mean.cpu().numpy().astype(np.float64), "var": var.cpu().numpy().astype(np.float64),
               "alpha_prev": ap.cpu().numpy().astype(np.float64), "count_f": count_f, "count_d": count_d}
        Fd, dFd = dev(F), dev(dF)
        # pi_next is the slot holding pi_{i-1} (per-element norms read it before overwriting)
        meta_step_raw(hp, cur, prev, Fd, dFd, m2f, m2d, mean, var, ap, 1, [0.05], [10.0], i, count_f, count_d, n2,
                      True, out)
        torch.cuda.synchronize()
        post = {"pi": prev.cpu().numpy().astype(np.float64), "m2f": m2f.cpu().numpy().astype(np.float64),
                "m2d": m2d.cpu().numpy().astype(np.float64), "mean": mean.cpu().numpy().astype(np.float64),
                "var": var.cpu().numpy().astype(np.float64), "alpha_prev": ap.cpu().numpy().astype(np.float64)}
        F64, dF64 = F.astype(np.float64), dF.astype(np.float64)
        if mode == "meta":
            _, ref_n2, _ = _update_close(pre, post, F64, dF64, H, n2, i, lo_e, hi_e, flags=meta.PER_ELEMENT,
                                         pi_prev=lam_p)
            count_d += 1 if (i >= 1 and n2 > 0) else 0
        else:
            ast = meta.AdamState(pre["mean"].copy(), pre["m2f"].copy(), i)
            ref_pi, ref_n2 = meta.adam_update(lam_g, F64, ast, H, lo_e, hi_e)
            assert np.allclose(post["m2f"], ast.v, rtol=1e-5, atol=0)
            scale_m = H.beta1 * np.abs(pre["mean"]) + (1 - H.beta1) * np.abs(F64)
            assert np.all(np.abs(post["mean"] - ast.m) <= 1e-5 * scale_m + 1e-30)
            step_scale = H.lr * scale_m / (1 - H.beta1 ** (i + 1)) / (np.sqrt(ast.v / (1 - H.beta2 ** (i + 1))) + H.eps)
            assert np.all(np.abs(post["pi"] - ref_pi) <= 1e-5 * step_scale + 2 ** -23 * np.abs(lam_g) + 1e-12), i
        count_f += 1
        assert abs(out.item() - ref_n2) <= 1e-5 * ref_n2 + 1e-12 * R, (i, out.item(), ref_n2)
        n2 = out.item()
        cur, prev = prev, cur
        # the oracle's own trajectory
        Fo = _toy_grad(o_lam, u, v)
        if mode == "meta":
            dFo = _toy_grad(o_lam, u2, v2) - _toy_grad(o_prev, u2, v2) if i else np.zeros(R)
            nxt, o_n2, _ = meta.meta_update(o_lam, Fo, dFo, o_st, H, o_n2, lo_e, hi_e, flags=meta.PER_ELEMENT,
                                            pi_prev=o_prev)
        else:
            nxt, o_n2 = meta.adam_update(o_lam, Fo, o_ad, H, lo_e, hi_e)
        o_prev, o_lam = o_lam, nxt
        gap = max(gap, float(np.abs(cur.cpu().numpy().astype(np.float64) - o_lam).max()))
    lam_g = cur.cpu().numpy().astype(np.float64)
    assert gap < 1e-3, gap
    for lam in (lam_g, o_lam):
        assert abs(np.median(lam) - 0.5) < 0.02, np.median(lam)
        assert np.mean(np.abs(lam - 0.5) < 0.1) > 0.95

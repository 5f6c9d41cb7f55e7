"""The fused update's variant flags (per-element step norm of Sec. 4.2; the ablations of Sec. 6;
growing beta_F of appendix A; naive Adam on <F>_M of Sec. 5) against the FP64 oracle on identical
inputs: one step of mer_meta_step_raw_ex from a random state, every state array and the applied
step within 1e-5 relative (spec tolerance for the update)."""
import numpy as np
import pytest

from oracle import meta

from .gpu_common import need_gpu

pytestmark = pytest.mark.gpu

PE, NC, CE, GB, NA, UN = 1, 2, 4, 8, 16, 32


def _state(rng, n, iteration):
    pi = rng.uniform(0.05, 0.95, n).astype(np.float32)
    d = rng.normal(0, 3e-3, n).astype(np.float32)
    d[::7] = 0.0                                     # elements whose own previous step was zero
    pprev = (pi - d).astype(np.float32)
    F = rng.normal(0, 1e-2, n).astype(np.float32)
    dF = rng.normal(0, 1e-3, n).astype(np.float32)
    Fv = rng.normal(0, 1e-2, n).astype(np.float32)
    dFv = rng.normal(0, 1e-3, n).astype(np.float32)
    if iteration == 0:
        z = np.zeros(n, np.float32)
        s = dict(m2f=z, m2d=z, mean=z, var=z, ap=np.full(n, -np.inf, np.float32), mu_f=z, mu_d=z, am=z, av=z)
    else:
        m2f = (rng.normal(0, 1e-2, n) ** 2).astype(np.float32)
        m2f[::97] = 0.0
        m2d = (rng.normal(0, 1e-1, n) ** 2).astype(np.float32)
        s = dict(m2f=m2f, m2d=m2d,
                 mean=rng.normal(0, 1e-2, n).astype(np.float32),
                 var=(rng.uniform(0.1, 1, n) * m2f).astype(np.float32),
                 ap=rng.uniform(0, iteration / (iteration + 1), n).astype(np.float32),
                 # CENTRED first moments well inside sqrt(m2): m2 - mu^2 keeps most of m2
                 mu_f=(0.3 * np.sqrt(m2f) * rng.uniform(-1, 1, n)).astype(np.float32),
                 mu_d=(0.3 * np.sqrt(m2d) * rng.uniform(-1, 1, n)).astype(np.float32),
                 am=rng.normal(0, 1e-2, n).astype(np.float32),
                 av=(rng.normal(0, 1e-2, n) ** 2).astype(np.float32))
    s.update(pi=pi, pprev=pprev, F=F, dF=dF, Fv=Fv, dFv=dFv)
    return {k: v.copy() for k, v in s.items()}


@pytest.mark.parametrize("n,C,iteration,n2,flags", [
    (4099, 3, 5, 2.5e-5, PE), (4099, 3, 0, 0.0, NC), (4099, 5, 6, 1e-3, NC), (50001, 5, 4, 1e-3, CE),
    (4099, 5, 40, 1e-4, GB), (4099, 5, 150, 1e-4, GB), (4099, 3, 0, 0.0, NA), (4099, 5, 7, 1e-4, NA),
    (4099, 5, 3, 1e-3, UN), (4099, 5, 120, 1e-3, PE | NC | CE | GB | NA | UN), (17, 5, 2, 4e-6, PE | CE | NA)])
def test_variant_update_matches_oracle(n, C, iteration, n2, flags):
    torch = need_gpu()
    from paper_2309_15676_gb300.api import HyperParams, meta_step_raw_ex
    rng = np.random.default_rng(1000 + n + iteration + flags)
    s = _state(rng, n, iteration)
    lo = np.array([0.0, 0.0, 0.0, 0.0, 0.05][:C], np.float32)
    hi = np.ones(C, np.float32)
    h = HyperParams(lr=0.01, beta_f=0.99, beta_d=0.9, flags=flags)
    count_f, count_d = iteration, max(0, iteration - 2)
    d = {k: torch.from_numpy(v).cuda() for k, v in s.items()}
    pi_next = d["pprev"].clone()                     # holds pi_{i-1} on entry (PER_ELEMENT)
    arrays = dict(pi=d["pi"], pi_next=pi_next, F=d["F"], dF=d["dF"], m2f=d["m2f"], m2d=d["m2d"], mean=d["mean"],
                  var=d["var"], alpha_prev=d["ap"], mu_f=d["mu_f"], mu_d=d["mu_d"], adam_m=d["am"],
                  adam_v=d["av"], F_var=d["Fv"], dF_var=d["dFv"])
    out = meta_step_raw_ex(h, arrays, C, lo, hi, iteration, count_f, count_d, n2, zero_grads=False)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy().astype(np.float64) for k, v in d.items()}
    got_pi = pi_next.cpu().numpy().astype(np.float64)

    f32 = lambda v: float(np.float32(v))
    H = meta.Hyper(lr=f32(0.01), beta_f=f32(0.99), beta_d=f32(0.9), eps=f32(1e-8), eps_alpha=f32(1e-30),
                   beta1=f32(0.9), beta2=f32(0.999))
    x = {k: v.astype(np.float64) for k, v in s.items()}
    prod = 1.0
    for k in range(count_f):
        prod *= meta.growing_decay(H.beta_f, k)
    st = meta.MetaState(x["m2f"].copy(), x["m2d"].copy(), x["mean"].copy(), x["var"].copy(), x["ap"].copy(),
                        count_f, count_d, iteration, x["mu_f"].copy(), x["mu_d"].copy(), x["am"].copy(),
                        x["av"].copy(), prod)
    ch = np.arange(n) % C
    ref_pi, ref_n2, alpha = meta.meta_update(x["pi"], x["F"], x["dF"], st, H, n2, lo[ch].astype(np.float64),
                                             hi[ch].astype(np.float64), flags=flags, pi_prev=x["pprev"],
                                             F_var=x["Fv"], dF_var=x["dFv"])
    rel = lambda a, b, scale: np.all(np.abs(a - b) <= 1e-5 * scale + 1e-30)
    assert rel(g["m2f"], st.m2f, np.abs(st.m2f)), "m2f"
    assert rel(g["m2d"], st.m2d, np.abs(st.m2d)), "m2d"
    if flags & CE:
        assert rel(g["mu_f"], st.mu_f, np.abs(x["mu_f"]) + np.abs(x["Fv" if flags & UN else "F"])), "mu_f"
        assert rel(g["mu_d"], st.mu_d, np.abs(st.mu_d) + np.sqrt(st.m2d)), "mu_d"
    # alpha and the carried moments: alpha within 1e-5 (absolute on [0, 1] plus relative)
    assert np.all(np.abs(g["ap"] - st.alpha_prev) <= 1e-5 * np.abs(st.alpha_prev) + 2e-6), "alpha"
    dfu = x["dF"] if (iteration >= 1 and n2 > 0) else 0.0
    scale_mean = np.abs(x["mean"] + dfu) + np.abs(x["F"])
    assert rel(g["mean"], st.mean, scale_mean), "mean"
    var_scale = np.abs(x["var"]) + st.m2f + st.m2d * max(n2, 0.0) + (x["pi"] - x["pprev"]) ** 2 * st.m2d
    assert rel(g["var"], st.var, var_scale), "var"
    if flags & NA:
        assert rel(g["am"], st.adam_m, np.abs(x["am"]) + scale_mean), "adam_m"
        assert rel(g["av"], st.adam_v, np.abs(x["av"]) + scale_mean ** 2), "adam_v"
        t = iteration + 1
        step_scale = H.lr * (np.abs(st.adam_m) / (1 - H.beta1 ** t) + 1e-3 * scale_mean) / (
            np.sqrt(st.adam_v / (1 - H.beta2 ** t)) + H.eps) + 1e-5 * H.lr
    else:
        step_scale = H.lr * scale_mean / (np.sqrt(st.var) + H.eps)
    err = np.abs(got_pi - ref_pi)
    assert np.all(err <= 1e-5 * step_scale + 2 ** -23 * np.abs(x["pi"]) + 1e-12), err.max()
    assert abs(out.item() - ref_n2) <= 1e-5 * ref_n2 + 1e-12 * n


def test_context_iterations_with_variants_match_oracle():
    """Three context iterations of a META problem with PER_ELEMENT | CENTRED | GROWING_BETA |
    NAIVE_ADAM: the fused update inside the iteration equals the oracle step on the GPU's own
    F, dF and state (the per-element norm reading the previous parameters from the second slot)."""
    torch = need_gpu()
    from paper_2309_15676_gb300 import synth
    from paper_2309_15676_gb300.api import Context, HyperParams
    flags = PE | CE | GB | NA
    w = synth.workload_spiral(24, 24, 32, 8, 16, max_depth=3, spp_prop=2, spp_fd=1)
    ctx = Context(0)
    pid = ctx.add_scene(w.scene, HyperParams(lr=0.02, flags=flags))
    rng = np.random.default_rng(4)
    ctx.set_target(pid, rng.uniform(0, 1, (24, 24, 3)).astype(np.float32))
    ctx.set_params(pid, w.init_tex)
    f32 = lambda v: float(np.float32(v))
    H = meta.Hyper(lr=f32(0.02), beta_f=f32(0.99), beta_d=f32(0.9), eps=f32(1e-8), eps_alpha=f32(1e-30),
                   beta1=f32(0.9), beta2=f32(0.999))
    lo = np.asarray(w.scene["clamp_lo"], np.float64)[None, None, :]
    hi = np.asarray(w.scene["clamp_hi"], np.float64)[None, None, :]
    for it in range(3):
        pre = {k: v.cpu().numpy().astype(np.float64) for k, v in ctx.state(pid).items()}
        assert {"mu_f", "mu_d", "adam_m", "adam_v"} <= set(pre)
        sp = ctx.stats(pid)
        ctx.gradient_step()
        F, dF = (x.cpu().numpy().astype(np.float64) for x in ctx.grads(pid))
        prod = 1.0
        for k in range(sp["count_f"]):
            prod *= meta.growing_decay(H.beta_f, k)
        st = meta.MetaState(pre["m2f"], pre["m2d"], pre["mean"], pre["var"], pre["alpha_prev"], sp["count_f"],
                            sp["count_d"], it, pre["mu_f"], pre["mu_d"], pre["adam_m"], pre["adam_v"], prod)
        ref_pi, ref_n2, _ = meta.meta_update(pre["pi_cur"], F, dF, st, H, sp["dpi_norm2"], lo, hi, flags=flags,
                                             pi_prev=pre["pi_prev"])
        ctx.update_step()
        got = ctx.get_params(pid).cpu().numpy().astype(np.float64)
        post = {k: v.cpu().numpy().astype(np.float64) for k, v in ctx.state(pid).items()}
        assert np.allclose(post["m2f"], st.m2f, rtol=1e-5, atol=1e-30)
        assert np.allclose(post["adam_v"], st.adam_v, rtol=1e-5, atol=1e-30)
        assert np.all(np.abs(got - ref_pi) <= 1e-4 * H.lr + 2 ** -23 * np.abs(ref_pi)), (it, np.abs(got - ref_pi).max())
        assert abs(ctx.stats(pid)["dpi_norm2"] - ref_n2) <= 1e-4 * ref_n2 + 1e-12
    ctx.close()


def test_uncorrelated_variance_samples_in_context():
    """MER_META_UNCORRELATED: the context renders a second, independent gradient evaluation from
    the four gradient streams shifted by 8 into F_var / dF_var; each equals the oracle's
    proportional / FD gradient on those streams (image-summed gradient tolerance), and F_var
    differs from F sample by sample."""
    torch = need_gpu()
    from oracle import orc
    from paper_2309_15676_gb300 import synth
    from paper_2309_15676_gb300.api import Context, HyperParams
    from .test_gpu_parity import _grad_check
    w = synth.workload_box(24, 24, 8, max_depth=3)
    ctx = Context(0)
    pid = ctx.add_scene(w.scene, HyperParams(lr=0.02, flags=UN))
    target = np.random.default_rng(6).uniform(0, 1, (24, 24, 3)).astype(np.float32)
    ctx.set_target(pid, target)
    ctx.set_params(pid, w.init_tex)
    s = orc.Scene(w.scene)
    spp_p, spp_f = w.scene["spp_prop"], w.scene["spp_fd"]
    for it in range(2):
        pre = {k: v.cpu().numpy().astype(np.float64) for k, v in ctx.state(pid).items()}
        ctx.gradient_step()
        st = ctx.state(pid)
        F, Fv = st["F"].cpu().numpy().astype(np.float64), st["F_var"].cpu().numpy().astype(np.float64)
        ref, _, _ = orc.prop_gradient(s, pre["pi_cur"], target, spp_p, it, stream_offset=8)
        e, f = _grad_check(Fv, ref)
        assert e < 1e-3 and f > 0.999, ("F_var", it, e, f)
        assert not np.array_equal(F, Fv)
        if it >= 1:
            dref = orc.fd_gradient(s, pre["pi_cur"], pre["pi_prev"], target, spp_f, it, stream_offset=8)
            e, f = _grad_check(st["dF_var"].cpu().numpy().astype(np.float64), dref)
            assert e < 1e-3 and f > 0.999, ("dF_var", it, e, f)
        ctx.update_step()
    ctx.close()

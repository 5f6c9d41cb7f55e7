"""Emissive-absorptive volume on the GPU (mer_volume_*) against the FP64 oracle on the same
counters: images (>= 99.9% of pixels within 1e-4 relative, floor 1e-6), replay adjoints and FD-pair
adjoints (image-summed gradient tolerance 1e-3), the standalone image loss, and sampled pixels of
the full 256^3 x 4, four-view workload."""
import numpy as np
import pytest

from oracle import orc
from paper_2309_15676_gb300 import synth

from .gpu_common import frac_within, need_gpu, params_match
from .test_gpu_parity import _grad_check

pytestmark = pytest.mark.gpu


def _small(n=16):
    sc = synth.volume_scene(n=n, views=2, width=24, height=20, bg=(0.1, 0.2, 0.3))
    rng = np.random.default_rng(5)
    p = rng.uniform(0.1, 1.0, (n, n, n, 4)).astype(np.float32)
    p[..., 3] *= 6.0
    return sc, p


def test_volume_render_matches_oracle():
    torch = need_gpu()
    from paper_2309_15676_gb300.api import Volume
    sc, p = _small()
    v = Volume(sc)
    got = v.render(p, spp=2, stream=0, iteration=4).cpu().numpy()
    ref = orc.vol_render_image(orc.Volume(sc), p, 2, 4, 0)
    assert frac_within(got, ref, 1e-4, 1e-6) >= 0.999
    v.close()


def test_volume_adjoint_and_pair_match_oracle():
    torch = need_gpu()
    from paper_2309_15676_gb300.api import Volume
    sc, p = _small()
    v = Volume(sc)
    ov = orc.Volume(sc)
    rng = np.random.default_rng(6)
    dA = rng.normal(size=ov.image_shape).astype(np.float32)
    got = v.adjoint(p, dA, spp=2, stream=1, iteration=4).cpu().numpy()
    ref = orc.vol_adjoint_image(ov, p, 2, 4, 1, dA)
    e, f = _grad_check(got, ref)
    assert e < 1e-3 and f > 0.999, (e, f)
    pB = np.clip(p + rng.normal(0, 0.05, p.shape), 0.0, None).astype(np.float32)
    dB = rng.normal(size=ov.image_shape).astype(np.float32)
    got = v.adjoint_pair(p, pB, dA, dB, spp=1, stream=3, iteration=4).cpu().numpy()
    ref = orc.vol_adjoint_image(ov, p, 1, 4, 3, dA) - orc.vol_adjoint_image(ov, pB, 1, 4, 3, dB)
    e, f = _grad_check(got, ref)
    assert e < 1e-3 and f > 0.999, (e, f)
    v.close()


def test_image_loss_matches_oracle():
    torch = need_gpu()
    from paper_2309_15676_gb300.api import image_loss
    rng = np.random.default_rng(7)
    img = rng.uniform(0, 2, (3, 17, 11, 3)).astype(np.float32)
    tgt = rng.uniform(0, 1, img.shape).astype(np.float32)
    for kind, fn in ((0, orc.l2_loss), (1, orc.mrse_loss)):
        loss, d = image_loss(torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda(), kind)
        lo, do = fn(img.reshape(-1, 3), tgt.reshape(-1, 3))
        assert abs(loss.item() - lo) <= 1e-5 * lo
        assert np.allclose(d.cpu().numpy().reshape(-1, 3), do, rtol=1e-5, atol=1e-9)


def test_volume_full_size_sampled():
    torch = need_gpu()
    from paper_2309_15676_gb300.api import Volume
    w = synth.workload_volume()
    v = Volume(w.scene)
    got = v.render(w.target_tex, spp=1, stream=0, iteration=2).cpu().numpy().reshape(-1, 3)
    v.close()
    idx = np.sort(np.random.default_rng(8).choice(got.shape[0], 400, replace=False)).astype(np.uint32)
    ref = orc.vol_render_samples(orc.Volume(w.scene), w.target_tex, idx, np.zeros(len(idx), np.uint32), 2, 0)
    ok = np.all(np.abs(got[idx] - ref) <= 1e-4 * np.abs(ref) + 1e-6, axis=1)
    assert ok.mean() >= 0.999, ok.mean()


# ---------------------------------------------------------------------------------------
# the volume optimiser (mer_volume_opt_*) iteration by iteration against the oracle
# ---------------------------------------------------------------------------------------
def _opt_setup(torch, mode, flags=0, loss=0, lr=0.05):
    from oracle import meta
    from paper_2309_15676_gb300.api import MODE_ADAM, MODE_META, HyperParams, Volume, VolumeOptimizer
    sc = synth.volume_scene(n=12, views=2, width=16, height=16, bg=(0.05, 0.1, 0.2))
    rng = np.random.default_rng(9)
    tgt_p = rng.uniform(0.0, 1.0, (12, 12, 12, 4)).astype(np.float32)
    tgt_p[..., 3] *= 8.0
    ov = orc.Volume(sc)
    target = orc.vol_render_image(ov, tgt_p, 4, 0, orc.ST_TARGET).astype(np.float32)
    init = np.full((12, 12, 12, 4), 0.3, np.float32)
    init[..., 3] = 2.0
    v = Volume(sc)
    hp = HyperParams(lr=lr, mode=MODE_META if mode == "meta" else MODE_ADAM, flags=flags)
    opt = VolumeOptimizer(v, torch.from_numpy(target).cuda(), torch.from_numpy(init).cuda(), hp, loss=loss)
    H = meta.Hyper(lr=float(np.float32(lr)), beta_f=float(np.float32(0.99)), beta_d=float(np.float32(0.9)))
    lo = np.asarray(sc["clamp_lo"], np.float64)
    hi = np.asarray(sc["clamp_hi"], np.float64)
    return v, opt, ov, target, H, lo, hi


def _oracle_F(ov, p, target, it, loss, soff=0):
    img = orc.vol_render_image(ov, p, 1, it, orc.ST_PROP_PRIMAL + soff)
    l, d = orc.image_loss(img.reshape(-1, 3), target.reshape(-1, 3), loss)
    return orc.vol_adjoint_image(ov, p, 1, it, orc.ST_PROP_ADJ + soff, d.reshape(img.shape)), l


def _oracle_dF(ov, pa, pb, target, it, loss, soff=0):
    ia = orc.vol_render_image(ov, pa, 1, it, orc.ST_FD_PRIMAL + soff)
    ib = orc.vol_render_image(ov, pb, 1, it, orc.ST_FD_PRIMAL + soff)
    _, da = orc.image_loss(ia.reshape(-1, 3), target.reshape(-1, 3), loss)
    _, db = orc.image_loss(ib.reshape(-1, 3), target.reshape(-1, 3), loss)
    return (orc.vol_adjoint_image(ov, pa, 1, it, orc.ST_FD_ADJ + soff, da.reshape(ia.shape)) -
            orc.vol_adjoint_image(ov, pb, 1, it, orc.ST_FD_ADJ + soff, db.reshape(ib.shape)))


def _f64(d):
    return {k: x.cpu().numpy().astype(np.float64) for k, x in d.items()}


@pytest.mark.parametrize("loss", [0, 1])
def test_volume_optimiser_meta_matches_oracle(loss):
    torch = need_gpu()
    from oracle import meta
    v, opt, ov, target, H, lo, hi = _opt_setup(torch, "meta", loss=loss)
    for it in range(3):
        pre, sp = _f64(opt.state()), opt.stats()
        opt.iterate(1, use_graph=it > 0)
        post, so = _f64(opt.state()), opt.stats()
        assert so["iteration"] == it + 1
        Fo, lo_ = _oracle_F(ov, pre["pi_cur"], target, it, loss)
        e, f = _grad_check(post["F"], Fo)
        assert e < 1e-3 and f > 0.999, ("F", it, e, f)
        assert abs(so["loss"] - lo_) <= 1e-4 * lo_
        if it >= 1:
            e, f = _grad_check(post["dF"], _oracle_dF(ov, pre["pi_cur"], pre["pi_prev"], target, it, loss))
            assert e < 1e-3 and f > 0.999, ("dF", it, e, f)
        else:   # both slots hold pi_0: the pair cancels up to the order of the reductions
            assert np.abs(post["dF"]).max() <= 1e-5 * np.abs(post["F"]).max()
        ost = meta.MetaState(pre["m2f"], pre["m2d"], pre["mean"], pre["var"], pre["alpha_prev"],
                             sp["count_f"], sp["count_d"], it)
        ref_pi, ref_n2, _ = meta.meta_update(pre["pi_cur"], post["F"], post["dF"], ost, H, sp["dpi_norm2"], lo, hi)
        step_ref = ref_pi - pre["pi_cur"]
        err = np.abs((post["pi_cur"] - pre["pi_cur"]) - step_ref)
        assert np.all(err <= 1e-4 * np.abs(step_ref) + 1e-4 * H.lr), (it, err.max())
        assert np.array_equal(post["pi_prev"], pre["pi_cur"])
        assert abs(so["dpi_norm2"] - ref_n2) <= 1e-4 * ref_n2
    assert opt.launches() > 0
    opt.close()
    v.close()


def test_volume_optimiser_adam_and_variants_match_oracle():
    torch = need_gpu()
    from oracle import meta
    # Adam: only the proportional branch, the update against the oracle's Adam on the same F
    v, opt, ov, target, H, lo, hi = _opt_setup(torch, "adam", lr=0.02)
    ast = meta.AdamState.zeros(opt.shape)
    for it in range(2):
        pre = _f64(opt.state())
        opt.iterate(1, use_graph=True)
        post = _f64(opt.state())
        assert "dF" not in post
        e, f = _grad_check(post["F"], _oracle_F(ov, pre["pi_cur"], target, it, 0)[0])
        assert e < 1e-3 and f > 0.999, ("F", it, e, f)
        ref_pi, _ = meta.adam_update(pre["pi_cur"], post["F"], ast, H, lo, hi)
        step_ref = ref_pi - pre["pi_cur"]
        assert np.all(np.abs((post["pi_cur"] - pre["pi_cur"]) - step_ref) <= 1e-4 * np.abs(step_ref) + 1e-4 * H.lr)
    opt.close()
    v.close()
    # UNCORRELATED + GROWING_BETA + PER_ELEMENT: independent variance samples on the shifted streams,
    # the update with all three against the oracle's. (CENTRED is left to the texture variant tests:
    # its first step has m2 - mu^2 = 0 exactly, so the step divides by rounding residue.)
    fl = meta.UNCORRELATED | meta.GROWING_BETA | meta.PER_ELEMENT
    v, opt, ov, target, H, lo, hi = _opt_setup(torch, "meta", flags=fl)
    ost = meta.MetaState.zeros(opt.shape)     # carries the oracle's growing-beta product
    for it in range(3):
        pre, sp = _f64(opt.state()), opt.stats()
        opt.iterate(1, use_graph=False)
        post = _f64(opt.state())
        Fv = _oracle_F(ov, pre["pi_cur"], target, it, 0, soff=8)[0]
        e, f = _grad_check(post["F_var"], Fv)
        assert e < 1e-3 and f > 0.999, ("F_var", it, e, f)
        if it >= 1:
            e, f = _grad_check(post["dF_var"], _oracle_dF(ov, pre["pi_cur"], pre["pi_prev"], target, it, 0, soff=8))
            assert e < 1e-3 and f > 0.999, ("dF_var", it, e, f)
        for k, a in (("m2f", "m2f"), ("m2d", "m2d"), ("mean", "mean"), ("var", "var"), ("alpha_prev", "alpha_prev")):
            setattr(ost, k, pre[a])
        ost.count_f, ost.count_d, ost.iteration = sp["count_f"], sp["count_d"], it
        ref_pi, _, _ = meta.meta_update(pre["pi_cur"], post["F"], post["dF"], ost, H, sp["dpi_norm2"], lo, hi,
                                        flags=fl, pi_prev=pre["pi_prev"], F_var=post["F_var"], dF_var=post["dF_var"])
        step_ref = ref_pi - pre["pi_cur"]
        err = np.abs((post["pi_cur"] - pre["pi_cur"]) - step_ref)
        assert np.all(err <= 1e-4 * np.abs(step_ref) + 1e-4 * H.lr), (it, err.max())
    opt.close()
    v.close()


def test_volume_optimiser_graph_equals_launches_and_rejects_bad_input():
    torch = need_gpu()
    from paper_2309_15676_gb300._lib import MerError
    from paper_2309_15676_gb300.api import HyperParams, VolumeOptimizer
    v, a, *_ = _opt_setup(torch, "meta")
    _, b, *_ = _opt_setup(torch, "meta")
    a.iterate(4, use_graph=False)
    b.iterate(4, use_graph=True)
    pa, pb = a.params().cpu().numpy(), b.params().cpu().numpy()
    assert params_match(pa, pb)
    assert a.stats()["iteration"] == b.stats()["iteration"] == 4
    # reset: back to iteration 0 and the same first step
    init = np.full(a.shape, 0.3, np.float32)
    init[..., 3] = 2.0
    a.set_params(torch.from_numpy(init).cuda())
    assert a.stats()["iteration"] == 0
    tgt = torch.zeros(v.image_shape, device="cuda")
    with pytest.raises(MerError):
        VolumeOptimizer(v, tgt, torch.from_numpy(init).cuda(), HyperParams(precond_lambda=1.0))
    with pytest.raises(MerError):
        VolumeOptimizer(v, tgt, torch.from_numpy(init).cuda(), HyperParams(), loss=7)
    a.close()
    b.close()
    v.close()


@pytest.mark.parametrize("dims,step", [((3, 5, 2), 0.3), ((1, 1, 1), 0.05)])
def test_volume_anisotropic_and_single_voxel(dims, step):
    """A grid with nx != ny != nz and a coarse step, and a one-voxel volume (every tap clamps to it):
    render and adjoint against the oracle."""
    need_gpu()
    from paper_2309_15676_gb300.api import Volume
    sc = synth.volume_scene(n=4, views=2, width=9, height=7, step=step, bg=(0.2, 0.1, 0.05))
    sc["nx"], sc["ny"], sc["nz"] = dims
    nx, ny, nz = dims
    rng = np.random.default_rng(8)
    p = rng.uniform(0.1, 1.0, (nz, ny, nx, 4)).astype(np.float32)
    p[..., 3] *= 3.0
    v = Volume(sc)
    ov = orc.Volume(sc)
    got = v.render(p, spp=2, stream=0, iteration=1).cpu().numpy()
    ref = orc.vol_render_image(ov, p, 2, 1, 0)
    assert frac_within(got, ref, 1e-4, 1e-6) >= 0.999
    dA = rng.normal(size=ov.image_shape).astype(np.float32)
    g = v.adjoint(p, dA, spp=2, stream=1, iteration=1).cpu().numpy()
    gr = orc.vol_adjoint_image(ov, p, 2, 1, 1, dA)
    e, f = _grad_check(g, gr)
    assert e < 1e-3 and f > 0.999, (dims, e, f)
    v.close()

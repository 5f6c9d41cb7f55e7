"""Emissive-absorptive volume on the GPU (mer_volume_*) against the FP64 oracle on the same
counters: images (>= 99.9% of pixels within 1e-4 relative, floor 1e-6), replay adjoints and FD-pair
adjoints (image-summed gradient tolerance 1e-3), the standalone image loss, and sampled pixels of
the full 256^3 x 4, four-view workload."""
import numpy as np
import pytest

from oracle import orc
from paper_2309_15676_gb300 import synth

from .gpu_common import frac_within, need_gpu
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

"""Oracle emissive-absorptive volume (Sec. 6 high-dimensional experiment): the march's bookkeeping
and its replay gradient, pinned by identities of the quadrature and by per-seed central
differences (the march's random numbers do not depend on the parameters)."""
import numpy as np

from oracle import orc
from paper_2309_15676_gb300 import synth


def _small(bg=(0.0, 0.0, 0.0), n=6):
    sc = synth.volume_scene(n=n, views=2, width=5, height=4, bg=bg)
    return sc


def test_emission_and_transmittance_telescope():
    """Constant emission e and density s: the march gives e (1 - T_end) + T_end bg per sample with
    T_end = exp(-s K delta), K the number of samples inside; so e = bg = 1 gives exactly 1, emission
    enters linearly, and -log(T_end) / (s delta) is a whole number of steps."""
    n = 6
    p = np.zeros((n, n, n, 4))
    p[..., 3] = 0.7
    sc1 = _small(bg=(1.0, 1.0, 1.0))
    ones = p.copy()
    ones[..., :3] = 1.0
    img1 = orc.vol_render_image(orc.Volume(sc1), ones, 2, 3, 0)
    assert np.allclose(img1, 1.0, rtol=0, atol=1e-13)
    sc0 = _small()
    twos = p.copy()
    twos[..., :3] = 2.0
    a = orc.vol_render_image(orc.Volume(sc0), ones, 1, 3, 0)
    b = orc.vol_render_image(orc.Volume(sc0), twos, 1, 3, 0)
    assert np.allclose(b, 2.0 * a, rtol=1e-13, atol=0)
    t_end = 1.0 - a                                      # e = 1, bg = 0
    hit = t_end < 1.0 - 1e-12
    assert hit.any()
    k = -np.log(t_end[hit]) / (0.7 * sc0["step"])
    assert np.allclose(k, np.round(k), atol=1e-9)


def test_adjoint_matches_central_differences_per_seed():
    rng = np.random.default_rng(3)
    n = 6
    sc = _small(bg=(0.1, 0.2, 0.3), n=n)
    vol = orc.Volume(sc)
    p = rng.uniform(0.2, 1.0, (n, n, n, 4))
    p[..., 3] *= 4.0
    dimg = rng.normal(size=vol.image_shape)
    g = orc.vol_adjoint_image(vol, p, 2, 7, 1, dimg)
    J = lambda q: float(np.sum(dimg * orc.vol_render_image(vol, q, 2, 7, 1)))
    nz = np.argwhere(np.abs(g).sum(-1) > 0)
    assert len(nz) > 20
    h = 1e-6
    for (z, y, x) in nz[:: max(1, len(nz) // 10)]:
        for c in range(4):
            a, b = p.copy(), p.copy()
            a[z, y, x, c] += h
            b[z, y, x, c] -= h
            fd = (J(a) - J(b)) / (2 * h)
            assert abs(g[z, y, x, c] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (z, y, x, c, g[z, y, x, c], fd)


def test_empty_volume_shows_background():
    sc = _small(bg=(0.25, 0.5, 0.75))
    img = orc.vol_render_image(orc.Volume(sc), np.zeros((6, 6, 6, 4)), 1, 0, 0)
    assert np.allclose(img, np.array([0.25, 0.5, 0.75]), rtol=0, atol=1e-15)


def test_emission_gradient_sums_to_the_pixel_opacity():
    """With a uniform density the emission gradient of one pixel and channel, summed over all voxels,
    is sum_k T_k a_k = 1 - T_end whatever the emission: the trilinear weights of every sample sum to
    one (clamped taps included) and the opacity is what a render with unit emission and a black
    background returns for the same counters."""
    n = 6
    sc = _small(n=n)
    vol = orc.Volume(sc)
    rng = np.random.default_rng(11)
    p = rng.uniform(0.1, 2.0, (n, n, n, 4))
    p[..., 3] = 0.9                                    # uniform density
    ones = p.copy()
    ones[..., :3] = 1.0
    opacity = orc.vol_render_image(vol, ones, 3, 5, 1)   # unit emission, black background
    shape = vol.image_shape
    checked = 0
    for flat in rng.choice(int(np.prod(shape[:3])), 12, replace=False):
        v, y, x = np.unravel_index(flat, shape[:3])
        for ch in range(3):
            dimg = np.zeros(shape)
            dimg[v, y, x, ch] = 1.0
            g = orc.vol_adjoint_image(vol, p, 3, 5, 1, dimg)
            assert abs(g[..., ch].sum() - opacity[v, y, x, ch]) <= 1e-12, (v, y, x, ch)
            other = [c for c in range(3) if c != ch]
            assert np.all(g[..., other] == 0.0)
            checked += opacity[v, y, x, ch] > 0
    assert checked > 0


def test_jittered_march_counts_the_chord():
    """Uniform density s and emission 1 over a black background: each sample returns 1 - T_end with
    T_end = exp(-s delta K), K the number of march samples inside the box. With a 1x1 image and a
    field of view of 1e-3 degrees every sample's ray is the eye-to-target ray, whose chord l through
    [-1, 1]^3 is a slab intersection here in numpy. A march started at a uniform jitter within the
    first step takes floor(l/delta) or ceil(l/delta) samples, l/delta on average; a start without
    jitter or at a fixed offset gives a biased mean."""
    n = 6
    rng = np.random.default_rng(19)
    for eye, tg in (([2.7, 1.3, -2.1], [0.15, -0.2, 0.3]), ([-0.4, 2.9, 1.1], [0.3, 0.1, -0.5]),
                    ([3.0, -0.6, 0.2], [-0.2, 0.45, 0.05])):
        sc = _small(n=n)
        sc["n_views"], sc["width"], sc["height"] = 1, 1, 1
        sc["cameras"] = np.asarray([eye + tg + [0.0, 1.0, 0.0] + [1e-3]], np.float32)
        vol = orc.Volume(sc)
        p = np.zeros((n, n, n, 4))
        p[..., :3] = 1.0
        p[..., 3] = 0.7
        N = 20000
        L = orc.vol_render_samples(vol, p, np.zeros(N, np.uint32), np.arange(N, dtype=np.uint32),
                                   int(rng.integers(100)), 0)
        delta = float(np.float32(sc["step"]))
        K = -np.log(1.0 - L[:, 0]) / (0.7 * delta)
        e = np.float32(eye).astype(np.float64)
        t = np.float32(tg).astype(np.float64)
        d = (t - e) / np.linalg.norm(t - e)
        ta, tb = (-1.0 - e) / d, (1.0 - e) / d
        chord = np.min(np.maximum(ta, tb)) - np.max(np.minimum(ta, tb))
        x = chord / delta
        assert np.all(np.isclose(K, np.floor(x), atol=1e-6) | np.isclose(K, np.ceil(x), atol=1e-6))
        assert abs(K.mean() - x) <= 5.0 * K.std() / np.sqrt(N) + 1e-6, (K.mean(), x)

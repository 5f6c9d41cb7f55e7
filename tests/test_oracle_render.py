"""Oracle path tracer against closed-form radiance (white furnace, Lambertian plane under a
constant environment, emitting closed box) and the depth convention."""
import numpy as np
import pytest
from scipy import integrate

from oracle import orc
from paper_2309_15676_gb300 import synth


@pytest.mark.parametrize("depth", [2, 3, 5])
@pytest.mark.parametrize("albedo", [1.0, 0.6])
def test_white_furnace_per_sample(oracle_lib, depth, albedo):
    """Convex Lambert sphere in a constant environment: with NEE (cosine env sampling) and BSDF
    sampling at equal densities the power-heuristic weights are 1/2 each, so each sample that
    hits the sphere is exactly albedo * L_env, and each miss is L_env."""
    env = np.array([0.5, 1.0, 2.0])
    sc = orc.Scene(synth.furnace_scene(albedo=albedo, max_depth=depth, env=tuple(env)))
    n = sc.n_pix * 2
    L = orc.render_samples(sc, np.zeros((8, 8, 3)), np.arange(n) % sc.n_pix, np.arange(n) // sc.n_pix, 3,
                           orc.ST_PROP_PRIMAL)
    a = np.float64(np.float32(albedo))
    hit = np.isclose(L, a * env, rtol=1e-12, atol=0).all(1)
    miss = np.isclose(L, env, rtol=1e-12, atol=0).all(1)
    assert np.all(hit | miss)
    assert hit.sum() > 0.2 * n


def test_depth_one_shows_only_emitters(oracle_lib):
    sc = orc.Scene(synth.furnace_scene(albedo=0.6, max_depth=1, env=(0.5, 1.0, 2.0)))
    L = orc.render_samples(sc, np.zeros((8, 8, 3)), np.arange(sc.n_pix), np.zeros(sc.n_pix), 0, 0)
    # sphere hits show no light (not emissive), misses show the environment
    ok = np.isclose(L, 0).all(1) | np.isclose(L, [0.5, 1.0, 2.0]).all(1)
    assert ok.all() and np.isclose(L, 0).all(1).sum() > 0


@pytest.mark.parametrize("depth", [2, 4])
def test_lambert_plane_constant_env(oracle_lib, depth):
    """rho(uv) * L_env per sample for a constant albedo on a plane that occludes nothing."""
    env = np.array([0.7, 0.8, 0.9])
    sc = orc.Scene(synth.plane_scene(max_depth=depth, env=tuple(env)))
    tex = np.full((8, 8, 3), 0.3)
    L = orc.render_samples(sc, tex, np.arange(sc.n_pix), np.ones(sc.n_pix), 5, 1)
    assert np.allclose(L, 0.3 * env, rtol=1e-12)


def test_lambert_plane_textured_mean(oracle_lib):
    """With a textured albedo each sample is rho(uv_s) L_env: the image lies in the texture's
    value range times L_env and its mean over pixels is a bilinear average of texels."""
    env = np.array([1.0, 1.0, 1.0])
    sc = orc.Scene(synth.plane_scene(max_depth=3, env=tuple(env)))
    tex = np.random.default_rng(0).uniform(0.1, 0.9, (8, 8, 3))
    img = orc.render_image(sc, tex, 2, 0, 0)
    assert img.min() >= tex.min() - 1e-12 and img.max() <= tex.max() + 1e-12


def test_depth_one_emitting_box_exact(oracle_lib):
    sc = orc.Scene(synth.emitting_box_scene(albedo=0.5, le=2.0, max_depth=1))
    img = orc.render_image(sc, np.zeros((4, 4, 3)), 3, 0, 0)
    assert np.allclose(img, 2.0, rtol=1e-12)


@pytest.mark.parametrize("depth", [2, 3, 4])
def test_emitting_box_mean(oracle_lib, depth):
    """Closed box whose walls all emit Le with albedo rho: radiance Le * sum_{k<D} rho^k everywhere.
    Checked within 5 sigma (NEE to area lights + MIS is unbiased, not exact per sample)."""
    rho, le = 0.5, 1.0
    sc = orc.Scene(synth.emitting_box_scene(albedo=rho, le=le, max_depth=depth))
    spp = 600
    pix = np.repeat(np.arange(sc.n_pix), spp)
    smp = np.tile(np.arange(spp), sc.n_pix)
    L = orc.render_samples(sc, np.zeros((4, 4, 3)), pix, smp, 0, orc.ST_EVAL)[:, 0]
    expect = le * sum(rho ** k for k in range(depth))
    se = L.std() / np.sqrt(len(L))
    assert abs(L.mean() - expect) < 5 * se + 1e-12, (L.mean(), expect, se)


def test_streams_and_iterations_decorrelate(oracle_lib):
    w = synth.workload_box(8, 8, 8, max_depth=3)
    sc = orc.Scene(w.scene)
    tex = w.init_tex.astype(np.float64)
    a = orc.render_image(sc, tex, 1, 0, orc.ST_PROP_PRIMAL)
    b = orc.render_image(sc, tex, 1, 0, orc.ST_PROP_ADJ)
    c = orc.render_image(sc, tex, 1, 1, orc.ST_PROP_PRIMAL)
    a2 = orc.render_image(sc, tex, 1, 0, orc.ST_PROP_PRIMAL)
    assert np.array_equal(a, a2)
    assert not np.allclose(a, b) and not np.allclose(a, c)


def test_mrse_loss_constant_target_and_fd(oracle_lib):
    """MRSE with a constant target c is the L2 loss divided by c^2 + 0.01 (loss and adjoint); its
    adjoint image is the derivative of the loss (central differences on a tiny image)."""
    rng = np.random.default_rng(31)
    img = rng.uniform(0, 2, (3, 4, 3))
    c = 0.7
    tgt = np.full_like(img, c)
    l2, d2 = orc.l2_loss(img, tgt)
    lm, dm = orc.mrse_loss(img, tgt)
    assert np.isclose(lm, l2 / (c * c + 0.01), rtol=1e-14) and np.allclose(dm, d2 / (c * c + 0.01), rtol=1e-14)
    tgt = rng.uniform(0, 1, img.shape)
    _, dm = orc.mrse_loss(img, tgt)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 2, 1), (2, 3, 2)]:
        a, b = img.copy(), img.copy()
        a[idx] += h
        b[idx] -= h
        fd = (orc.mrse_loss(a, tgt)[0] - orc.mrse_loss(b, tgt)[0]) / (2 * h)
        assert abs(fd - dm[idx]) <= 1e-7 * abs(dm[idx]) + 1e-12


@pytest.mark.parametrize("th", [[0.2, 0.5, 0.8, 0.3, 0.4], [0.9, 0.6, 0.3, 0.8, 0.15], [0.5, 0.5, 0.5, 0.0, 1.0]])
def test_glossy_plane_constant_env_is_env_times_albedo(oracle_lib, th):
    """Direct light only (D = 2) on a principled plane that occludes nothing, under a constant
    environment: the expected pixel value is L_env times the directional albedo
    int f(wo, wi) cos_i dw_i, whatever the MIS weights are, as long as the two strategies' weights
    sum to one. Unlike the Lambert plane, BSDF and environment sampling have different densities
    here, so a heuristic applied inconsistently between them biases the mean. Pixels at the image
    centre see the plane at normal incidence, where the albedo is a 1D quadrature of the BSDF."""
    env = np.array([0.7, 0.8, 0.9])
    sc = orc.Scene(synth.plane_scene(width=64, height=64, max_depth=2, principled=True, env=tuple(env)))
    th = np.array(th)
    tex = np.tile(th, (8, 8, 1))
    n = 200_000
    pix = np.array([31 * 64 + 31, 31 * 64 + 32, 32 * 64 + 31, 32 * 64 + 32], np.uint32)
    L = orc.render_samples(sc, tex, np.tile(pix, n // 4), np.repeat(np.arange(n // 4, dtype=np.uint32), 4), 3, 0)
    mean, se = L.mean(0), L.std(0) / np.sqrt(n)
    up = np.array([0.0, 1.0, 0.0])

    def f_cos(theta, c):
        wi = np.array([np.sin(theta), np.cos(theta), 0.0])
        return orc.bsdf(1, th, up, up, wi)[0][c] * np.cos(theta) * np.sin(theta) * 2.0 * np.pi

    albedo = np.array([integrate.quad(f_cos, 0.0, np.pi / 2, args=(c,), epsabs=1e-12, epsrel=1e-10, limit=200)[0]
                       for c in range(3)])
    assert np.all(np.abs(mean - env * albedo) <= 5.0 * se + 1e-6), (mean, env * albedo, se)


def _glossy_plane_under_quad_light(le, res, eye):
    """A principled plane (y = 0, normal +y) seen at its centre from `eye`, and one quad light
    (centre (0.5, 0.8, 0), side 0.4) facing down at it; no environment."""
    mb = synth._MeshBuilder()
    mb.quad((-0.6, 0, 0.6), (1.2, 0, 0), (0, 0, -1.2), mat=0)
    p0, e1, e2, le = synth._light_quad((0.5, 0.8, 0.0), 0.4, le)
    mb.quad(p0, e1, e2, mat=1, light=0)
    up = (0, 0, -1) if eye[0] == 0.0 else (0, 1, 0)
    return synth._scene(mb.arrays(), mat_type=[synth.PRINCIPLED, synth.LAMBERT], mat_textured=[1, 0],
                        mat_const=[[0.5] * 5, [0.0] * 5], quads=[synth._quad_row(p0, e1, e2, le)], env=None,
                        eye=eye, target=(0.0, 0.0, -0.001), up=up, fov_deg=50,
                        width=res, height=res, tex_c=5, tex_h=8, tex_w=8, max_depth=2)


# eye straight above (the light is off the specular lobe: light sampling dominates), and eye at
# the mirror image of the light (the lobe points at the light: both strategies carry weight)
@pytest.mark.parametrize("eye,th", [((0.0, 1.0, 0.0), [0.2, 0.5, 0.8, 0.3, 0.4]),
                                    ((-0.5, 0.8, 0.0), [0.2, 0.5, 0.8, 0.7, 0.3]),
                                    ((-0.5, 0.8, 0.0), [0.6, 0.4, 0.2, 0.2, 0.6])])
def test_glossy_plane_under_quad_light_is_the_area_integral(oracle_lib, eye, th):
    """Direct light only (D = 2) from an area light on a principled surface: the expected value at
    the point the centre pixels see is the integral over the light's area of
    Le f(wo, wi) cos_i cos_l / r^2, here by 2D quadrature of the BSDF. It pins the area-to-solid-
    angle conversion of the light's density and the MIS of light and BSDF sampling for a glossy
    lobe. The four centre pixels of a 256^2 image cover a region symmetric about that point to
    first order, so the footprint moves the mean only at second order (about 1e-4 relative, a tenth
    of the tolerance)."""
    le = np.array([4.0, 5.0, 6.0])
    res = 256
    sc = orc.Scene(_glossy_plane_under_quad_light(tuple(le), res, eye))
    th = np.array(th)
    tex = np.tile(th, (8, 8, 1))
    n = 200_000
    c0 = res // 2
    pix = np.array([(c0 - 1) * res + c0 - 1, (c0 - 1) * res + c0, c0 * res + c0 - 1, c0 * res + c0], np.uint32)
    L = orc.render_samples(sc, tex, np.tile(pix, n // 4), np.repeat(np.arange(n // 4, dtype=np.uint32), 4), 3, 0)
    mean, se = L.mean(0), L.std(0) / np.sqrt(n)
    up = np.array([0.0, 1.0, 0.0])
    wo = np.array(eye) / np.linalg.norm(eye)
    expected = []
    for c in range(3):
        def integrand(z, x):
            d = np.array([x, 0.8, z])
            r2 = d @ d
            wi = d / np.sqrt(r2)
            return le[c] * orc.bsdf(1, th, up, wo, wi)[0][c] * wi[1] * wi[1] / r2   # cos_i = cos_l = wi_y
        expected.append(integrate.dblquad(integrand, 0.3, 0.7, -0.2, 0.2, epsabs=1e-10, epsrel=1e-8)[0])
    expected = np.array(expected)
    assert np.all(np.abs(mean - expected) <= 5.0 * se), (mean, expected, se)

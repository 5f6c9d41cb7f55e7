"""Oracle gradients: PRB replay against the stored-vertex derivation, against central finite
differences with common random numbers, and against the Lambertian-plane closed form."""
import numpy as np
import pytest

from oracle import orc
from paper_2309_15676_gb300 import synth


def _box(depth=4):
    w = synth.workload_box(8, 8, 8, max_depth=depth)
    return orc.Scene(w.scene), w.init_tex.astype(np.float64)


def _spiral(depth=4):
    w = synth.workload_spiral(8, 8, 32, 8, 8, max_depth=depth)
    return orc.Scene(w.scene), w.init_tex.astype(np.float64)


@pytest.mark.parametrize("make", [_box, _spiral])
def test_prb_equals_stored_vertex_adjoint(oracle_lib, make):
    sc, tex = make()
    dimg = np.random.default_rng(0).normal(size=(sc.st.height, sc.st.width, 3))
    g1 = orc.adjoint_image(sc, tex, 4, 3, orc.ST_PROP_ADJ, dimg)
    g2 = orc.adjoint_image(sc, tex, 4, 3, orc.ST_PROP_ADJ, dimg, stored=True)
    assert np.abs(g2).max() > 0
    assert np.abs(g1 - g2).max() <= 1e-12 * np.abs(g2).max()


@pytest.mark.parametrize("make,channels", [(_box, (0, 1, 2)), (_spiral, (0, 1, 2))])
def test_adjoint_matches_central_fd_per_seed(oracle_lib, make, channels):
    """For albedo / base colour the sampling does not depend on the parameter, so the gradient of
    J(theta) = sum_p dimg_p . I_p(theta; u) at fixed random numbers u is exact per seed."""
    sc, tex = make()
    dimg = np.random.default_rng(1).normal(size=(sc.st.height, sc.st.width, 3))
    g = orc.adjoint_image(sc, tex, 2, 5, orc.ST_EVAL, dimg)
    J = lambda t: np.sum(dimg * orc.render_image(sc, t, 2, 5, orc.ST_EVAL))
    nz = np.argwhere(np.abs(g).sum(-1) > 0)
    assert len(nz) >= 4
    h = 1e-6
    for (y, x) in nz[:: max(1, len(nz) // 6)]:
        for c in channels:
            tp, tm = tex.copy(), tex.copy()
            tp[y, x, c] += h
            tm[y, x, c] -= h
            fd = (J(tp) - J(tm)) / (2 * h)
            assert abs(g[y, x, c] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (y, x, c, g[y, x, c], fd)


def test_plane_gradient_closed_form(oracle_lib):
    """Lambertian plane under env: each sample is rho(uv) L_env, so the gradient of sum_p dimg_p I_p
    summed over all texels of channel c is L_env[c] * sum_p dimg[p, c] (bilinear weights sum to 1)."""
    env = np.array([0.7, 0.8, 0.9])
    sc = orc.Scene(synth.plane_scene(max_depth=3, env=tuple(env)))
    tex = np.random.default_rng(2).uniform(0.1, 0.9, (8, 8, 3))
    dimg = np.random.default_rng(3).normal(size=(sc.st.height, sc.st.width, 3))
    g = orc.adjoint_image(sc, tex, 2, 0, orc.ST_PROP_ADJ, dimg)
    env32 = env.astype(np.float32).astype(np.float64)
    assert np.allclose(g.sum((0, 1)), env32 * dimg.sum((0, 1)), rtol=1e-10)


@pytest.mark.slow
def test_metal_rough_gradient_unbiased(oracle_lib):
    """Metal and roughness steer the sampling, so the detached-sampling gradient matches finite
    differences only in expectation: compare means over seeds within 5 sigma."""
    w = synth.workload_spiral(4, 4, 32, 8, 4, max_depth=3)
    sc = orc.Scene(w.scene)
    tex = w.init_tex.astype(np.float64)
    dimg = np.random.default_rng(4).normal(size=(4, 4, 3))
    g_all = orc.adjoint_image(sc, tex, 64, 0, orc.ST_EVAL, dimg)
    (y, x) = np.unravel_index(np.argmax(np.abs(g_all[..., 3])), g_all.shape[:2])
    n = 300
    a = np.zeros((n, 2))
    b = np.zeros((n, 2))
    h = 2e-3
    for s in range(n):
        g = orc.adjoint_image(sc, tex, 1, s, orc.ST_EVAL, dimg)
        a[s] = g[y, x, 3], g[y, x, 4]
        for k, c in enumerate((3, 4)):
            tp, tm = tex.copy(), tex.copy()
            tp[y, x, c] += h
            tm[y, x, c] -= h
            b[s, k] = (np.sum(dimg * orc.render_image(sc, tp, 1, s, orc.ST_EVAL))
                       - np.sum(dimg * orc.render_image(sc, tm, 1, s, orc.ST_EVAL))) / (2 * h)
    for k in range(2):
        se = np.sqrt(a[:, k].var() / n + b[:, k].var() / n)
        assert abs(a[:, k].mean() - b[:, k].mean()) < 5 * se + 1e-9, (k, a[:, k].mean(), b[:, k].mean(), se)


def test_fd_estimator_is_difference_of_same_seed_gradients(oracle_lib):
    """Eq. est_triv: <dF_i> uses the same random numbers at both parameter vectors; with
    identical parameters it is exactly zero, and it is antisymmetric in the pair."""
    w = synth.workload_box(8, 8, 8, max_depth=3)
    sc = orc.Scene(w.scene)
    t0 = w.init_tex.astype(np.float64)
    t1 = t0 + 0.01 * np.random.default_rng(5).normal(size=t0.shape)
    tgt = np.full((8, 8, 3), 0.2)
    assert np.all(orc.fd_gradient(sc, t0, t0, tgt, 1, 2) == 0)
    d01 = orc.fd_gradient(sc, t1, t0, tgt, 1, 2)
    d10 = orc.fd_gradient(sc, t0, t1, tgt, 1, 2)
    assert np.array_equal(d01, -d10) and np.abs(d01).max() > 0


@pytest.mark.slow
def test_fd_estimator_unbiased(oracle_lib):
    """E[<dF_i>] = F(pi_i) - F(pi_{i-1}) (Sec. 3.1): the mean over seeds of the FD estimate
    matches the difference of two independently estimated mean gradients within 5 sigma."""
    w = synth.workload_box(4, 4, 4, max_depth=3)
    sc = orc.Scene(w.scene)
    t0 = w.init_tex.astype(np.float64)
    t1 = np.clip(t0 + 0.2 * np.random.default_rng(6).normal(size=t0.shape), 0.05, 0.95)
    tgt = np.full((4, 4, 3), 0.1)
    n = 200
    d = np.stack([orc.fd_gradient(sc, t1, t0, tgt, 1, s) for s in range(n)])
    g1 = np.stack([orc.prop_gradient(sc, t1, tgt, 1, 10_000 + s)[0] for s in range(n)])
    g0 = np.stack([orc.prop_gradient(sc, t0, tgt, 1, 20_000 + s)[0] for s in range(n)])
    diff = d.mean(0) - (g1.mean(0) - g0.mean(0))
    se = np.sqrt(d.var(0) / n + g1.var(0) / n + g0.var(0) / n) + 1e-12
    z = np.abs(diff) / se
    assert np.mean(z < 5) > 0.99 and np.var(d, 0).mean() < (np.var(g1, 0) + np.var(g0, 0)).mean()


def test_shared_path_branch_reduces_to_the_ordinary_estimator(oracle_lib):
    """Sampling and evaluating with the same parameters is the ordinary estimator (bit for bit)."""
    w = synth.workload_spiral(6, 5, 32, 8, 8, max_depth=4)
    sc = orc.Scene(w.scene)
    tex = w.init_tex.astype(np.float64)
    dimg = np.random.default_rng(7).normal(size=(5, 6, 3))
    assert np.array_equal(orc.render_image_shared(sc, tex, tex, 2, 3, orc.ST_FD_PRIMAL),
                          orc.render_image(sc, tex, 2, 3, orc.ST_FD_PRIMAL))
    assert np.array_equal(orc.adjoint_image_shared(sc, tex, tex, 2, 3, orc.ST_FD_ADJ, dimg),
                          orc.adjoint_image(sc, tex, 2, 3, orc.ST_FD_ADJ, dimg))


def test_shared_path_equals_replay_on_lambertian_box(oracle_lib):
    """On the Lambertian box the sampling and every density are independent of the albedo, so the
    pi_{i-1} branch that shares the pi_i path is exactly the branch that replays the numbers."""
    w = synth.workload_box(8, 8, 8, max_depth=3)
    sc = orc.Scene(w.scene)
    a = w.init_tex.astype(np.float64)
    b = np.clip(a + np.random.default_rng(8).normal(0, 0.05, a.shape), 0.05, 0.95)
    dimg = np.random.default_rng(9).normal(size=(8, 8, 3))
    assert np.allclose(orc.render_image_shared(sc, a, b, 2, 1, orc.ST_FD_PRIMAL),
                       orc.render_image(sc, b, 2, 1, orc.ST_FD_PRIMAL), rtol=1e-13, atol=1e-15)
    assert np.allclose(orc.adjoint_image_shared(sc, a, b, 2, 1, orc.ST_FD_ADJ, dimg),
                       orc.adjoint_image(sc, b, 2, 1, orc.ST_FD_ADJ, dimg), rtol=1e-12, atol=1e-15)


def test_shared_path_branch_unbiased_on_glossy_scene(oracle_lib):
    """On the principled spiral the shared-path image of pi_{i-1} (paths and densities of pi_i)
    has the same expectation as the ordinary image of pi_{i-1}: means over seeds within 5 sigma."""
    w = synth.workload_spiral(4, 4, 32, 8, 4, max_depth=3)
    sc = orc.Scene(w.scene)
    a = w.init_tex.astype(np.float64)
    b = w.target_tex.astype(np.float64)
    n = 200
    x = np.array([orc.render_image_shared(sc, a, b, 1, s, orc.ST_EVAL) for s in range(n)])
    y = np.array([orc.render_image(sc, b, 1, s + 10_000, orc.ST_EVAL) for s in range(n)])
    se = np.sqrt(x.var(0) / n + y.var(0) / n) + 1e-12
    z = (x.mean(0) - y.mean(0)) / se
    assert np.all(np.abs(z) < 5), np.abs(z).max()
    assert np.mean(z * z) < 3

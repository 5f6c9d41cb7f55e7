"""Oracle meta-estimator / Moment2 / Adam against closed forms, invariants and a library Adam."""
import numpy as np
import pytest
import torch

from oracle import meta


def test_moment2_closed_form():
    """Start-up-corrected EMA: m2_n = sum_j (1-b) b^(n-j) x_j^2 / (1 - b^n)."""
    rng = np.random.default_rng(0)
    for b in (0.5, 0.9, 0.99):
        x = rng.normal(size=20)
        m2, cnt = 0.0, 0
        for n in range(1, 21):
            m2, cnt = meta.moment2_step(m2, cnt, x[n - 1], b)
            j = np.arange(1, n + 1)
            closed = np.sum((1 - b) * b ** (n - j) * x[:n] ** 2) / (1 - b ** n)
            assert np.isclose(m2, closed, rtol=1e-12)
        assert cnt == 20


def test_first_step_is_sign_step():
    """i = 0: alpha_{-1} = -inf clips alpha to 0, so <F_0>_M = <F_0>, Var = F^2 and
    dpi = -eta F / (|F| + eps)."""
    h = meta.Hyper(lr=0.01)
    F = np.array([0.3, -2.0, 1e-3, 0.0])
    st = meta.MetaState.zeros(F.shape)
    pi1, n2, alpha = meta.meta_update(np.zeros(4), F, np.zeros(4), st, h, 0.0)
    assert np.all(alpha == 0)
    assert np.allclose(st.mean, F) and np.allclose(st.var, F * F)
    assert np.allclose(pi1, -h.lr * F / (np.abs(F) + h.eps), rtol=1e-14)
    assert np.isclose(n2, np.sum(pi1 ** 2))


def test_perfect_average_closed_form():
    """|F_i| = c constant and dF = 0: Var[<F>] = c^2 for any decay, Var_dF = 0, so alpha_i = i/(i+1)
    (unclipped value equals the clip bound) and the meta-estimate is the running arithmetic mean
    of F_0..F_i with variance c^2/(i+1) (the 'perfect average' that Eq. alpha_clip bounds)."""
    rng = np.random.default_rng(1)
    c = 0.7
    h = meta.Hyper(lr=1e-3, beta_f=0.9, beta_d=0.5)
    st = meta.MetaState.zeros((50,))
    Fs = []
    pi = np.zeros(50)
    n2 = 0.0
    for i in range(30):
        F = c * rng.choice([-1.0, 1.0], size=50)
        Fs.append(F)
        pi, n2, alpha = meta.meta_update(pi, F, np.zeros(50), st, h, n2)
        assert np.allclose(alpha, i / (i + 1), rtol=1e-12)
        assert np.allclose(st.mean, np.mean(Fs, 0), rtol=1e-10, atol=1e-14)
        assert np.allclose(st.var, c * c / (i + 1), rtol=1e-10)


def test_telescoping_with_consistent_differences():
    """If dF_i = F_i - F_{i-1} exactly, Eq. recurrent_meta gives <F_i>_M = F_i for any alphas."""
    rng = np.random.default_rng(2)
    h = meta.Hyper(lr=1e-2)
    F_prev = rng.normal(size=64)
    st = meta.MetaState.zeros((64,))
    pi, n2 = np.zeros(64), 0.0
    pi, n2, _ = meta.meta_update(pi, F_prev, np.zeros(64), st, h, n2)
    for i in range(1, 25):
        F = F_prev + 0.3 * rng.normal(size=64)
        pi, n2, _ = meta.meta_update(pi, F, F - F_prev, st, h, n2)
        assert np.allclose(st.mean, F, rtol=1e-9, atol=1e-12)
        F_prev = F


def test_alpha_bounded_by_iteration():
    """Eq. alpha_clip_2 from alpha_{-1} = -inf implies Eq. alpha_clip: alpha_i <= 1 - 1/(i+1)."""
    rng = np.random.default_rng(3)
    h = meta.Hyper(lr=1e-2, beta_f=0.99, beta_d=0.9)
    st = meta.MetaState.zeros((256,))
    pi, n2 = np.zeros(256), 0.0
    for i in range(40):
        F = rng.normal(size=256) * rng.uniform(0.1, 3)
        dF = 0.05 * rng.normal(size=256) if i else np.zeros(256)
        pi, n2, alpha = meta.meta_update(pi, F, dF, st, h, n2)
        assert np.all(alpha <= 1 - 1 / (i + 1) + 1e-15) and np.all(alpha >= 0)


def test_weight_one_on_plain_estimator_is_adam_beta1_zero():
    """When Var[<dF>] dominates, alpha -> 0: the meta-estimate is the plain estimate, Var_M is the
    Moment2 of F, and the update equals Adam with beta1 = 0, beta2 = beta_F (torch.optim.Adam)."""
    rng = np.random.default_rng(4)
    h = meta.Hyper(lr=1e-2, beta_f=0.95, beta_d=0.5, eps=1e-8)
    n = 32
    pi = rng.normal(size=n)
    st = meta.MetaState.zeros((n,))
    p_t = torch.tensor(pi.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p_t], lr=h.lr, betas=(0.0, h.beta_f), eps=h.eps)
    n2 = 0.0
    for i in range(20):
        F = rng.normal(size=n)
        dF = 1e12 * np.ones(n) if i else np.zeros(n)     # enormous FD variance
        pi, n2, alpha = meta.meta_update(pi, F, dF, st, h, n2)
        opt.zero_grad()
        p_t.grad = torch.tensor(F)
        opt.step()
        assert np.all(alpha < 1e-20)
        assert np.allclose(pi, p_t.detach().numpy(), rtol=1e-9, atol=1e-12), i


def test_adam_matches_torch():
    rng = np.random.default_rng(5)
    h = meta.Hyper(lr=3e-3, beta1=0.9, beta2=0.999, eps=1e-8)
    n = 40
    pi = rng.normal(size=n)
    st = meta.AdamState.zeros((n,))
    p_t = torch.tensor(pi.copy(), dtype=torch.float64)
    p_t.requires_grad_(True)
    opt = torch.optim.Adam([p_t], lr=h.lr, betas=(h.beta1, h.beta2), eps=h.eps)
    for i in range(30):
        F = rng.normal(size=n) + 0.5
        pi, _ = meta.adam_update(pi, F, st, h)
        p_t.grad = torch.tensor(F)
        opt.step()
        assert np.allclose(pi, p_t.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_clamp_and_applied_step_norm():
    h = meta.Hyper(lr=0.5)
    st = meta.MetaState.zeros((4,))
    pi = np.array([0.1, 0.9, 0.5, 0.5])
    F = np.array([1.0, -1.0, 1.0, -1.0])
    pi1, n2, _ = meta.meta_update(pi, F, np.zeros(4), st, h, 0.0, lo=np.zeros(4), hi=np.ones(4))
    assert np.allclose(pi1, [0.0, 1.0, 0.0, 1.0], atol=1e-7)
    assert np.isclose(n2, np.sum((pi1 - pi) ** 2))


@pytest.mark.parametrize("method", ["meta", "adam"])
def test_exposition_toy_converges(method):
    """The exposition figure's toy: the rate of an exponential distribution is optimised so
    that the mean of 32 samples per iteration matches 2.0 under an L2 loss; the optimum rate
    is 0.5. Samples x = -ln(u)/lambda; the FD sample reuses the same u at lambda_{i-1}."""
    rng = np.random.default_rng(6)
    h = meta.Hyper(lr=0.02, beta_f=0.99, beta_d=0.9)
    lam = np.array([2.0])
    lam_prev = lam.copy()
    st = meta.MetaState.zeros((1,))
    ad = meta.AdamState.zeros((1,))
    n2 = 0.0

    def grad(l, u, v):
        y = -np.log1p(-v) / l            # independent samples for the loss residual
        # d/dl of x = -ln(1-u)/l is ln(1-u)/l^2 (samples u drive the gradient)
        return 2.0 * (y.mean() - 2.0) * np.mean(np.log1p(-u) / (l * l))

    for i in range(600):
        u, v = rng.random(32), rng.random(32)
        F = np.array([grad(lam[0], u, v)])
        if method == "meta":
            u2, v2 = rng.random(32), rng.random(32)
            dF = np.array([grad(lam[0], u2, v2) - grad(lam_prev[0], u2, v2)]) if i else np.zeros(1)
            lam_prev = lam.copy()
            lam, n2, _ = meta.meta_update(lam, F, dF, st, h, n2, lo=np.array([0.05]), hi=np.array([10.0]))
        else:
            lam, _ = meta.adam_update(lam, F, ad, h, lo=np.array([0.05]), hi=np.array([10.0]))
    assert abs(lam[0] - 0.5) < 0.05, lam


# ---- variants (module docstring of oracle.meta) ----

def test_per_element_uniform_steps_equal_global():
    """With every |pi_i - pi_{i-1}| equal to c, dF/|dpi_e| = sqrt(n) dF/||dpi|| and
    |dpi_e|^2 = ||dpi||^2 / n, so Var[<dF>] and every result coincide with the global norm."""
    rng = np.random.default_rng(21)
    n, c = 12, 0.003
    h = meta.Hyper(lr=0.01)
    F0, F1, dF1 = rng.normal(size=n), rng.normal(size=n), rng.normal(size=n) * 0.1
    pi0 = rng.uniform(0.3, 0.7, n)
    sg, sp = meta.MetaState.zeros((n,)), meta.MetaState.zeros((n,))
    # iteration 0 without FD, identical for both; then force a uniform previous step of size c
    meta.meta_update(pi0, F0, np.zeros(n), sg, h, 0.0)
    meta.meta_update(pi0, F0, np.zeros(n), sp, h, 0.0, flags=meta.PER_ELEMENT, pi_prev=pi0)
    sign = np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    pi1 = pi0 + sign * c
    a, _, al_a = meta.meta_update(pi1, F1, dF1, sg, h, n * c * c)
    b, _, al_b = meta.meta_update(pi1, F1, dF1, sp, h, n * c * c, flags=meta.PER_ELEMENT, pi_prev=pi0)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-15) and np.allclose(al_a, al_b, rtol=1e-12)
    assert np.allclose(sp.m2d, n * sg.m2d, rtol=1e-12)


def test_per_element_zero_step_keeps_var_d():
    """An element whose own previous step was zero keeps Var_D and adds Var[<dF>] = 0."""
    rng = np.random.default_rng(22)
    n = 6
    h = meta.Hyper()
    st = meta.MetaState.zeros((n,))
    st.iteration, st.count_f, st.count_d = 3, 3, 2
    st.m2f[:] = 1.0
    st.m2d[:] = 0.5
    st.alpha_prev[:] = 0.4
    pi_prev = rng.uniform(0.3, 0.7, n)
    pi = pi_prev.copy()
    pi[1::2] += 0.01                     # odd elements moved, even elements did not
    dF = rng.normal(size=n)
    var0 = st.var.copy()
    meta.meta_update(pi, rng.normal(size=n), dF, st, h, float(np.sum((pi - pi_prev) ** 2)),
                     flags=meta.PER_ELEMENT, pi_prev=pi_prev)
    assert np.all(st.m2d[0::2] == 0.5) and np.all(st.m2d[1::2] != 0.5)
    # even elements: var went through var += 0, then the varmeta recurrence only
    a = st.alpha_prev[0::2]
    m2f = st.m2f[0::2]
    assert np.allclose(st.var[0::2], a * a * var0[0::2] + (1 - a) ** 2 * m2f, rtol=1e-12)


def test_no_clip_iteration_zero_closed_form():
    """Without Eq. alpha_clip_2 the first alpha is m2f / (m2f + 1e-30) (the carried variance
    is 0), so <F_0>_M = alpha * 0 + (1 - alpha) F = (1e-30 / (F^2 + 1e-30)) F and the step is
    its (vanishing) multiple; with the clip alpha_0 = 0 and <F_0>_M = F."""
    F = np.array([0.5, -2.0, 1e-3])
    h = meta.Hyper(lr=0.1)
    st = meta.MetaState.zeros((3,))
    _, _, al = meta.meta_update(np.full(3, 0.5), F, np.zeros(3), st, h, 0.0, flags=meta.NO_CLIP)
    assert np.allclose(al, F * F / (F * F + 1e-30), rtol=1e-15)
    assert np.allclose(st.mean, (1e-30 / (F * F + 1e-30)) * F, rtol=1e-12)
    st2 = meta.MetaState.zeros((3,))
    _, _, al2 = meta.meta_update(np.full(3, 0.5), F, np.zeros(3), st2, h, 0.0)
    assert np.all(al2 == 0.0) and np.allclose(st2.mean, F)


def test_centred_two_samples_weighted_variance():
    """Start-up-corrected EMAs of x1, x2 weight them w1 = beta / (1 + beta), w2 = 1 / (1 + beta);
    the centred variance m2 - mu^2 is then w1 w2 (x1 - x2)^2."""
    beta = 0.7
    h = meta.Hyper(beta_f=beta)
    x1, x2 = np.array([0.3, -1.0]), np.array([1.1, 2.0])
    st = meta.MetaState.zeros((2,))
    pi = np.full(2, 0.5)
    meta.meta_update(pi, x1, np.zeros(2), st, h, 0.0, flags=meta.CENTRED)
    meta.meta_update(pi, x2, np.zeros(2), st, h, 0.0, flags=meta.CENTRED)
    w1, w2 = beta / (1 + beta), 1 / (1 + beta)
    assert np.allclose(st.mu_f, w1 * x1 + w2 * x2, rtol=1e-12)
    assert np.allclose(st.m2f - st.mu_f ** 2, w1 * w2 * (x1 - x2) ** 2, rtol=1e-10)


def test_growing_beta_weights_become_uniform():
    """With decays b_k = max(beta, k/(k+1)) the recurrence equals sum_k w_k x_k^2 with
    w_k = (1 - b_k) prod_{j>k} b_j / (1 - prod_j b_j); once k/(k+1) > beta the weights of the
    later samples are all 1/(n+1) of the mass, i.e. equal."""
    beta, n = 0.75, 12
    h = meta.Hyper(beta_f=beta)
    rng = np.random.default_rng(5)
    xs = rng.normal(size=(n, 1))
    st = meta.MetaState.zeros((1,))
    for k in range(n):
        meta.meta_update(np.full(1, 0.5), xs[k], np.zeros(1), st, h, 0.0, flags=meta.GROWING_BETA)
    b = np.array([max(beta, k / (k + 1.0)) for k in range(n)])
    w = np.array([(1 - b[k]) * np.prod(b[k + 1:]) for k in range(n)]) / (1 - np.prod(b))
    assert np.isclose(w.sum(), 1.0)
    assert np.allclose(st.m2f, np.sum(w[:, None] * xs ** 2, axis=0), rtol=1e-12)
    K = int(np.argmax(np.arange(n) / (np.arange(n) + 1.0) > beta))
    assert K > 0 and np.allclose(w[K - 1:], w[-1], rtol=1e-12)


def test_naive_adam_reduces_to_adam_on_meta_estimate():
    """At iteration 0 <F_0>_M = F (alpha_0 = 0), so the naive coupling's first step is Adam's
    first step on F; afterwards it is Adam run on the sequence of <F_i>_M."""
    rng = np.random.default_rng(9)
    n = 5
    h = meta.Hyper(lr=0.05)
    pi = rng.uniform(0.3, 0.7, n)
    st = meta.MetaState.zeros((n,))
    ad = meta.AdamState.zeros((n,))
    F0 = rng.normal(size=n)
    a, n2, _ = meta.meta_update(pi, F0, np.zeros(n), st, h, 0.0, flags=meta.NAIVE_ADAM)
    b, _ = meta.adam_update(pi, F0, ad, h)
    assert np.allclose(a, b, rtol=1e-13)
    F1, dF1 = rng.normal(size=n), rng.normal(size=n) * 0.1
    a2, _, _ = meta.meta_update(a, F1, dF1, st, h, n2, flags=meta.NAIVE_ADAM)
    b2, _ = meta.adam_update(b, st.mean, ad, h)
    assert np.allclose(a2, b2, rtol=1e-13)


def test_uncorrelated_variance_samples():
    """The variances follow F_var, dF_var only: with F_var = F and dF_var = dF the variant is the
    default; with other F_var, m2f is that of a default run on F_var while <F>_M still uses F."""
    rng = np.random.default_rng(13)
    n = 7
    h = meta.Hyper()
    pi = rng.uniform(0.3, 0.7, n)
    F, Fv = rng.normal(size=n), rng.normal(size=n)
    s0, s1, s2 = (meta.MetaState.zeros((n,)) for _ in range(3))
    a, _, _ = meta.meta_update(pi, F, np.zeros(n), s0, h, 0.0)
    b, _, _ = meta.meta_update(pi, F, np.zeros(n), s1, h, 0.0, flags=meta.UNCORRELATED, F_var=F, dF_var=np.zeros(n))
    assert np.array_equal(a, b)
    meta.meta_update(pi, F, np.zeros(n), s2, h, 0.0, flags=meta.UNCORRELATED, F_var=Fv, dF_var=np.zeros(n))
    s3 = meta.MetaState.zeros((n,))
    meta.meta_update(pi, Fv, np.zeros(n), s3, h, 0.0)
    assert np.allclose(s2.m2f, s3.m2f) and np.allclose(s2.mean, F)


@pytest.mark.parametrize("clip", [True, False])
def test_meta_variance_recurrence_matches_monte_carlo(clip):
    """Eq. varmeta against simulation: each element is an independent trial of a drifting target
    theta_i, with F_i = theta_i + N(0, sF^2) and dF_i = theta_i - theta_{i-1} + N(0, sD^2), all
    noises independent. Fed the true variances, the recurrence's Var must equal the empirical
    variance of <F_i>_M - theta_i over the trials, the estimate must be unbiased, and the weight
    (unclipped) must be the one that minimises that variance. Iteration 0 takes the clip in both
    cases (alpha_0 = 0: the zero initial state carries no information)."""
    rng = np.random.default_rng(31)
    n, iters = 400_000, 6
    sF2, sD2 = 1.0, 0.09
    h = meta.Hyper()
    st = meta.MetaState.zeros((n,))
    theta = np.zeros(n)
    for i in range(iters):
        theta_prev = theta
        theta = theta_prev + 0.3 * np.sin(i + 1.0)
        F = theta + rng.normal(0.0, np.sqrt(sF2), n)
        dF = (theta - theta_prev + rng.normal(0.0, np.sqrt(sD2), n)) if i > 0 else np.zeros(n)
        var_d = np.full(n, sD2 if i > 0 else 0.0)
        mean_prev, var_prev = st.mean.copy(), st.var.copy()
        meta.meta_combine(st, F, dF, np.full(n, sF2), var_d, h, clip=clip or i == 0)
        err = st.mean - theta
        emp = err.var()
        assert abs(err.mean()) <= 5.0 * np.sqrt(emp / n), (i, err.mean())
        assert abs(emp - st.var[0]) <= 5.0 * np.sqrt(2.0 / n) * st.var[0], (i, emp, st.var[0])
        if i > 0 and not clip:
            # the same draws recombined with other weights give a larger empirical variance
            a = st.alpha_prev[0]
            for da in (-0.1, 0.1):
                b = a + da
                other = b * (mean_prev + dF) + (1.0 - b) * F - theta
                assert other.var() > emp
            assert np.isclose(a, sF2 / (sF2 + var_prev[0] + sD2), rtol=1e-12)

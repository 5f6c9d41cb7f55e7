"""FP64 meta-estimator and Adam updates (numpy).

TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the benchmark's
CPU-baseline leg; never by the product path.

Follows, step by step and in the paper's order:
  - the zero-centred second-moment EMA with start-up correction (appendix
    pseudocode "Moment2"; Eq. varest for Var[<F_i>], the EMA of Sec. 4.2 for the
    decoupled Var[<dF_i>]_D);
  - the rescaling Var[<dF_i>] = Var_D * ||dpi_i||^2 (Eq. vardiff);
  - the meta-estimator recurrence (Eq. recurrent_meta), its inverse-variance weight
    (Eq. alpha, with 1e-30 added to the denominator), the clipping rule of
    Eq. alpha_clip_2 starting from alpha_{-1} = -inf, and the variance recurrence
    (Eq. varmeta) (appendix pseudocode "Meta");
  - the update rule of Sec. 5 that replaces Adam's moments:
    dpi_{i+1} = -eta <F_i>_M / (sqrt(Var[<F_i>_M]) + eps);
  - Adam (Sec. 5, Eqs. adam_moment, adam_ema_startup, adam_step) with a first
    moment beta1 and bias correction of both moments (Kingma & Ba 2014).

Readings where the paper is silent (each also listed in the design notes):
  - iteration 0 has no previous parameters: <dF_0> = 0 and the Var_D EMA is not
    stepped; the same holds for any iteration whose previous step was exactly zero;
  - ||dpi_i|| is the Euclidean norm of the applied (post-clamp) step of the whole
    problem's parameter vector;
  - after the step, parameters are clamped channel-wise to their valid range.

Variants (bit flags; Sec. 4.2 for the norm, the ablation paragraphs of Sec. 6 and
the appendix on start-up bias for the rest):
  PER_ELEMENT   ||dpi_i|| read per element as |pi_i - pi_{i-1}| (the appendix loop
                writes sqrt(dpi_i^2)); an element whose own step was zero keeps its
                Var_D and contributes Var[<dF>] = 0;
  NO_CLIP       Eq. alpha_clip_2 is not applied (the "alpha clipping" ablation);
  CENTRED       non-zero-centred variances: a start-up-corrected EMA of the sample
                itself, mu, is kept beside each Moment2 and the variance is
                max(m2 - mu^2, 0) (the "zero-centred EMAs" ablation);
  GROWING_BETA  beta_F grows over the run as beta_{F,k} = max(beta_F, k / (k + 1))
                for the k-th Var[<F>] step (k = 0, 1, ...), with the start-up
                correction (1 - beta_k) / (1 - prod_{j<=k} beta_j) (appendix A);
  NAIVE_ADAM    <F_i>_M is fed to Adam's moments (beta1, beta2, bias-corrected)
                instead of the update rule of Sec. 5 (the naive coupling of Sec. 5);
  UNCORRELATED  Var[<F>] and Var[<dF>]_D are stepped with independent samples
                F_var, dF_var of the same estimators (the "sample reuse" ablation),
                while <F_i>_M still combines F and dF.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Hyper:
    lr: float = 0.01
    beta_f: float = 0.99      # Moment2 decay for Var[<F>]
    beta_d: float = 0.9       # Moment2 decay for Var[<dF>]_D
    eps: float = 1e-8         # step epsilon
    eps_alpha: float = 1e-30  # added to the alpha denominator
    beta1: float = 0.9        # Adam
    beta2: float = 0.999      # Adam


PER_ELEMENT = 1
NO_CLIP = 2
CENTRED = 4
GROWING_BETA = 8
NAIVE_ADAM = 16
UNCORRELATED = 32


def moment2_step(m2, count, x, decay):
    """One start-up-corrected zero-centred EMA step; returns (m2, count)."""
    count = count + 1
    w = 1.0 - decay
    w_sum = 1.0 - decay ** count
    return m2 + (w / w_sum) * (x * x - m2), count


def growing_decay(beta, k):
    """beta_{F,k} of the GROWING_BETA variant for the k-th step (k = 0, 1, ...)."""
    return max(beta, k / (k + 1.0))


@dataclass
class MetaState:
    m2f: np.ndarray
    m2d: np.ndarray
    mean: np.ndarray
    var: np.ndarray
    alpha_prev: np.ndarray
    count_f: int = 0
    count_d: int = 0
    iteration: int = 0
    # variant state: CENTRED first moments, NAIVE_ADAM moments, GROWING_BETA decay product
    mu_f: np.ndarray = None
    mu_d: np.ndarray = None
    adam_m: np.ndarray = None
    adam_v: np.ndarray = None
    prod_f: float = 1.0

    @staticmethod
    def zeros(shape):
        z = lambda: np.zeros(shape, np.float64)
        return MetaState(z(), z(), z(), z(), np.full(shape, -np.inf), mu_f=z(), mu_d=z(), adam_m=z(), adam_v=z())

    def copy(self):
        c = lambda a: None if a is None else a.copy()
        return MetaState(self.m2f.copy(), self.m2d.copy(), self.mean.copy(), self.var.copy(),
                         self.alpha_prev.copy(), self.count_f, self.count_d, self.iteration,
                         c(self.mu_f), c(self.mu_d), c(self.adam_m), c(self.adam_v), self.prod_f)


def meta_combine(st: MetaState, F, dF, var_f, var_d, h: Hyper, clip=True):
    """The 'Meta.step' of the appendix: returns dpi and the alpha used (state updated in place)."""
    st.mean = st.mean + dF
    st.var = st.var + var_d
    alpha = var_f / (var_f + st.var + h.eps_alpha)
    if clip:
        alpha = np.minimum(alpha, 1.0 / (2.0 - st.alpha_prev))
    st.alpha_prev = alpha
    st.mean = alpha * st.mean + (1.0 - alpha) * F
    st.var = alpha ** 2 * st.var + (1.0 - alpha) ** 2 * var_f
    return -h.lr * st.mean / (np.sqrt(st.var) + h.eps), alpha


def meta_update(pi, F, dF, st: MetaState, h: Hyper, dpi_norm2: float, lo=None, hi=None, flags=0,
                pi_prev=None, F_var=None, dF_var=None):
    """One optimisation step of the appendix loop snippet.

    pi, F, dF: parameter-shaped float64 arrays; st: state (updated in place);
    dpi_norm2: ||pi_i - pi_{i-1}||^2 of the step that produced pi (0 at iteration 0).
    lo/hi: per-channel clamp bounds broadcast against the last axis.
    flags: variant bits (module docstring); pi_prev (= pi_{i-1}) is needed by
    PER_ELEMENT, F_var and dF_var by UNCORRELATED.
    Returns (pi_next, dpi_norm2_next, alpha).
    """
    F = np.asarray(F, np.float64)
    dF = np.asarray(dF, np.float64)
    xF = np.asarray(F_var, np.float64) if flags & UNCORRELATED else F
    xD = np.asarray(dF_var, np.float64) if flags & UNCORRELATED else dF
    # Var[<F_i>]: Eq. varest as the start-up-corrected Moment2 (decay fixed or growing)
    if flags & GROWING_BETA:
        b = growing_decay(h.beta_f, st.count_f)
        st.prod_f *= b
        cF = (1.0 - b) / (1.0 - st.prod_f)
        st.m2f = st.m2f + cF * (xF * xF - st.m2f)
        st.count_f += 1
    else:
        cF = (1.0 - h.beta_f) / (1.0 - h.beta_f ** (st.count_f + 1))
        st.m2f, st.count_f = moment2_step(st.m2f, st.count_f, xF, h.beta_f)
    var_f = st.m2f
    if flags & CENTRED:
        st.mu_f = st.mu_f + cF * (xF - st.mu_f)
        var_f = np.maximum(st.m2f - st.mu_f * st.mu_f, 0.0)
    # Var[<dF_i>]: the decoupled EMA of Sec. 4.2 rescaled by the step size (Eq. vardiff)
    have_fd = st.iteration >= 1 and dpi_norm2 > 0.0
    if have_fd:
        cD = (1.0 - h.beta_d) / (1.0 - h.beta_d ** (st.count_d + 1))
        st.count_d += 1
        if flags & PER_ELEMENT:
            d2 = (np.asarray(pi, np.float64) - np.asarray(pi_prev, np.float64)) ** 2
            live = d2 > 0.0
            x = np.where(live, xD / np.sqrt(np.where(live, d2, 1.0)), 0.0)
        else:
            d2 = np.full_like(F, dpi_norm2)
            live = np.ones(F.shape, bool)
            x = xD / np.sqrt(dpi_norm2)
        st.m2d = np.where(live, st.m2d + cD * (x * x - st.m2d), st.m2d)
        var_dd = st.m2d
        if flags & CENTRED:
            st.mu_d = np.where(live, st.mu_d + cD * (x - st.mu_d), st.mu_d)
            var_dd = np.maximum(st.m2d - st.mu_d * st.mu_d, 0.0)
        var_d = var_dd * d2
        dF_used = dF
    else:
        var_d = np.zeros_like(F)
        dF_used = np.zeros_like(F)
    dpi, alpha = meta_combine(st, F, dF_used, var_f, var_d, h, clip=not (flags & NO_CLIP))
    if flags & NAIVE_ADAM:
        # <F_i>_M into Adam's moments (Eqs. adam_moment, adam_ema_startup, adam_step)
        t = st.iteration + 1
        st.adam_m = h.beta1 * st.adam_m + (1.0 - h.beta1) * st.mean
        st.adam_v = h.beta2 * st.adam_v + (1.0 - h.beta2) * st.mean * st.mean
        dpi = -h.lr * (st.adam_m / (1.0 - h.beta1 ** t)) / (np.sqrt(st.adam_v / (1.0 - h.beta2 ** t)) + h.eps)
    pi_next = np.asarray(pi, np.float64) + dpi
    if lo is not None:
        pi_next = np.minimum(np.maximum(pi_next, lo), hi)
    st.iteration += 1
    step = pi_next - np.asarray(pi, np.float64)
    return pi_next, float(np.sum(step * step)), alpha


@dataclass
class AdamState:
    m: np.ndarray
    v: np.ndarray
    iteration: int = 0

    @staticmethod
    def zeros(shape):
        return AdamState(np.zeros(shape), np.zeros(shape))


def adam_update(pi, F, st: AdamState, h: Hyper, lo=None, hi=None):
    """Adam with bias-corrected first and second moments; returns (pi_next, dpi_norm2_next)."""
    F = np.asarray(F, np.float64)
    t = st.iteration + 1
    st.m = h.beta1 * st.m + (1.0 - h.beta1) * F
    st.v = h.beta2 * st.v + (1.0 - h.beta2) * F * F
    m_hat = st.m / (1.0 - h.beta1 ** t)
    v_hat = st.v / (1.0 - h.beta2 ** t)
    pi_next = np.asarray(pi, np.float64) - h.lr * m_hat / (np.sqrt(v_hat) + h.eps)
    if lo is not None:
        pi_next = np.minimum(np.maximum(pi_next, lo), hi)
    st.iteration = t
    step = pi_next - np.asarray(pi, np.float64)
    return pi_next, float(np.sum(step * step))

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


def moment2_step(m2, count, x, decay):
    """One start-up-corrected zero-centred EMA step; returns (m2, count)."""
    count = count + 1
    w = 1.0 - decay
    w_sum = 1.0 - decay ** count
    return m2 + (w / w_sum) * (x * x - m2), count


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

    @staticmethod
    def zeros(shape):
        z = lambda: np.zeros(shape, np.float64)
        return MetaState(z(), z(), z(), z(), np.full(shape, -np.inf))

    def copy(self):
        return MetaState(self.m2f.copy(), self.m2d.copy(), self.mean.copy(), self.var.copy(),
                         self.alpha_prev.copy(), self.count_f, self.count_d, self.iteration)


def meta_combine(st: MetaState, F, dF, var_f, var_d, h: Hyper):
    """The 'Meta.step' of the appendix: returns dpi and the alpha used (state updated in place)."""
    st.mean = st.mean + dF
    st.var = st.var + var_d
    alpha = var_f / (var_f + st.var + h.eps_alpha)
    alpha = np.minimum(alpha, 1.0 / (2.0 - st.alpha_prev))
    st.alpha_prev = alpha
    st.mean = alpha * st.mean + (1.0 - alpha) * F
    st.var = alpha ** 2 * st.var + (1.0 - alpha) ** 2 * var_f
    return -h.lr * st.mean / (np.sqrt(st.var) + h.eps), alpha


def meta_update(pi, F, dF, st: MetaState, h: Hyper, dpi_norm2: float, lo=None, hi=None):
    """One optimisation step of the appendix loop snippet.

    pi, F, dF: parameter-shaped float64 arrays; st: state (updated in place);
    dpi_norm2: ||pi_i - pi_{i-1}||^2 of the step that produced pi (0 at iteration 0).
    lo/hi: per-channel clamp bounds broadcast against the last axis.
    Returns (pi_next, dpi_norm2_next, alpha).
    """
    F = np.asarray(F, np.float64)
    dF = np.asarray(dF, np.float64)
    st.m2f, st.count_f = moment2_step(st.m2f, st.count_f, F, h.beta_f)
    have_fd = st.iteration >= 1 and dpi_norm2 > 0.0
    if have_fd:
        st.m2d, st.count_d = moment2_step(st.m2d, st.count_d, dF / np.sqrt(dpi_norm2), h.beta_d)
        var_d = st.m2d * dpi_norm2
        dF_used = dF
    else:
        var_d = np.zeros_like(F)
        dF_used = np.zeros_like(F)
    dpi, alpha = meta_combine(st, F, dF_used, st.m2f, var_d, h)
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

"""FP64 gradient preconditioning of texture gradients (numpy / scipy).

TEST INFRASTRUCTURE ONLY: used by tests and the benchmark's CPU-baseline leg; never by the
product path.

The experiments of Sec. 6 precondition texture gradients after Nicolet et al. 2021: per channel
g <- (I + lambda L)^{-1} g, L the graph Laplacian of the W x H texel grid with Neumann boundary,
(L x)_p = sum over the grid neighbours q of p of (x_p - x_q). The solve uses the orthonormal
DCT-II, in which L is diagonal with eigenvalues (2 - 2 cos(pi k / W)) + (2 - 2 cos(pi l / H))
(scipy.fft as the library step); `laplacian` is the plain stencil the tests check it against.
"""
from __future__ import annotations

import numpy as np
from scipy.fft import dctn, idctn


def laplacian(x):
    """Neumann graph Laplacian of a 2-D grid (stencil, no transform)."""
    y = np.zeros_like(x)
    d = x[:, 1:] - x[:, :-1]
    y[:, 1:] += d
    y[:, :-1] -= d
    d = x[1:, :] - x[:-1, :]
    y[1:, :] += d
    y[:-1, :] -= d
    return y


def precondition(g, lam):
    """(I + lam L)^{-1} applied to each channel of an (H, W, C) gradient."""
    g = np.asarray(g, np.float64)
    H, W = g.shape[:2]
    mu = (2.0 - 2.0 * np.cos(np.pi * np.arange(W) / W))[None, :] + (2.0 - 2.0 * np.cos(np.pi * np.arange(H) / H))[:, None]
    out = np.empty_like(g)
    for c in range(g.shape[2]):
        out[..., c] = idctn(dctn(g[..., c], type=2, norm="ortho") / (1.0 + lam * mu), type=2, norm="ortho")
    return out

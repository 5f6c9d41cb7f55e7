"""Oracle gradient preconditioner against the stencil it inverts."""
import numpy as np

from oracle import precond


def test_solves_the_stencil_system():
    """(I + lam L) x = g to rounding for the plain Neumann stencil, on non-square grids."""
    rng = np.random.default_rng(0)
    for H, W, lam in ((8, 16, 3.0), (32, 32, 25.0), (5, 7, 0.5)):
        g = rng.normal(size=(H, W, 3))
        x = precond.precondition(g, lam)
        for c in range(3):
            r = x[..., c] + lam * precond.laplacian(x[..., c]) - g[..., c]
            assert np.abs(r).max() <= 1e-11 * np.abs(g).max()


def test_identity_constant_and_channels():
    rng = np.random.default_rng(1)
    g = rng.normal(size=(6, 9, 5))
    assert np.allclose(precond.precondition(g, 0.0), g, atol=1e-14)
    const = np.full((6, 9, 2), 0.75)
    assert np.allclose(precond.precondition(const, 10.0), const, atol=1e-14)   # L has constants in its kernel
    a = precond.precondition(g, 4.0)
    b = precond.precondition(g[..., 2:3], 4.0)
    assert np.allclose(a[..., 2:3], b, atol=1e-15)
    # smoothing: the preconditioned gradient has less energy at high frequencies
    assert np.sum(precond.laplacian(a[..., 0]) ** 2) < np.sum(precond.laplacian(g[..., 0]) ** 2)

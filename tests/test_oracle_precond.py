"""Oracle gradient preconditioner against the stencil it inverts."""
import numpy as np
import pytest

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


def test_matches_the_grid_graph_laplacian_of_a_graph_library():
    """L is the graph Laplacian D - A of the W x H grid graph (4-neighbour, Neumann boundary =
    no edges leaving the grid): built here by networkx, independently of the oracle, then the
    system (I + lam L) x = g solved by a sparse direct solver."""
    nx = pytest.importorskip("networkx")
    from scipy.sparse import identity
    from scipy.sparse.linalg import spsolve
    rng = np.random.default_rng(2)
    for H, W, lam in ((5, 7, 2.0), (9, 4, 11.0)):
        G = nx.grid_2d_graph(H, W)
        order = [(y, x) for y in range(H) for x in range(W)]       # row-major texels
        Lg = nx.laplacian_matrix(G, nodelist=order).astype(np.float64).tocsc()
        g = rng.normal(size=(H, W, 2))
        for c in range(2):
            v = g[..., c].reshape(-1)
            assert np.allclose(precond.laplacian(g[..., c]).reshape(-1), Lg @ v, rtol=0, atol=1e-13)
            x = spsolve((identity(H * W, format="csc") + lam * Lg), v)
            assert np.allclose(precond.precondition(g, lam)[..., c].reshape(-1), x, rtol=0, atol=1e-11)

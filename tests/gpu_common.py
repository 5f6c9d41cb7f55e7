"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    return torch


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def frac_within(a, ref, rtol, atol):
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.mean(np.abs(a - ref) <= rtol * np.abs(ref) + atol))


def params_match(a, b, frac=0.999, atol=1e-5, cap=0.1):
    """Parameters of two runs that differ only in the order of float reductions (gradients
    accumulate with float atomics, and the dynamic ray fetching reorders records): at least `frac`
    of them within `atol`, none further apart than `cap`. A texel whose samples cancel to within a
    rounding of zero can take a full normalised step in one run and none in the other, so a bound
    on every element would test the rounding, not the method."""
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))
    return float(np.mean(d <= atol)) >= frac and float(d.max()) <= cap

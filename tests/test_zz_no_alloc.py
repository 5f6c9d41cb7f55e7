"""The allocation-free update entry point (mer_meta_step_raw_noalloc), called through the C ABI,
gives the same results as mer_meta_step_raw on identical inputs, on two calls in a row.

It exists for callers that may not allocate device memory (applications that hand out all device
memory through their own pool, real-time loops that may not allocate or synchronise); its scratch
is a fixed array inside the library. This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import ctypes as ct

import pytest

from .gpu_common import need_gpu

pytestmark = pytest.mark.gpu

N, C = 50001, 5        # ragged: not a multiple of 4, several blocks


def _state(torch, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    r = lambda *s: torch.rand(*s, generator=g)
    st = dict(pi=0.05 + 0.9 * r(N), F=(r(N) - 0.5) * 0.02, dF=(r(N) - 0.5) * 0.006, m2f=(r(N) * 0.01) ** 2,
              m2d=(r(N) * 0.1) ** 2, mean=(r(N) - 0.5) * 0.02, var=(r(N) * 0.01) ** 2, ap=r(N) * 0.8)
    return {k: v.float().cuda() for k, v in st.items()}


def _call(L, fn, torch, st, nxt, out, it, cf, cd, n2):
    from paper_2309_15676_gb300 import _lib
    h = _lib.Hyper(0, 0.01, 0.99, 0.9, 1e-8, 1e-30, 0.9, 0.999)
    lo = (ct.c_float * 8)(0, 0, 0, 0, 0.05, 0, 0, 0)
    hi = (ct.c_float * 8)(1, 1, 1, 1, 1, 0, 0, 0)
    p = lambda t: ct.c_void_p(t.data_ptr())
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    return getattr(L, fn)(ct.byref(h), N, C, lo, hi, p(st["pi"]), p(nxt), p(st["F"]), p(st["dF"]), p(st["m2f"]),
                          p(st["m2d"]), p(st["mean"]), p(st["var"]), p(st["ap"]), it, cf, cd, n2, 1, p(out), stream)


def test_noalloc_matches_allocating_entry_point_twice():
    torch = need_gpu()
    from paper_2309_15676_gb300 import _lib
    L = _lib.load()
    a, b = _state(torch, 1), _state(torch, 1)
    na, nb = torch.empty_like(a["pi"]), torch.empty_like(b["pi"])
    oa = torch.zeros(1, dtype=torch.float64, device="cuda")
    ob = torch.zeros(1, dtype=torch.float64, device="cuda")
    n2 = 2.5e-5
    for call in range(2):
        # fresh gradients for this call (the previous call cleared them)
        g = torch.Generator(device="cpu").manual_seed(10 + call)
        F = ((torch.rand(N, generator=g) - 0.5) * 0.02).cuda()
        dF = ((torch.rand(N, generator=g) - 0.5) * 0.006).cuda()
        for s in (a, b):
            s["F"].copy_(F)
            s["dF"].copy_(dF)
        assert _call(L, "mer_meta_step_raw", torch, a, na, oa, 3 + call, 3 + call, 2 + call, n2) == 0
        assert _call(L, "mer_meta_step_raw_noalloc", torch, b, nb, ob, 3 + call, 3 + call, 2 + call, n2) == 0, \
            L.mer_last_error(None)
        torch.cuda.synchronize()
        for k in ("m2f", "m2d", "mean", "var", "ap", "F", "dF"):
            x, y = a[k].double(), b[k].double()
            assert torch.allclose(y, x, rtol=1e-5, atol=1e-12), (call, k)
        assert torch.allclose(nb.double(), na.double(), rtol=1e-5, atol=1e-12), call
        assert abs(ob.item() - oa.item()) <= 1e-5 * abs(oa.item()), (call, ob.item(), oa.item())
        n2 = oa.item()
        a["pi"], na = na, a["pi"]
        b["pi"], nb = nb, b["pi"]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = need_gpu()
    from paper_2309_15676_gb300 import _lib
    L = _lib.load()
    s = _state(torch, 2)
    nxt = torch.empty_like(s["pi"])
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    h = _lib.Hyper(0, 0.01, 0.99, 0.9, 1e-8, 1e-30, 0.9, 0.999)
    lo = (ct.c_float * 8)(*([0.0] * 8))
    hi = (ct.c_float * 8)(*([1.0] * 8))
    p = lambda t: ct.c_void_p(t.data_ptr())
    too_many = 268435456 + 1          # validated before any device work; arrays are never touched
    st = L.mer_meta_step_raw_noalloc(ct.byref(h), too_many, C, lo, hi, p(s["pi"]), p(nxt), p(s["F"]), p(s["dF"]),
                                     p(s["m2f"]), p(s["m2d"]), p(s["mean"]), p(s["var"]), p(s["ap"]), 1, 1, 0, 0.0,
                                     1, p(out), ct.c_void_p(0))
    assert st == 1 and b"exceeds" in L.mer_last_error(None)

"""Philox4x32-10 (Salmon et al. 2011) of the library against the CUDA library's own
Philox4_32_10 device generator (curand_kernel.h), an implementation independent of both the
library and the oracle: the first draw of subsequence i under a 64-bit seed is Philox of one
128-bit counter under the seed's two 32-bit halves. The test finds which of the candidate
key/counter conventions the generator uses from the first draws and then requires every one of
4096 draws to match bit for bit."""
import ctypes as ct
import os
import shutil
import subprocess

import numpy as np
import pytest

from .gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def _build(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = os.path.join(os.path.dirname(__file__), "curand_philox_ref.cu")
    so = str(tmp_path / "libcurandref.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    src, "-o", so], check=True)
    return ct.CDLL(so)


def test_philox_matches_curand(tmp_path):
    torch = need_gpu()
    from paper_2309_15676_gb300.api import philox
    lib = _build(tmp_path)
    lib.ref_curand_philox.argtypes = [ct.c_ulonglong, ct.c_int, ct.c_void_p]
    n = 4096
    seed = 0x9E3779B97F4A7C15
    ref = np.zeros((n, 4), np.uint32)
    assert lib.ref_curand_philox(seed, n, ref.ctypes.data) == 0
    k0, k1 = seed & 0xFFFFFFFF, seed >> 32
    i = np.arange(n, dtype=np.uint64)
    lo, hi = (i & 0xFFFFFFFF).astype(np.uint32), (i >> 32).astype(np.uint32)
    z = np.zeros(n, np.uint32)
    conventions = {"(0,0,sub_lo,sub_hi)": np.stack([z, z, lo, hi], 1), "(sub_lo,sub_hi,0,0)": np.stack([lo, hi, z, z], 1)}
    matched = []
    for name, ctr in conventions.items():
        got = philox(k0, k1, torch.from_numpy(ctr.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
        if np.array_equal(got[:8], ref[:8]):
            matched.append(name)
            assert np.array_equal(got, ref), name
    assert len(matched) == 1, matched

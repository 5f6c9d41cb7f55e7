"""The fused update's per-iteration coefficients (start-up corrections of both Moment2 EMAs, Adam's
bias corrections, 1/||dpi||, the growing-beta start-up correction) as the library computes them
(update_coef, a host/device function), compiled for the host with nvcc and run on the CPU, against
the oracle's definitions: (1 - beta) / (1 - beta^(count + 1)) for Moment2 (appendix pseudocode),
1 / (1 - beta^t) for Adam, and for GROWING_BETA (1 - beta_k) / (1 - prod_{j<=k} beta_j) with the
product taken step by step over the oracle's growing_decay."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import meta

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2309_15676_gb300", "csrc")

# (mode, beta_f, beta_d, beta1, beta2, flags, iteration, count_f, count_d, n2)
CASES = [
    (0, 0.99, 0.9, 0.9, 0.999, 0, 0, 0, 0, 0.0),
    (0, 0.99, 0.9, 0.9, 0.999, 0, 1, 1, 0, 2.5e-3),
    (0, 0.99, 0.9, 0.9, 0.999, 0, 7, 7, 6, 1e-4),
    (0, 0.99, 0.9, 0.9, 0.999, 0, 999, 999, 998, 3.0),
    (0, 0.5, 0.95, 0.9, 0.999, 0, 40, 40, 12, 7e-7),
    (0, 0.99, 0.9, 0.9, 0.999, 8, 0, 0, 0, 0.0),       # GROWING_BETA
    (0, 0.99, 0.9, 0.9, 0.999, 8, 5, 5, 4, 1e-3),
    (0, 0.99, 0.9, 0.9, 0.999, 8, 98, 98, 97, 1e-3),
    (0, 0.99, 0.9, 0.9, 0.999, 8, 99, 99, 98, 1e-3),
    (0, 0.99, 0.9, 0.9, 0.999, 8, 100, 100, 99, 1e-3),
    (0, 0.99, 0.9, 0.9, 0.999, 8, 5000, 5000, 4999, 1e-3),
    (0, 0.9, 0.9, 0.9, 0.999, 8, 37, 37, 36, 1e-2),
    (1, 0.99, 0.9, 0.9, 0.999, 0, 0, 0, 0, 0.0),       # ADAM
    (1, 0.99, 0.9, 0.8, 0.99, 0, 12, 12, 0, 5e-2),
    (1, 0.99, 0.9, 0.9, 0.999, 0, 20000, 20000, 0, 1.0),
]

PROG = r'''
#include <cstdio>
#include "update.cuh"
int main() {
    int mode, flags, it, cf, cd; double bf, bd, b1, b2, n2;
    while (scanf("%d %lf %lf %lf %lf %d %d %d %d %lf", &mode, &bf, &bd, &b1, &b2, &flags, &it, &cf, &cd, &n2) == 10) {
        mer_hyper h{};
        h.mode = mode; h.beta_f = (float)bf; h.beta_d = (float)bd; h.beta1 = (float)b1; h.beta2 = (float)b2;
        h.flags = flags;
        const mer::UpdCoef k = mer::update_coef(h, it, cf, cd, n2);
        printf("%.9g %.9g %.9g %.9g %.9g %.9g %d\n", k.cF, k.cD, k.norm2, k.inv_norm, k.c1, k.c2, k.stepD);
    }
    return 0;
}
'''


def _reference(mode, bf, bd, b1, b2, flags, it, cf, cd, n2):
    bf, bd, b1, b2 = (float(np.float32(x)) for x in (bf, bd, b1, b2))   # the hyper-parameters are FP32
    t = it + 1
    c1, c2 = 1.0 / (1.0 - b1 ** t), 1.0 / (1.0 - b2 ** t)
    if mode == 1:
        return [0.0, 0.0, 0.0, 0.0, c1, c2, 0]
    if flags & meta.GROWING_BETA:
        prod = 1.0
        for j in range(cf + 1):
            prod *= meta.growing_decay(bf, j)
        cF = (1.0 - meta.growing_decay(bf, cf)) / (1.0 - prod)
    else:
        cF = (1.0 - bf) / (1.0 - bf ** (cf + 1))
    step_d = 1 if (it >= 1 and n2 > 0.0) else 0
    cD = (1.0 - bd) / (1.0 - bd ** (cd + 1)) if step_d else 0.0
    return [cF, cD, n2, (1.0 / np.sqrt(n2)) if step_d else 0.0, c1, c2, step_d]


def test_update_coefficients_match_definitions():
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "coef.cu")
        exe = os.path.join(d, "coef")
        open(src, "w").write(PROG)
        r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                            "-gencode", "arch=compute_103a,code=sm_103a", src, "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        inp = "\n".join(" ".join(str(x) for x in c) for c in CASES) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    out = [line for line in out if line.strip()]
    assert len(out) == len(CASES), out
    for case, line in zip(CASES, out):
        got = [float(x) for x in line.split()]
        ref = _reference(*case)
        assert got[6] == ref[6], (case, got, ref)
        for g, e in zip(got[:6], ref[:6]):
            assert abs(g - e) <= 2e-7 * abs(e) + 1e-30, (case, got, ref)

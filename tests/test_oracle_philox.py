"""Oracle Philox4x32-10 against the algorithm's published known answers and uniformity."""
import os

import numpy as np
from scipy import stats

from oracle import orc

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[:4], v[4:6], v[6:10]))
    return rows


def test_known_answers(oracle_lib):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert list(orc.philox(ctr, key)) == out


def test_counter_words_all_matter(oracle_lib):
    base = orc.philox([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert list(orc.philox(c, [5, 6])) != list(base)
    assert list(orc.philox([1, 2, 3, 4], [5, 7])) != list(base)


def test_uniformity_chi2(oracle_lib):
    n = 20000
    u = []
    for i in range(n // 4):
        o = orc.philox([i, 7, 3, (1 << 16) | (2 << 4)], [11, 0])
        u.extend(((o >> 8).astype(np.float64) * 2.0 ** -24).tolist())
    u = np.asarray(u)
    assert u.min() >= 0.0 and u.max() < 1.0
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    chi2, p = stats.chisquare(hist)
    assert p > 1e-4, (chi2, p)

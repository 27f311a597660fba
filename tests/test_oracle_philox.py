"""Pins of the oracle's counter-based generator (Philox4x32-10, Salmon et al. 2011).

The known-answer vectors in tests/golden/philox4x32_10_kat.txt were published
with the generator's definition; they fix every round constant, the word
permutation and the key schedule.  The uniform map (26 + 26 bits, +1/2) is
checked for its exact end points and for uniformity.
"""
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_known_answers(oracle):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = oracle.philox(ctr, key)
        assert [int(g) for g in got] == want


def test_u01_open_interval_and_exact_ends(oracle):
    lo = oracle.u01(0, 0)
    hi = oracle.u01(0xFFFFFFFF, 0xFFFFFFFF)
    assert lo == 0.5 * 2.0 ** -52
    assert hi == (2.0 ** 52 - 0.5) * 2.0 ** -52
    assert 0.0 < lo < hi < 1.0


def test_u01_uniform(oracle):
    key = [0x12345678, 0x9ABCDEF0]
    u = []
    for i in range(20000):
        w = oracle.philox([i, 7, 0, 0], key)
        u.append(oracle.u01(int(w[0]), int(w[1])))
        u.append(oracle.u01(int(w[2]), int(w[3])))
    u = np.array(u)
    assert abs(u.mean() - 0.5) < 5 * (1 / np.sqrt(12)) / np.sqrt(len(u))
    hist, _ = np.histogram(u, bins=20, range=(0, 1))
    expect = len(u) / 20
    chi2 = ((hist - expect) ** 2 / expect).sum()
    assert chi2 < 50.0          # 19 dof; p ~ 1e-4

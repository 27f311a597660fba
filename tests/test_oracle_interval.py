"""Pins of the oracle's interval controller (Sect. 2.5.3) against hand-computed toys."""
import numpy as np
import pytest

from paper_2609_35967_gb300 import workloads as W


def _P(oracle, **kw):
    d = dict(geometry=W.PATCH, K=32, eps=0.1, dt_coll=1e9, dt_fn_max=1e9, audit=1)
    d.update(kw)
    return oracle.params(d)


def test_fine_bins_exact_edges(oracle):
    # edges at 2^e {1/2, 2^(1/3)/2, 2^(2/3)/2}: a third of an octave per bin
    b0 = oracle.fine_bin(1.0)
    assert oracle.fine_bin(2.0) == b0 + 3
    assert oracle.fine_bin(2.0 ** (1 / 3) * 1.0000001) == b0 + 1
    assert oracle.fine_bin(2.0 ** (1 / 3) * 0.9999999) == b0
    assert oracle.fine_bin(np.nextafter(1.0, 0.0)) == b0 - 1
    assert oracle.fine_bin(1e-300) == 0
    assert oracle.fine_bin(1e300) == 95
    # ~0.1 dex per bin
    assert abs(np.log10(2.0) / 3 - 0.1) < 0.0004


def test_two_bin_toy(oracle):
    P = _P(oracle)
    st = oracle.new_state(P)
    n = 128
    s = np.where(np.arange(n) < 64, 1e-3, 1e-2)
    M = np.where(np.arange(n) % 2 == 0, 1.0, 3.0)
    # group 1 (small): mA alternates 1e-9 / 3e-9 with M 1 / 3 -> A_1 = (1e-9 + 9e-9)/4
    mA = np.where(np.arange(n) < 64, np.where(np.arange(n) % 2 == 0, 1e-9, 3e-9), 5e-9)
    mB = np.where(np.arange(n) < 64, 1e-9, 4e-10)
    grp, A, B = oracle.choose_interval(P, st, s, M, mA, mB, moments=True)
    assert st.n_groups == 2
    assert list(np.unique(grp[:64])) == [0] and list(np.unique(grp[64:])) == [1]
    A1, A2, B1, B2 = 2.5e-9, 5e-9, 1e-9, 4e-10
    # the controller-bin moments themselves: mass-weighted means of each bin
    assert A == pytest.approx([A1, A2], rel=1e-15) and B == pytest.approx([B1, B2], rel=1e-15)
    want = min(1e9, 0.1 / A1, 0.1 / A2, 0.01 / B1, 0.01 / B2)
    assert want == pytest.approx(1e7)
    assert st.dt_req == pytest.approx(want, rel=1e-14)
    assert st.dt_exe == 1e9 / 128            # 1e9/2^7 <= 1e7 < 1e9/2^6
    assert st.dt_remain == 1e9 - 1e9 / 128


def test_merging_and_remainder(oracle):
    P = _P(oracle)
    st = oracle.new_state(P)
    # 10 tiny, 100 small, 70 medium, 20 large: thresholds at 64 particles
    s = np.concatenate([np.full(10, 1e-4), np.full(100, 1e-3), np.full(70, 1e-2),
                        np.full(20, 1e-1)])
    n = len(s)
    grp = oracle.choose_interval(P, st, s, np.ones(n), np.zeros(n), np.zeros(n))
    # (10 + 100) >= 64 -> group 0; 70 -> group 1; the trailing 20 join group 1
    assert st.n_groups == 2
    assert set(grp[:110]) == {0} and set(grp[110:]) == {1}
    # no constraint from zero moments: dt_req = min(dt_remain, dt_fn_max)
    assert st.dt_exe == 1e9 and st.dt_remain == 1e9
    # a single small instance is one group
    st2 = oracle.new_state(P)
    oracle.choose_interval(P, st2, np.full(5, 1e-3), np.ones(5), np.ones(5), np.ones(5))
    assert st2.n_groups == 1


def test_remaining_time_and_halving(oracle):
    P = _P(oracle, dt_fn_max=1e9)
    st = oracle.new_state(P)
    n = 64
    s = np.full(n, 1e-3)
    # constrain to 0.3 dt_coll: executed 1/4, then remain 3/4 -> 1/4 ... until the step ends
    A = 0.1 / 3e8
    seq = []
    for _ in range(5):
        oracle.choose_interval(P, st, s, np.ones(n), np.full(n, A), np.zeros(n))
        seq.append((st.dt_exe, st.dt_remain))
    assert [e for e, _ in seq] == [2.5e8] * 5
    assert [r for _, r in seq] == [7.5e8, 5e8, 2.5e8, 1e9, 7.5e8]


def test_audit_rule(oracle):
    P = _P(oracle)
    st = oracle.new_state(P)
    n = 128
    M = np.ones(n)
    grp = np.where(np.arange(n) < 64, 0, 1).astype(np.int32)
    # realised mean |dln s| of group 1 = 0.25 > 2 eps C = 0.2 -> C halves
    js = np.where(grp == 1, 0.25, 0.0)
    oracle.audit(P, st, M, js, grp, 2)
    assert st.C == 0.5
    oracle.audit(P, st, M, js, grp, 2)          # 0.25 > 0.1 -> 0.25 (floor)
    assert st.C == 0.25
    oracle.audit(P, st, M, js, grp, 2)
    assert st.C == 0.25
    oracle.audit(P, st, M, np.zeros(n), grp, 2)  # calm interval: grow by 1.25
    assert st.C == 0.3125
    P.audit = 0
    oracle.audit(P, st, M, js, grp, 2)
    assert st.C == 1.0

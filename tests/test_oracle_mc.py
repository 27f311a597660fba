"""Pins of the oracle's whole Monte Carlo interval (Sect. 2.5.3, Appendix A).

* Constant kernel (Appendix A): with lambda_ij = (1/t0)(1/N_K)(m0/m_j), the
  expected gain of every particle is sum_j lambda_ij m_j = m0/t0 whatever the
  lists, grouping or frozen intervals, so the mass-weighted mean grain mass is
  m0 (1 + t/t0) exactly in expectation; and the mass-weighted distribution
  approaches the Smoluchowski solution n ~ (t/2)^(m-1) / (1 + t/2)^(m+1)
  (measured by the W1 distance of Appendix B).
* The represented mass M_i is never changed and N_i m_i = M_i.
"""
import math

import numpy as np

from paper_2609_35967_gb300 import workloads as W


def _run(oracle, ins, t_end):
    P = oracle.params(ins["params"])
    st = oracle.new_state(P)
    s = ins["s"].copy()
    t = 0.0
    while t < t_end - 1e-12:
        oracle.interval_step(P, st, ins["x"], ins["y"], ins["z"], s, ins["M"], want=())
        t += st.dt_exe
        assert st.status == 0
    return P, st, s, t


def _w1_constant(m, M, t):
    mt = np.rint(m).astype(np.int64)
    k = np.arange(1, max(int(mt.max()), 200) + 1)
    x = t / 2.0
    nk = x ** (k - 1) / (1 + x) ** (k + 1)
    fe = np.cumsum(k * nk) / np.sum(k * nk)
    order = np.argsort(mt)
    cm = np.cumsum(M[order]) / M.sum()
    fs = np.zeros(len(k))
    idx = np.searchsorted(mt[order], k, side="right")
    fs[idx > 0] = cm[idx[idx > 0] - 1]
    return float(np.sum(np.abs(fs - fe)[:-1] * np.diff(np.log10(k))))


def test_constant_kernel_mean_mass_and_w1(oracle):
    devs, ses = [], []
    for seed in (11, 12, 13, 14):
        ins = W.coag_instance(1024, K=16, mode=W.CONSTANT, seed=seed)
        P, st, s, t = _run(oracle, ins, 4.0)
        m = math.pi * P.rho_s * s ** 3 / 6.0
        # masses stay integer multiples of m0 (coagulation of unit grains)
        assert np.abs(m - np.rint(m)).max() < 1e-9
        devs.append(m.mean() - (1.0 + t))
        ses.append(m.std() / math.sqrt(len(m)))
        assert _w1_constant(m, ins["M"], t) < 0.04
    se = math.sqrt(sum(x * x for x in ses)) / len(ses)
    assert abs(np.mean(devs)) < 5 * se


def test_mass_is_conserved(oracle):
    ins = W.patch_instance(600, K=16, seed=7, v_frag=100.0)
    M0 = ins["M"].copy()
    P = oracle.params(dict(ins["params"], v_frag=5.0))   # fragmentation and erosion too
    st = oracle.new_state(P)
    s = ins["s"].copy()
    ev = 0
    for _ in range(12):
        oracle.interval_step(P, st, ins["x"], ins["y"], ins["z"], s, ins["M"], want=())
        ev += st.events
    assert ev > 0 and st.status == 0
    assert np.array_equal(ins["M"], M0)
    m = math.pi * P.rho_s * s ** 3 / 6.0
    N = ins["M"] / m
    assert abs((N * m).sum() - M0.sum()) <= 1e-12 * M0.sum()
    assert (s >= P.s_min * (1 - 1e-12)).all()


def test_config0_short_run(oracle):
    ins = W.config0(n=1024)[0]
    P = oracle.params(ins["params"])
    st = oracle.new_state(P)
    s = ins["s"].copy()
    res = oracle.interval_step(P, st, ins["x"], ins["y"], ins["z"], s, ins["M"])
    assert st.status == 0
    assert 0 < st.dt_exe <= P.dt_coll
    # the executed interval is dt_coll / 2^k
    k = math.log2(P.dt_coll / st.dt_exe)
    assert k == int(k)
    assert (res["nbr"][:, 0] == np.arange(1024)).all()
    assert (np.diff(res["nbr"][:, 1:], axis=1) > 0).all()
    assert res["ev_count"].sum() == st.events

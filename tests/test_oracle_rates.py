"""Pins of the oracle's rate model (Sect. 2.2, 2.3.1, 2.5.1-2.5.3).

Each test checks the oracle against something other than its own formula:
closed forms of special cases, known physical limits, numerical quadrature,
exact invariants and sampling statistics.
"""
import math

import numpy as np
import pytest
import mpmath as mp
from scipy import integrate

from paper_2609_35967_gb300 import workloads as W

KB, MH, MU, G = 1.380649e-16, 1.6735575e-24, 2.34, 6.674e-8


def _patch(oracle, **kw):
    ins = W.patch_instance(64, **kw)
    return oracle.params(ins["params"]), ins


def test_gas_reference_values(oracle):
    """c_s, Omega_K, H_g at 10 au / 50 K; power laws of Sigma_g, T and h_g (Sect. 2.2)."""
    P, _ = _patch(oracle)
    g = oracle.gas(P, 0.0, 0.0, 0.0)
    assert g["cs"] == pytest.approx(4.19854e4, rel=1e-5)
    assert g["Om"] == pytest.approx(6.296836e-9, rel=1e-6)
    assert g["H"] / W.AU == pytest.approx(0.445708, rel=1e-5)
    # h_g ~ R^((q+1)/2) and Sigma ~ R^p along the disk midplane
    D = oracle.params(W.disk_instance(8)["params"])
    g1 = oracle.gas(D, 10 * W.AU, 0.0, 0.0)
    g2 = oracle.gas(D, 40 * W.AU, 0.0, 0.0)
    assert g2["h"] / g1["h"] == pytest.approx(4.0 ** ((D.q + 1) / 2), rel=1e-12)
    assert g2["Sigma"] / g1["Sigma"] == pytest.approx(4.0 ** D.p, rel=1e-12)
    assert g1["Sigma"] == pytest.approx(170.0, rel=1e-12)
    # hydrostatic vertical profile: rho_g(Z)/rho_g(0) = exp(-(1 - R/r)/h^2)
    gz = oracle.gas(D, 10 * W.AU, 0.0, 2 * g1["H"])
    R, r = gz["R"], math.hypot(gz["R"], gz["Z"])
    assert gz["rho_g"] / g1["rho_g"] == pytest.approx(math.exp(-(1 - R / r) / g1["h"] ** 2),
                                                      rel=1e-12)
    # eta at the midplane: -(p + q/2 - 3/2) h^2 / 2
    assert g1["eta"] == pytest.approx(1.375 * g1["h"] ** 2, rel=1e-12)


def test_stokes_scalings(oracle):
    """St is linear in s, ~ R^-p in the midplane, and grows as 1/rho_g with height (Sect. 2.3.1)."""
    D = oracle.params(W.disk_instance(8)["params"])
    g1 = oracle.gas(D, 10 * W.AU, 0.0, 0.0)
    g2 = oracle.gas(D, 20 * W.AU, 0.0, 0.0)
    assert g2["gst"] / g1["gst"] == pytest.approx(2.0 ** (-D.p), rel=1e-12)
    gz = oracle.gas(D, 10 * W.AU, 0.0, 1.5 * g1["H"])
    assert gz["gst"] / g1["gst"] == pytest.approx(g1["rho_g"] / gz["rho_g"], rel=1e-12)
    # Epstein: St = rho_o a / (rho_g v_th) * Omega with a = s/2, v_th = sqrt(8/pi) c_s
    s = 2e-4
    st = D.rho_s * (s / 2) / (g1["rho_g"] * math.sqrt(8 / math.pi) * g1["cs"]) * g1["Om"]
    assert g1["gst"] * s == pytest.approx(st, rel=1e-12)


def test_monodisperse_closed_form(oracle):
    """Equal grains in the tiny-eddy regime: every differential term and the turbulent
    term vanish, so lambda_ij = N_j pi s^2 min(c_s, sqrt(16 k_B T/(pi m))) / V_i."""
    P, ins = _patch(oracle, sigma=1000.0, a_um=0.1)      # St << Re^-1/2
    g = oracle.gas_struct(P, 0.01 * P.box_x, 0.02 * P.box_x, 0.05 * P.box_x)
    s = ins["s"][0]
    m = oracle.grain_mass(P, s)
    assert m == pytest.approx(math.pi * P.rho_s * s ** 3 / 6, rel=1e-15)
    assert g.gst * s < g.Re ** -0.5
    N = ins["M"][0] / m
    V = 1.234e36
    pr = oracle.pair(P, g, s, m, s, m, N, V)
    assert pr["dvR"] == 0.0 and pr["dvZ"] == 0.0 and pr["dvphi"] == 0.0 and pr["dvt"] == 0.0
    cs = math.sqrt(KB * g.T / (MU * MH))
    dvb = min(cs, math.sqrt(16 * KB * g.T / (math.pi * m)))
    assert pr["dv"] == pytest.approx(dvb, rel=1e-14)
    assert pr["lam"] == pytest.approx(N * math.pi * s * s * dvb / V, rel=1e-14)
    assert pr["outcome"] == 0 and pr["ncoll"] == 1.0
    assert pr["c"][0] == pr["lam"] and pr["c"][1] == 0.0
    assert pr["J1"][0] == pytest.approx(math.log(2.0) / 3.0, rel=1e-15)


def test_drift_limits_and_symmetry(oracle):
    """St_i = 1 against St_j -> 0: |dv_R| = eta v_K and |dv_phi| = eta v_K / 2 (the
    classic drift maxima); swapping i and j flips every signed term."""
    D = oracle.params(W.disk_instance(8)["params"])
    g = oracle.gas_struct(D, 30 * W.AU, 0.0, 0.0)
    s1 = 1.0 / g.gst
    s2 = 1e-9 / g.gst
    m1, m2 = oracle.grain_mass(D, s1), oracle.grain_mass(D, s2)
    a = oracle.pair(D, g, s1, m1, s2, m2, 1.0, 1.0)
    vk = g.R * g.Om
    assert abs(a["dvR"]) == pytest.approx(g.eta * vk, rel=1e-8)
    assert abs(a["dvphi"]) == pytest.approx(0.5 * g.eta * vk, rel=1e-8)
    b = oracle.pair(D, g, s2, m2, s1, m1, 1.0, 1.0)
    for k in ("dvR", "dvZ", "dvphi"):
        assert b[k] == -a[k]
    for k in ("dvB", "dvt", "dv"):
        assert b[k] == a[k]


def test_turbulence_limits(oracle):
    """Ormel & Cuzzi (2007) limits: symmetric; zero for equal grains below the Kolmogorov
    time; ~3 alpha St c_s^2 for equal grains in the intermediate regime; heavy regime
    V_g^2 (1/(1+St1) + 1/(1+St2)) which decays for St >> 1."""
    vg2, re = 1.0, 1e8
    assert oracle.turb_dv2(1e-5, 1e-5, vg2, re) == 0.0
    assert oracle.turb_dv2(3e-5, 1e-6, vg2, re) == oracle.turb_dv2(1e-6, 3e-5, vg2, re)
    alpha, cs, st = 1e-3, 1.0, 0.01
    dv2 = oracle.turb_dv2(st, st, 1.5 * alpha * cs * cs, re)
    assert dv2 / (alpha * st * cs * cs) == pytest.approx(3.0, rel=0.02)
    assert oracle.turb_dv2(10.0, 10.0, vg2, re) == pytest.approx(2.0 / 11.0, rel=1e-15)
    assert oracle.turb_dv2(1e4, 1e4, vg2, re) < 3e-4
    # tiny regime grows with the size contrast
    assert oracle.turb_dv2(5e-5, 1e-6, vg2, re) > oracle.turb_dv2(5e-5, 4e-5, vg2, re)


@pytest.mark.parametrize("ratio", [1.0000004, 1.0003, 1.002, 1.5, 10.0, 1e3, 1e8])
def test_fragment_moments_by_quadrature(oracle, ratio):
    """<J> and <J^2> of Eq. frag against direct quadrature over U (Sect. 2.5.3)."""
    s_min = 2e-5
    s_i = ratio * s_min

    mp.mp.dps = 40
    a = mp.sqrt(mp.mpf(s_min) / mp.mpf(s_i))

    def J(u):
        return -2 * mp.log(a + u * (1 - a))

    q1 = float(mp.quad(J, [0, 1]))
    q2 = float(mp.quad(lambda u: J(u) ** 2, [0, 1]))
    j1, j2 = oracle.frag_moments(s_i, s_min)
    assert j1 == pytest.approx(q1, rel=1e-9)
    assert j2 == pytest.approx(q2, rel=1e-9)
    assert oracle.frag_moments(s_min, s_min) == (0.0, 0.0)


def test_outcomes_and_grouping_invariance(oracle):
    """Sticking / erosion / fragmentation choice, the grouping factor, and the invariant
    that grouping leaves the expected mass-change rate unchanged (Sect. 2.5.2)."""
    P, _ = _patch(oracle, v_frag=100.0)
    g = oracle.gas_struct(P, 0.0, 0.0, 0.0)
    s_i = 1e-1
    m_i = oracle.grain_mass(P, s_i)
    for psi in (3e-9, 5e-7, 2e-6, 0.05, 0.1, 0.5, 2.0):
        s_j = s_i * psi ** (1 / 3)
        m_j = psi * m_i
        pr = oracle.pair(P, g, s_i, m_i, s_j, m_j, 1e10, 1e30)
        nc = math.floor(1e-4 / pr["psi"]) if pr["psi"] <= 1e-6 else 1.0
        assert pr["ncoll"] == nc
        lam = pr["lam"]
        if pr["dv"] < P.v_frag:
            assert pr["outcome"] == 0
            gain = pr["c"][0] * (nc * m_j)
            assert gain == pytest.approx(lam * m_j, rel=1e-13)
        elif pr["psi"] <= 0.1:
            assert pr["outcome"] == 1
            gain = pr["c"][0] * (-nc * m_j) + pr["c"][1] * (m_j - m_i)
            assert gain == pytest.approx(-2.0 * (1.0 - pr["psi"]) * lam * m_j, rel=1e-10)
            assert pr["c"][0] + pr["c"][1] * nc == pytest.approx(
                ((1 - pr["psi"]) + pr["psi"] * nc) * lam / nc * nc, rel=1e-13)
        else:
            assert pr["outcome"] == 2 and pr["c"][0] == lam
    # force the fast branch with a tiny v_frag: psi <= 0.1 erodes, larger psi fragments
    Pf, _ = _patch(oracle, v_frag=1e-6)
    pe = oracle.pair(Pf, g, s_i, m_i, s_i * 0.1 ** (1 / 3), 0.1 * m_i, 1.0, 1.0)
    pf = oracle.pair(Pf, g, s_i, m_i, s_i * 0.2 ** (1 / 3), 0.2 * m_i, 1.0, 1.0)
    assert pe["outcome"] == 1 and pf["outcome"] == 2
    assert pe["J1"][1] == pytest.approx(math.log(10.0) / 3.0, rel=1e-14)
    assert pe["J1"][0] == pytest.approx(-math.log(0.9) / 3.0, rel=1e-14)


def test_volume_caps_by_integration(oracle):
    """Locally flat boundary: the sphere's part inside the domain (Sect. 2.5.1)."""
    D = oracle.params(W.disk_instance(8)["params"])
    d = 0.3 * W.AU
    full = 4.0 * math.pi * d ** 3 / 3.0
    assert oracle.volume(D, d, 50 * W.AU) == pytest.approx(full, rel=1e-15)
    for h_frac in (0.0, 0.2, 0.5, 0.999):
        h = h_frac * d
        inside = integrate.quad(lambda t: math.pi * (d * d - t * t), -h, d, epsrel=1e-13)[0]
        assert oracle.volume(D, d, D.R_in + h) == pytest.approx(inside, rel=1e-10) or h == 0.0
        assert oracle.volume(D, d, D.R_out - h) == pytest.approx(inside, rel=1e-10) or h == 0.0
    P, _ = _patch(oracle)
    assert oracle.volume(P, d, P.r0) == pytest.approx(full, rel=1e-15)


def test_partner_choice_frequencies(oracle):
    """Two particles, K = 2: the first event picks channel c with probability
    lambda*_c / lambda*_i (Sect. 2.5.3), checked over independent seeds."""
    ins = W.disk_instance(2, seed=4)
    ins["x"][:] = [30 * W.AU, 30 * W.AU + 1e10]
    ins["y"][:] = 0.0
    ins["z"][:] = 0.0
    ins["s"][:] = [2e-3, 5e-4]
    base = dict(ins["params"], K=2, max_events=1)
    P = oracle.params(base)
    nbr, d = oracle.knn(P, ins["x"], ins["y"], ins["z"], [0])
    r = oracle.rates_subset(P, ins["x"], ins["y"], ins["z"], ins["s"], ins["M"], [0], nbr, d,
                            chan=True)
    ch = r["chan"][0].ravel()
    p = ch / ch.sum()
    trials = 4000
    hits = np.zeros(4)
    for t in range(trials):
        P.seed = 1000 + t
        o = oracle.sample_subset(P, ins["x"], ins["y"], ins["z"], ins["s"], ins["M"], [0],
                                 nbr, d, 1e300, 0)
        assert o["ev_count"][0] == 1
        hits[int(o["ev_hash"][0]) - 1] += 1
    for c in range(4):
        sd = math.sqrt(trials * p[c] * (1 - p[c])) + 1e-9
        assert abs(hits[c] - trials * p[c]) <= 5 * sd

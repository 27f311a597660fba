"""Pins of the oracle's dust diffusion step (Sect. 2.4; the ring test of Sect. 3.2).

* Ring test: ln(R/R0) starts N(0, 0.05^2); with D = D0 (R/R0)^2 the analytic solution
  keeps it Gaussian with mean (2 + chi p) D0 t / R0^2 and variance 0.05^2 + 2 D0 t / R0^2
  (0.2025 at t~ = 0.1, the value the paper quotes), for both prescriptions.
* The drift terms of the physical model against central finite differences of D and
  ln rho_g computed from the gas disk itself (the derivative algebra is a reading).
* Vertical equilibrium: concentration diffusion (chi = 1) keeps dust that follows the gas
  density (rho_d ~ rho_g is its stationary state); density diffusion (chi = 0) spreads it
  by 2 D t.
* The normal draws: mean 0, variance 1, independent components.
"""
import math

import numpy as np

from paper_2609_35967_gb300 import workloads as W


def _ring(oracle, chi, n=1 << 16, steps=100):
    rng = np.random.default_rng(5)
    lnR = rng.normal(0.0, 0.05, n)
    ph = rng.uniform(0.0, 2 * math.pi, n)
    x, y, z = np.exp(lnR) * np.cos(ph), np.exp(lnR) * np.sin(ph), np.zeros(n)
    P = oracle.params(dict(W.ring_params(chi=chi)))
    t0 = P.r0 ** 2 / P.D0
    dt = 0.1 * t0 / steps
    s = np.full(n, 1e-4)
    for k in range(steps):
        oracle.diffuse(P, dt, k, x, y, z, s)
    return np.log(np.sqrt(x * x + y * y) / P.r0), P


def test_ring_diffusion_mean_and_variance(oracle):
    for chi in (0, 1):
        l, P = _ring(oracle, chi)
        n = len(l)
        mu, var = (2.0 + chi * P.p) * 0.1, 0.05 ** 2 + 0.2
        se_mu = math.sqrt(var / n)
        se_var = var * math.sqrt(2.0 / n)
        # statistics plus the Euler-Maruyama bias of 100 steps (below 1e-3 here)
        assert abs(l.mean() - mu) < 4 * se_mu + 1e-3, (chi, l.mean(), mu)
        assert abs(l.var() - var) < 4 * se_var + 1e-3, (chi, l.var(), var)
    assert abs(var - 0.2025) < 1e-15


def test_drift_terms_match_finite_differences(oracle):
    ins = W.disk_instance(16, seed=1)
    base = dict(ins["params"], diff_chi=0, Sc_R=1.0, Sc_Z=1.0, Sc_phi=1.0)
    P = oracle.params(base)
    AU = W.AU

    def D_and_lnrho(R, Z, s):
        g = oracle.gas(P, R, 0.0, Z)
        St = g["gst"] * s
        return P.alpha * g["cs"] * g["H"] / (1.0 + St * St), math.log(g["rho_g"])

    for R_au, Z_frac, s in ((10.0, 0.0, 1e-2), (10.0, 1.3, 3e-1), (30.0, 0.7, 1e-4), (60.0, 2.0, 2.0)):
        R = R_au * AU
        H = oracle.gas(P, R, 0.0, 0.0)["H"]
        Z = Z_frac * H
        c = oracle.diff_coeffs(P, R, Z, s)
        hR, hZ = 1e-5 * R, 1e-4 * H
        DpR, lpR = D_and_lnrho(R + hR, Z, s)
        DmR, lmR = D_and_lnrho(R - hR, Z, s)
        DpZ, lpZ = D_and_lnrho(R, Z + hZ, s)
        DmZ, lmZ = D_and_lnrho(R, Z - hZ, s)
        D0, _ = D_and_lnrho(R, Z, s)
        assert c[0] == c[1] == c[2]
        assert abs(c[0] / D0 - 1.0) < 1e-14
        # chi = 0: drift_R = D/R + dD/dR, drift_Z = dD/dZ
        dDdR = (DpR - DmR) / (2 * hR)
        dDdZ = (DpZ - DmZ) / (2 * hZ)
        assert abs((c[3] - c[0] / R) - dDdR) < 1e-6 * (abs(dDdR) + D0 / R)
        assert abs(c[4] - dDdZ) < 1e-6 * (abs(dDdZ) + D0 / H)
        assert abs(c[5] - (lpR - lmR) / (2 * hR)) < 1e-6 / R
        assert abs(c[6] - (lpZ - lmZ) / (2 * hZ)) < 1e-5 / H
    # chi = 1 adds D dln rho_g
    P1 = oracle.params(dict(base, diff_chi=1))
    c0 = oracle.diff_coeffs(P, 20 * AU, 0.3 * AU, 1e-2)
    c1 = oracle.diff_coeffs(P1, 20 * AU, 0.3 * AU, 1e-2)
    assert abs(c1[3] - (c0[3] + c0[0] * c0[5])) < 1e-12 * abs(c1[3]) + 1e-30
    assert abs(c1[4] - (c0[4] + c0[1] * c0[6])) < 1e-12 * abs(c1[4]) + 1e-30


def _vertical(oracle, chi, n=1 << 15):
    R0 = 10.0 * W.AU
    ins = W.disk_instance(16, seed=1)
    P = oracle.params(dict(ins["params"], diff_chi=chi))
    g = oracle.gas(P, R0, 0.0, 0.0)
    H, Om = g["H"], g["Om"]
    rng = np.random.default_rng(7)
    ph = rng.uniform(0.0, 2 * math.pi, n)
    x, y = R0 * np.cos(ph), R0 * np.sin(ph)
    z = rng.normal(0.0, H, n)
    s = np.full(n, 2e-4)                       # St ~ 1e-4: D = nu = alpha c_s H
    t_end = 0.5 / (P.alpha * Om)               # D t = 0.5 H^2
    steps = 50
    for k in range(steps):
        oracle.diffuse(P, t_end / steps, k, x, y, z, s)
    R = np.sqrt(x * x + y * y)
    Hs = np.array([oracle.gas(P, r, 0.0, 0.0)["H"] for r in R])
    return z / Hs


def test_vertical_equilibrium(oracle):
    keep = _vertical(oracle, 1)
    spread = _vertical(oracle, 0)
    n = len(keep)
    se = math.sqrt(2.0 / n)
    # chi = 1: stationary (the Gaussian start differs from rho_g by O(h^2) = 0.3%)
    assert abs(keep.var() - 1.0) < 4 * se + 0.01, keep.var()
    # chi = 0: variance 1 + 2 D t / H^2 = 2
    assert abs(spread.var() - 2.0) < 4 * 2 * se + 0.03, spread.var()


def test_normal_draws(oracle):
    n = 1 << 15
    # with R = R0 huge the drift vanishes and dR = sqrt(2 D dt) zeta_R exactly
    x = np.full(n, 1e9)
    y = np.zeros(n)
    z = np.zeros(n)
    oracle.diffuse(oracle.params(dict(W.ring_params(chi=0), D0=1.0, r0=1e9)), 0.5, 3, x, y, z, np.ones(n))
    zeta = np.sqrt(x * x + y * y) - 1e9
    assert abs(zeta.mean()) < 4 / math.sqrt(n)
    assert abs(zeta.var() - 1.0) < 4 * math.sqrt(2.0 / n)
    assert abs(np.corrcoef(zeta[:-1], zeta[1:])[0, 1]) < 4 / math.sqrt(n)

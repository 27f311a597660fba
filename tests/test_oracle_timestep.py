"""Pins of the oracle's common transport timestep (Sect. 2.6): Delta t = min(Delta t_max,
Delta t_out, min_i Delta t_i), the local limit being the most restrictive of the orbital,
deterministic-displacement and diffusive-displacement limits (the reading stated in the
oracle).  Each limit is pinned through what it means, with other pinned parts of the
oracle or closed forms:

* orbital (f_orb = 1): a drag-free circular orbit pushed for Delta t_i comes back to its
  starting azimuth;
* deterministic: |u| Delta t_i = c_adv dx_H H_g, invariant under moving the speed between
  the radial, polar and azimuthal components (catches a wrong r or R), zero for a
  particle on the local circular Keplerian motion;
* diffusive: one Euler-Maruyama step of length Delta t_i spreads the radius by
  c_diff dx (ring test); with St -> 0 in the physical model Delta t_i Omega_K =
  c_diff^2 dx_H^2 / (2 alpha) (D = alpha c_s H_g, H_g = c_s / Omega_K);
* the minimum over particles and the global bounds.
"""
import math

import numpy as np

from paper_2609_35967_gb300 import workloads as W


def _disk(oracle, **kw):
    ins = W.disk_instance(8, seed=1)
    return oracle.params(dict(ins["params"], **kw))


def test_orbital_limit_is_one_orbit(oracle):
    P = oracle.params(dict(geometry=W.DISK, M_star=1.0 / 6.674e-8, r0=1.0, sigma0=1.0, T0=1.0, rho_s=1.0))
    R = 1.3
    rule = oracle.dt_rule(1e30, f_orb=1.0)
    T = oracle.local_dt(P, rule, R, 0.0, 0.0, 1.0)
    x, y, z = np.array([R]), np.array([0.0]), np.array([0.0])
    vr, lth, lph = np.array([0.0]), np.array([0.0]), np.array([math.sqrt(R)])   # circular: l = sqrt(GM R)
    n = 2000
    for _ in range(n):
        oracle.push(P, x, y, z, vr, lth, lph, np.array([1.0]), T / n, drag=False)
    phi = math.atan2(y[0], x[0])
    assert abs(phi) < 1e-5, phi
    assert abs(math.hypot(x[0], y[0]) / R - 1.0) < 1e-9
    # half the fraction, half the time
    assert abs(oracle.local_dt(P, oracle.dt_rule(1e30, f_orb=0.5), R, 0.0, 0.0, 1.0) / T - 0.5) < 1e-15


def test_deterministic_limit(oracle):
    P = _disk(oracle)
    R, Z = 20.0 * W.AU, 0.05 * 20.0 * W.AU
    r = math.hypot(R, Z)
    g = oracle.gas(P, R, 0.0, Z)
    Om = g["Om"]
    rule = oracle.dt_rule(1e30, dx_H=0.1, c_adv=0.5)
    kep = Om * R * R
    # on the local circular Keplerian motion: no deterministic limit
    assert oracle.local_dt(P, rule, R, 0.0, Z, 1e-4, (0.0, 0.0, kep)) == math.inf
    w = 3.0e3
    dts = [oracle.local_dt(P, rule, R, 0.0, Z, 1e-4, v)
           for v in ((w, 0.0, kep), (0.0, w * r, kep), (0.0, 0.0, kep + w * R),
                     (w / math.sqrt(2), w / math.sqrt(2) * r, kep))]
    for d in dts:
        assert abs(d / dts[0] - 1.0) < 1e-12, dts
    assert abs(w * dts[0] / (0.5 * 0.1 * g["H"]) - 1.0) < 1e-12
    # doubling the speed halves the limit
    assert abs(oracle.local_dt(P, rule, R, 0.0, Z, 1e-4, (2 * w, 0.0, kep)) / dts[0] - 0.5) < 1e-12
    # patches do not move: no deterministic limit there
    Pp = oracle.params(W.patch_instance(8, seed=2)["params"])
    assert oracle.local_dt(Pp, rule, 0.0, 0.0, 0.0, 1e-4, (w, 0.0, 0.0)) == math.inf


def test_diffusive_limit_spreads_by_one_spacing(oracle):
    P = oracle.params(dict(W.ring_params(chi=0), D0=1e-4))
    R0 = 1.0
    rule = oracle.dt_rule(1e30, dx_H=0.2, c_diff=0.3)
    dt = oracle.local_dt(P, rule, R0, 0.0, 0.0, 1e-4)
    H = oracle.gas(P, R0, 0.0, 0.0)["H"]
    n = 1 << 15
    x, y, z = np.full(n, R0), np.zeros(n), np.zeros(n)
    oracle.diffuse(P, dt, 0, x, y, z, np.full(n, 1e-4))
    dR = np.hypot(x, y) - R0
    spread = 0.3 * 0.2 * H
    assert abs(dR.std() / spread - 1.0) < 4 * math.sqrt(0.5 / n) + 1e-3, dR.std() / spread


def test_diffusive_limit_small_grains_closed_form(oracle):
    alpha = 3e-3
    P = _disk(oracle, alpha=alpha, Sc_R=1.0, Sc_Z=1.0, Sc_phi=1.0)
    rule_d = oracle.dt_rule(1e30, dx_H=0.1, c_diff=0.5)
    rule_o = oracle.dt_rule(1e30, f_orb=1.0)
    for R_au in (5.0, 30.0, 90.0):
        R = R_au * W.AU
        t_orb = oracle.local_dt(P, rule_o, R, 0.0, 0.0, 1e-9)      # 2 pi / Omega_K
        t_diff = oracle.local_dt(P, rule_d, R, 0.0, 0.0, 1e-9)     # St ~ 1e-9
        assert abs(t_diff * 2 * math.pi / t_orb / (0.5 ** 2 * 0.1 ** 2 / (2 * alpha)) - 1.0) < 1e-12
    # the largest directional coefficient sets it: Sc_Z = 1/2 doubles D_Z
    P2 = _disk(oracle, alpha=alpha, Sc_R=1.0, Sc_Z=0.5, Sc_phi=1.0)
    R = 30.0 * W.AU
    assert abs(oracle.local_dt(P2, rule_d, R, 0.0, 0.0, 1e-9)
               / oracle.local_dt(P, rule_d, R, 0.0, 0.0, 1e-9) - 0.5) < 1e-12
    # large grains diffuse less: D / (1 + St^2), St = pi rho_o s / (4 Sigma_g) in the midplane
    s_big = 100.0
    St = math.pi * P.rho_s * s_big / (4.0 * oracle.gas(P, R, 0.0, 0.0)["Sigma"])
    ratio = oracle.local_dt(P, rule_d, R, 0.0, 0.0, s_big) / oracle.local_dt(P, rule_d, R, 0.0, 0.0, 1e-9)
    assert St > 1.0 and abs(ratio / (1.0 + St * St) - 1.0) < 1e-12, (ratio, St)


def test_global_minimum_and_bounds(oracle):
    ins = W.disk_instance(500, seed=3, sizes=("lognormal", 10.0, 1.0), velocities=True)
    P = oracle.params(ins["params"])
    rule = oracle.dt_rule(1e30, f_orb=0.05, dx_H=0.1, c_adv=0.5, c_diff=0.5)
    args = [ins[k] for k in ("x", "y", "z", "s", "vr", "lth", "lph")]
    dt, dti = oracle.timestep(P, rule, *args)
    assert dt == dti.min() and np.isfinite(dt) and dt > 0.0
    # the inner edge orbits fastest: the orbital limit there binds
    R = np.hypot(ins["x"], ins["y"])
    i = int(np.argmin(dti))
    assert R[i] < 1.2 * R.min()
    for cap in (0.5 * dt, 2.0 * dt):
        d2, _ = oracle.timestep(P, oracle.dt_rule(cap, f_orb=0.05, dx_H=0.1, c_adv=0.5, c_diff=0.5), *args)
        assert d2 == min(cap, dt)
        d3, _ = oracle.timestep(P, oracle.dt_rule(1e30, dt_out=cap, f_orb=0.05, dx_H=0.1, c_adv=0.5,
                                                  c_diff=0.5), *args)
        assert d3 == min(cap, dt)
    # no particles, or every limit off: the global bounds alone
    e = np.zeros(0)
    assert oracle.timestep(P, oracle.dt_rule(7.0, dt_out=9.0), e, e, e, e)[0] == 7.0
    assert oracle.timestep(P, oracle.dt_rule(7.0, dt_out=3.0), *args)[0] == 3.0

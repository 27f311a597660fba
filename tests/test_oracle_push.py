"""Pins of the oracle's staggered semi-analytic step (Sect. 2.3.3, Sect. 3.1).

Drag-free eccentric Kepler orbit (e = 0.5, GM = R0 = 1, P0 = 2 pi) started at
pericentre (R, phi, v_r, l_phi) = (1/2, 0, 0, sqrt(3)/2), exact energy -1/2:
the maximum relative energy error over 100 P0 falls as dt^2 and is below 1e-4
at dt = P0/640 (the paper's Fig. 2 statement).  With drag, a grain with
t_s << dt relaxes to the terminal velocity y_g + t_s f.
"""
import math

import numpy as np
import pytest

from paper_2609_35967_gb300 import workloads as W


def _max_energy_error(oracle, steps_per_orbit, orbits=100):
    P = oracle.params(dict(geometry=W.DISK, M_star=1.0 / 6.674e-8, r0=1.0, sigma0=1.0,
                           T0=1.0, rho_s=1.0))
    x, y, z = np.array([0.5]), np.array([0.0]), np.array([0.0])
    vr, lth, lph = np.array([0.0]), np.array([0.0]), np.array([math.sqrt(3) / 2])
    s = np.array([1.0])
    dt = 2 * math.pi / steps_per_orbit
    GM = 6.674e-8 * P.M_star
    worst = 0.0
    for _ in range(orbits * steps_per_orbit):
        oracle.push(P, x, y, z, vr, lth, lph, s, dt, drag=False)
        r = math.sqrt(x[0] ** 2 + y[0] ** 2 + z[0] ** 2)
        st2 = (x[0] ** 2 + y[0] ** 2) / (r * r)
        E = 0.5 * (vr[0] ** 2 + (lth[0] / r) ** 2 + lph[0] ** 2 / (r * r * st2)) - GM / r
        worst = max(worst, abs(E + 0.5) / 0.5)
    return worst


def test_kepler_second_order(oracle):
    e80 = _max_energy_error(oracle, 80, orbits=20)
    e160 = _max_energy_error(oracle, 160, orbits=20)
    assert 3.0 < e80 / e160 < 5.0
    assert _max_energy_error(oracle, 640, orbits=100) < 1e-4


def test_terminal_drift_limit(oracle):
    ins = W.disk_instance(4, seed=3, velocities=True)
    P = oracle.params(ins["params"])
    x, y, z = ins["x"].copy(), ins["y"].copy(), ins["z"].copy()
    vr, lth, lph = np.zeros(4), np.zeros(4), ins["lph"].copy()
    s = np.full(4, 2e-4)                     # St ~ 1e-6: t_s << dt
    dt = 1e6
    oracle.push(P, x, y, z, vr, lth, lph, s, dt, drag=True)
    # terminal state: y -> y_g + t_s f (the linear ODE's fixed point)
    for i in range(4):
        r = math.sqrt(x[i] ** 2 + y[i] ** 2 + z[i] ** 2)
        assert abs(vr[i]) < 1e-3 * math.sqrt(6.674e-8 * P.M_star / r)

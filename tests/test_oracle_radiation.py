"""Pins of the oracle's radiation forces and optical depth (Sect. 2.3.2).

- The taper's closed values and smoothness; beta(s), kappa(s) ~ 1/s.
- tau of one particle: its kappa M dr over the cell volume, the volume integrated
  numerically in (r, theta, phi) (3D form) or as an area times sqrt(2 pi) H_g (2D form).
- tau of a uniform shell or annulus: the analytic integral of a constant density
  (statistical agreement).
- Interpolation: exact for fields linear in the face and column indices, continuous
  across phi = +-pi.
- Forces, through the staggered step: a circular orbit with GM (1 - beta) stays
  circular; Poynting-Robertson decay of a and e at the rates of Wyatt & Whipple (1950)
  (de/dt = -5/2 alpha e / (a^2 sqrt(1 - e^2)), da/dt = -alpha (2 + 3 e^2)/(a (1 - e^2)^1.5),
  alpha = beta GM / c), which also fixes the factor 2 on v_r; a grain behind a wall of
  tau = ln 2 moves exactly as one with beta / 2 and no wall; a taper of one half at the
  kick's time equals beta / 2; a grain with beta = 2 eta on a gas-speed circular orbit
  stays put (the gas then orbits at the grain's own circular speed).
"""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2609_35967_gb300 import workloads as W

G = 6.674e-8
C_LIGHT = 2.99792458e10
AU = W.AU


def _disk(**kw):
    d = dict(geometry=W.DISK, M_star=W.MSUN, r0=AU, sigma0=1700.0, p=-1.0, T0=280.0, q=-0.5,
             rho_s=1.67, alpha=1e-3)
    d.update(kw)
    return d


def test_taper_closed_values(oracle):
    P = oracle.params(_disk(t_beta=8.0))
    assert oracle.rad_taper(P, -1.0) == 0.0
    assert oracle.rad_taper(P, 0.0) == 0.0
    assert oracle.rad_taper(P, 2.0) == 5.0 / 32.0
    assert oracle.rad_taper(P, 4.0) == 0.5
    assert oracle.rad_taper(P, 8.0) == 1.0
    assert oracle.rad_taper(P, 80.0) == 1.0
    # smooth: zero slope at both ends, monotone between
    h = 1e-4
    assert oracle.rad_taper(P, h) / h < 1e-3
    assert (1.0 - oracle.rad_taper(P, 8.0 - h)) / h < 1e-3
    v = [oracle.rad_taper(P, t) for t in np.linspace(0, 8, 101)]
    assert all(b >= a for a, b in zip(v, v[1:]))
    assert oracle.rad_taper(oracle.params(_disk(t_beta=0.0)), 0.0) == 1.0


def test_beta_kappa_scale_inverse_with_size(oracle):
    P = oracle.params(_disk(beta0=0.3, kappa0=5.0, rad_s0=1e-3))
    assert oracle.rad_beta(P, 1e-3) == 0.3
    assert oracle.rad_beta(P, 2e-3) == 0.15
    assert oracle.rad_kappa(P, 1e-3) == 5.0
    assert oracle.rad_kappa(P, 4e-3) == 1.25


def _grid3d(**kw):
    d = _disk(kappa0=2.0, rad_s0=1e-3, tau_geom=0, tau_nr=8, tau_nmu=4, tau_nphi=6,
              tau_rmin=10 * AU, tau_rmax=18 * AU, tau_mu=0.2)
    d.update(kw)
    return d


def _sph(r, mu, phi):
    st = math.sqrt(1.0 - mu * mu)
    return r * st * math.cos(phi), r * st * math.sin(phi), r * mu


def _cell_volume_3d(r_lo, r_hi, mu_lo, mu_hi, ph_lo, ph_hi):
    # integral of r^2 sin(theta) over the cell, theta from the mu edges
    th_lo, th_hi = math.acos(mu_hi), math.acos(mu_lo)
    v, _ = integrate.tplquad(lambda ph, th, r: r * r * math.sin(th), r_lo, r_hi, th_lo, th_hi,
                             ph_lo, ph_hi, epsrel=1e-13, epsabs=0)
    return v


def test_single_particle_tau_3d(oracle):
    P = oracle.params(_grid3d())
    i, j, k = 3, 2, 4
    dr, dmu, dph = AU, 0.1, 2 * math.pi / 6
    r = 10 * AU + (i + 0.37) * dr
    mu = -0.2 + (j + 0.61) * dmu
    ph = -math.pi + (k + 0.45) * dph
    x, y, z = _sph(r, mu, ph)
    M = 3.0e20
    T = oracle.tau_grid(P, [x], [y], [z], [1e-3], [M]).reshape(4 * 6, 9)
    V = _cell_volume_3d(10 * AU + i * dr, 10 * AU + (i + 1) * dr, -0.2 + j * dmu, -0.2 + (j + 1) * dmu,
                        -math.pi + k * dph, -math.pi + (k + 1) * dph)
    wall = 2.0 * M * dr / V
    col = j * 6 + k
    for c in range(24):
        if c != col:
            assert np.all(T[c] == 0.0)
    assert np.all(T[col, :i + 1] == 0.0)
    np.testing.assert_allclose(T[col, i + 1:], wall, rtol=1e-12)
    # at the column centre: the face value beyond, a linear share inside the cell
    xc, yc, zc = _sph(10 * AU + (i + 2.5) * dr, -0.2 + (j + 0.5) * dmu, -math.pi + (k + 0.5) * dph)
    assert oracle.tau_at(P, T.ravel(), xc, yc, zc) == pytest.approx(wall, rel=1e-12)
    xc, yc, zc = _sph(10 * AU + (i + 0.25) * dr, -0.2 + (j + 0.5) * dmu, -math.pi + (k + 0.5) * dph)
    assert oracle.tau_at(P, T.ravel(), xc, yc, zc) == pytest.approx(0.25 * wall, rel=1e-9)
    # inside the grid's inner edge: no extinction
    assert oracle.tau_at(P, T.ravel(), *_sph(9 * AU, 0.0, 0.3)) == 0.0
    # outside the grid nothing is deposited
    T2 = oracle.tau_grid(P, [x, 0.0, 0.0], [y, 0.0, 19 * AU], [z, 25 * AU, 0.0], [1e-3] * 3, [M] * 3)
    np.testing.assert_array_equal(T2, T.ravel())


def test_single_particle_tau_2d(oracle):
    P = oracle.params(_grid3d(tau_geom=1, tau_nmu=0))
    i, k = 5, 1
    dr, dph = AU, 2 * math.pi / 6
    R = 10 * AU + (i + 0.5) * dr
    ph = -math.pi + (k + 0.2) * dph
    M = 1.0e21
    T = oracle.tau_grid(P, [R * math.cos(ph)], [R * math.sin(ph)], [0.3 * AU], [2e-3], [M]).reshape(6, 9)
    area, _ = integrate.dblquad(lambda p, RR: RR, 10 * AU + i * dr, 10 * AU + (i + 1) * dr,
                                -math.pi + k * dph, -math.pi + (k + 1) * dph, epsrel=1e-13, epsabs=0)
    H = oracle.gas(P, 10 * AU + (i + 0.5) * dr, 0.0, 0.0)["H"]
    kappa = 2.0 * 1e-3 / 2e-3
    wall = kappa * M / (area * math.sqrt(2 * math.pi) * H) * dr
    np.testing.assert_allclose(T[k, i + 1:], wall, rtol=1e-12)
    assert np.all(T[k, :i + 1] == 0.0)
    assert np.count_nonzero(T) == 9 - (i + 1)


def test_uniform_shell_tau_3d(oracle):
    """A uniform shell a < r < b, |mu| < 0.2, all phi: tau(r) = kappa rho (r - a)."""
    rng = np.random.default_rng(7)
    n = 200_000
    a, b = 10 * AU, 18 * AU
    r = np.cbrt(rng.uniform(a ** 3, b ** 3, n))
    mu = rng.uniform(-0.2, 0.2, n)
    ph = rng.uniform(-math.pi, math.pi, n)
    st = np.sqrt(1 - mu * mu)
    x, y, z = r * st * np.cos(ph), r * st * np.sin(ph), r * mu
    Mtot = 1e24
    P = oracle.params(_grid3d())
    T = oracle.tau_grid(P, x, y, z, np.full(n, 1e-3), np.full(n, Mtot / n)).reshape(24, 9)
    rho = Mtot / ((b ** 3 - a ** 3) / 3 * 0.4 * 2 * math.pi)
    faces = a + np.arange(9) * AU
    expect = 2.0 * rho * (faces - a)
    # Poisson noise: four standard deviations of the particle count behind each face
    count = n * (faces ** 3 - a ** 3) / (b ** 3 - a ** 3)
    for f in range(1, 9):
        assert T.mean(axis=0)[f] == pytest.approx(expect[f], rel=4 / math.sqrt(count[f]))
    np.testing.assert_allclose(T[:, -1], expect[-1], rtol=4 / math.sqrt(n / 24))
    # tau at points: the shell's profile
    for rr in (11.3, 14.0, 17.5):
        t = oracle.tau_at(P, T.ravel(), *_sph(rr * AU, 0.05, 1.0))
        assert t == pytest.approx(2.0 * rho * (rr * AU - a), rel=0.06)


def test_uniform_annulus_tau_2d(oracle):
    """Uniform Sigma_d over a < R < b: tau(R) = int kappa Sigma_d / (sqrt(2 pi) H_g) dR."""
    rng = np.random.default_rng(8)
    n = 200_000
    a, b = 10 * AU, 18 * AU
    R = np.sqrt(rng.uniform(a * a, b * b, n))
    ph = rng.uniform(-math.pi, math.pi, n)
    z = rng.normal(size=n) * 0.5 * AU
    Mtot = 1e24
    P = oracle.params(_grid3d(tau_geom=1, tau_nmu=1, tau_nphi=4))
    T = oracle.tau_grid(P, R * np.cos(ph), R * np.sin(ph), z, np.full(n, 1e-3), np.full(n, Mtot / n))
    T = T.reshape(4, 9)
    sig = Mtot / (math.pi * (b * b - a * a))
    H = lambda RR: oracle.gas(P, RR, 0.0, 0.0)["H"]
    for f in range(1, 9):
        ex, _ = integrate.quad(lambda RR: 2.0 * sig / (math.sqrt(2 * math.pi) * H(RR)), a, a + f * AU)
        # Poisson noise (four standard deviations) and the midpoint rule's H_g (< 0.2%)
        count = n * ((a + f * AU) ** 2 - a * a) / (b * b - a * a)
        assert T.mean(axis=0)[f] == pytest.approx(ex, rel=4 / math.sqrt(count) + 0.002)


def test_interpolation_linear_fields(oracle):
    P = oracle.params(_grid3d())
    nr, nm, npf = 8, 4, 6
    j, k, f = np.meshgrid(np.arange(nm), np.arange(npf), np.arange(nr + 1), indexing="ij")
    T = (0.3 + 0.11 * f + 0.07 * j + 0.05 * k).astype(np.float64).ravel()
    dmu, dph = 0.1, 2 * math.pi / 6
    rng = np.random.default_rng(3)
    for _ in range(200):
        u = rng.uniform(0.0, 8.0)          # radial position in cells
        wj = rng.uniform(0.0, 3.0)         # between the first and last column centres
        wk = rng.uniform(0.0, 5.0)         # away from the phi wrap
        x, y, z = _sph(10 * AU + u * AU, -0.2 + (wj + 0.5) * dmu, -math.pi + (wk + 0.5) * dph)
        assert oracle.tau_at(P, T, x, y, z) == pytest.approx(0.3 + 0.11 * u + 0.07 * wj + 0.05 * wk,
                                                             rel=1e-12)
    # beyond the outer edge: the outer face; polar edges clamp to the edge columns
    x, y, z = _sph(30 * AU, -0.2 + 2.5 * dmu, -math.pi + 3.5 * dph)
    assert oracle.tau_at(P, T, x, y, z) == pytest.approx(0.3 + 0.88 + 0.14 + 0.15, rel=1e-12)
    x, y, z = _sph(12 * AU, 0.5, -math.pi + 3.5 * dph)
    assert oracle.tau_at(P, T, x, y, z) == pytest.approx(0.3 + 0.22 + 0.21 + 0.15, rel=1e-12)
    # periodic in phi: continuous across +-pi
    Tr = np.random.default_rng(4).uniform(0, 1, T.size)
    lo = oracle.tau_at(P, Tr, *_sph(13 * AU, 0.01, math.pi - 1e-9))
    hi = oracle.tau_at(P, Tr, *_sph(13 * AU, 0.01, -math.pi + 1e-9))
    assert abs(lo - hi) < 1e-8


def _circular(oracle, P, r, lph, steps, dt, drag=False, t=0.0):
    x, y, z = np.array([r]), np.array([0.0]), np.array([0.0])
    vr, lth, lp = np.zeros(1), np.zeros(1), np.array([lph])
    s, M = np.array([1e-3]), np.array([1.0])
    rs = []
    for n in range(steps):
        oracle.push_rad(P, x, y, z, vr, lth, lp, s, M, dt, t + n * dt, drag=drag)
        rs.append(math.hypot(x[0], y[0]))
    return np.array(rs), (x, y, z, vr, lth, lp)


def test_radiation_pressure_circular_orbit(oracle):
    beta = 0.3
    P = oracle.params(_disk(beta0=beta, rad_s0=1e-3))
    r0 = AU
    GM = G * W.MSUN
    Porb = 2 * math.pi * math.sqrt(r0 ** 3 / (GM * (1 - beta)))
    dt = Porb / 400
    rs, st = _circular(oracle, P, r0, math.sqrt(GM * (1 - beta) * r0), 800, dt)
    assert np.abs(rs / r0 - 1).max() < 1e-9
    # one period later the grain is back at phi = 0 (to O(dt^2))
    ph = math.atan2(st[1][0], st[0][0])
    assert abs(ph) < 1e-3
    # the Keplerian speed without beta is not circular under radiation pressure
    rs2, _ = _circular(oracle, P, r0, math.sqrt(GM * r0), 400, dt)
    assert (rs2 / r0 - 1).max() > 0.5


def _elements(GMp, x, y, vr, lph):
    r = math.hypot(x, y)
    v2 = vr * vr + (lph / r) ** 2
    a = -GMp / (2 * (0.5 * v2 - GMp / r))
    e = math.sqrt(max(0.0, 1 - lph * lph / (GMp * a)))
    return a, e


def test_poynting_robertson_decay(oracle):
    beta = 0.5
    P = oracle.params(_disk(beta0=beta, rad_s0=1e-3, rad_pr=1))
    GM = G * W.MSUN
    GMp = GM * (1 - beta)
    a0, e0 = 0.1 * AU, 0.2
    rp = a0 * (1 - e0)
    lph0 = math.sqrt(GMp * a0 * (1 - e0 * e0))
    Porb = 2 * math.pi * math.sqrt(a0 ** 3 / GMp)
    steps_per, orbits = 400, 20
    dt = Porb / steps_per
    x, y, z = np.array([rp]), np.array([0.0]), np.array([0.0])
    vr, lth, lp = np.zeros(1), np.zeros(1), np.array([lph0])
    s, M = np.array([1e-3]), np.array([1.0])
    for n in range(steps_per * orbits):
        oracle.push_rad(P, x, y, z, vr, lth, lp, s, M, dt, 0.0, drag=False)
    a1, e1 = _elements(GMp, x[0], y[0], vr[0], lp[0])
    # secular rates of Wyatt & Whipple, integrated over the same time
    alpha = beta * GM / C_LIGHT

    def rhs(t, u):
        a, e = u
        return [-alpha * (2 + 3 * e * e) / (a * (1 - e * e) ** 1.5),
                -2.5 * alpha * e / (a * a * math.sqrt(1 - e * e))]

    sol = integrate.solve_ivp(rhs, (0, orbits * Porb), [a0, e0], rtol=1e-10, atol=1e-14)
    a_ex, e_ex = sol.y[0, -1], sol.y[1, -1]
    assert (a1 - a0) == pytest.approx(a_ex - a0, rel=0.01)
    assert (e1 - e0) == pytest.approx(e_ex - e0, rel=0.01)
    # without P-R drag the elements hold
    P0 = oracle.params(_disk(beta0=beta, rad_s0=1e-3, rad_pr=0))
    x, y, z = np.array([rp]), np.array([0.0]), np.array([0.0])
    vr, lth, lp = np.zeros(1), np.zeros(1), np.array([lph0])
    for n in range(steps_per * orbits):
        oracle.push_rad(P0, x, y, z, vr, lth, lp, s, M, dt, 0.0, drag=False)
    a2, e2 = _elements(GMp, x[0], y[0], vr[0], lp[0])
    assert abs(a2 - a0) < 0.01 * abs(a_ex - a0) and abs(e2 - e0) < 0.01 * abs(e_ex - e0)


def _wall_and_probe(oracle, P, r_probe):
    """Wall particles at the centres of radial cell 2 of every column, with masses that give
    each column tau = ln 2 beyond it (cell volumes integrated numerically), and a probe
    of negligible mass at r_probe."""
    nr, nm, npf = 8, 4, 6
    dr, dmu, dph = AU, 0.1, 2 * math.pi / 6
    xs, ys, zs, Ms = [], [], [], []
    i = 2
    for j in range(nm):
        for k in range(npf):
            V = _cell_volume_3d(10 * AU + i * dr, 10 * AU + (i + 1) * dr, -0.2 + j * dmu,
                                -0.2 + (j + 1) * dmu, -math.pi + k * dph, -math.pi + (k + 1) * dph)
            x, y, z = _sph(10 * AU + (i + 0.5) * dr, -0.2 + (j + 0.5) * dmu, -math.pi + (k + 0.5) * dph)
            xs.append(x); ys.append(y); zs.append(z)
            Ms.append(math.log(2.0) * V / (2.0 * dr))     # kappa = 2 at s = rad_s0
    x, y, z = _sph(r_probe, 0.02, 0.4)
    xs.append(x); ys.append(y); zs.append(z); Ms.append(1e-6)
    n = len(xs)
    GM = G * W.MSUN
    vr = np.zeros(n)
    lth = np.zeros(n)
    lph = np.array([math.sqrt(GM * math.hypot(a, b)) * 0.9 for a, b in zip(xs, ys)])
    return [np.array(v) for v in (xs, ys, zs)] + [vr, lth, lph, np.full(n, 1e-3), np.array(Ms)]


@pytest.mark.parametrize("pr", [0, 1])
def test_shadow_equals_half_beta(oracle, pr):
    """beta e^-tau enters as one factor: behind a tau = ln 2 wall a grain moves as one with
    beta / 2 in free space (gas drag on)."""
    base = _grid3d(beta0=0.4, rad_pr=pr)
    P = oracle.params(base)
    x, y, z, vr, lth, lph, s, M = _wall_and_probe(oracle, P, 15.3 * AU)
    dt = 0.05 * 2 * math.pi * math.sqrt((15 * AU) ** 3 / (G * W.MSUN))
    oracle.push_rad(P, x, y, z, vr, lth, lph, s, M, dt, 0.0)
    P2 = oracle.params(dict(base, beta0=0.2, kappa0=0.0))
    x2, y2, z2, vr2, lth2, lph2, _, _ = _wall_and_probe(oracle, P2, 15.3 * AU)
    oracle.push_rad(P2, x2, y2, z2, vr2, lth2, lph2, s, M, dt, 0.0)
    for a, b in ((x, x2), (y, y2), (z, z2), (vr, vr2), (lth, lth2), (lph, lph2)):
        assert a[-1] == pytest.approx(b[-1], rel=1e-12, abs=1e-12 * abs(b[-1]) + 1e-300)
    # and differs from the unshadowed grain
    P3 = oracle.params(dict(base, kappa0=0.0))
    x3, y3, z3, vr3, lth3, lph3, _, _ = _wall_and_probe(oracle, P3, 15.3 * AU)
    oracle.push_rad(P3, x3, y3, z3, vr3, lth3, lph3, s, M, dt, 0.0)
    assert abs(vr3[-1] - vr[-1]) > 1e-3 * abs(vr[-1])


def test_taper_at_kick_time(oracle):
    """A taper of one half at t + dt/2 equals beta / 2 without a taper."""
    dt = 1e6
    t_beta = 1e8
    base = _disk(beta0=0.4, rad_s0=1e-3, rad_pr=1, t_beta=t_beta)
    ins = W.disk_instance(64, seed=9, velocities=True)
    outs = []
    for P, t in ((oracle.params(base), 0.5 * t_beta - 0.5 * dt),
                 (oracle.params(dict(base, beta0=0.2, t_beta=0.0)), 0.0)):
        st = [ins[k].copy() for k in ("x", "y", "z", "vr", "lth", "lph")]
        oracle.push_rad(P, *st, ins["s"], ins["M"], dt, t)
        outs.append(st)
    for a, b in zip(*outs):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-300)
    # evaluated at t instead, the factor would not be one half
    st = [ins[k].copy() for k in ("x", "y", "z", "vr", "lth", "lph")]
    oracle.push_rad(oracle.params(base), *st, ins["s"], ins["M"], dt, 0.5 * t_beta)
    assert np.abs(st[3] - outs[1][3]).max() > 1e-6 * np.abs(outs[1][3]).max()


def test_beta_two_eta_balances_headwind(oracle):
    """beta = 2 eta: the gas orbits at sqrt(1 - 2 eta) v_K = sqrt(1 - beta) v_K, the grain's
    own circular speed, so a grain started on it in the midplane feels no drag and stays;
    with beta = 0 it drifts inwards at the terminal rate."""
    P0 = oracle.params(_disk())
    R0 = 10 * AU
    g = oracle.gas(P0, R0, 0.0, 0.0)
    eta = g["eta"]
    s = 1e-1                                   # St ~ 0.1 at 10 au
    beta = 2 * eta
    lph = math.sqrt(1 - 2 * eta) * g["Om"] * R0 * R0
    dt = 0.02 * 2 * math.pi / g["Om"]
    for b, expect_still in ((beta, True), (0.0, False)):
        P = oracle.params(_disk(beta0=b, rad_s0=s))
        x, y, z = np.array([R0]), np.array([0.0]), np.array([0.0])
        vr, lth, lp = np.zeros(1), np.zeros(1), np.array([lph])
        for n in range(500):
            oracle.push_rad(P, x, y, z, vr, lth, lp, np.array([s]), np.array([1.0]), dt, 0.0)
        dr = math.hypot(x[0], y[0]) / R0 - 1
        if expect_still:
            assert abs(dr) < 1e-9
        else:
            # the terminal drift -2 eta St/(1 + St^2) v_K (first order in eta)
            St = g["gst"] * s
            assert dr == pytest.approx(-2 * eta * St / (1 + St * St) * g["Om"] * 500 * dt, rel=0.1)

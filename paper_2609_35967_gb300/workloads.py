"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws initial conditions (positions, diameters, particle
masses, velocities) and fills the per-instance parameter dicts.  It holds none
of the collision method's arithmetic: the disk formulas below are used only to
place particles (scale heights, column masses), and both the CUDA library and
the CPU oracle read the same arrays.  Every generator is deterministic in its
seed (numpy PCG64).

Units: cgs.  Diameters s = 2a.  Recipes:

* local patch (Sect. 2.1, periodic sector): centred at radius r, x (radial)
  and y (azimuthal) uniform over one gas scale height, z ~ N(0, (0.1 H_g)^2);
  monodisperse a = 1 um, rho_o = 1.67, dust-to-gas 0.01 (equal particle
  masses carrying the column's dust mass);
* global disk: Sigma_g = 1700 (R/au)^-1, T = 280 (R/au)^-0.5 over 5-100 au;
  dN/dR is constant for Sigma ~ 1/R with equal particle masses, so R is uniform,
  phi uniform, z ~ N(0, H_d^2) with the settling equilibrium
  H_d = H_g sqrt(alpha/(alpha + St));
* coagulation test (Appendix A): uniform positions in a periodic unit box,
  unit masses (constant / product kernel) or Gamma(2) masses (linear kernel);
* diffusion ring test (Sect. 3.2): code units R_0 = 1, D_0 = 1e-4, p = -1,
  ln(R/R_0) ~ N(0, 0.05^2), phi uniform, z = 0.
"""
from __future__ import annotations

import math

import numpy as np

AU = 1.495978707e13
YR = 3.15576e7
MSUN = 1.989e33
_G = 6.674e-8
_KB = 1.380649e-16
_MH = 1.6735575e-24
_MU = 2.34

PATCH, DISK = 0, 1
PHYSICAL, CONSTANT, LINEAR, PRODUCT = 0, 1, 2, 3
DIFF_PHYSICAL, DIFF_RING = 0, 1
MODEL_3D, MODEL_RZ, MODEL_RPHI, MODEL_R = 0, 1, 2, 3
S_MIN = 2e-5          # minimum fragment diameter: a = 0.1 um


def _scale_height(T, r):
    cs = math.sqrt(_KB * T / (_MU * _MH))
    om = math.sqrt(_G * MSUN / r ** 3)
    return cs / om, om


def _base_params(**kw):
    d = dict(geometry=PATCH, kernel_mode=PHYSICAL, K=32, audit=1, r0=10 * AU, sigma0=10.0,
             p=-1.0, q=-0.5, T0=50.0, alpha=1e-3, M_star=MSUN, rho_s=1.67, s_min=S_MIN,
             v_frag=100.0, eps=0.08, dt_coll=0.0, dt_fn_max=0.0, R_in=0.0, R_out=0.0,
             box_x=0.0, box_y=0.0, t0=1.0, m0=1.0, seed=1, max_events=1 << 16,
             cell_size=0.0, diff_mode=DIFF_PHYSICAL, diff_chi=1, Sc_R=1.0, Sc_Z=1.0, Sc_phi=1.0,
             D0=0.0)
    d.update(kw)
    return d


def patch_instance(n, r_au=10.0, sigma=10.0, T=50.0, alpha=1e-3, v_frag=100.0, seed=1, K=32,
                   a_um=1.0, rho_s=1.67, d2g=0.01, eps=0.08, hz=0.1, **extra):
    """One local 3D patch (configurations 0 and 3)."""
    r = r_au * AU
    H, om = _scale_height(T, r)
    rng = np.random.default_rng(seed)
    L = H
    x = rng.uniform(-0.5 * L, 0.5 * L, n)
    y = rng.uniform(-0.5 * L, 0.5 * L, n)
    z = rng.normal(0.0, hz * H, n)
    s = np.full(n, 2.0 * a_um * 1e-4)
    M = np.full(n, d2g * sigma * L * L / n)
    P = _base_params(geometry=PATCH, K=K, r0=r, sigma0=sigma, T0=T, alpha=alpha, rho_s=rho_s,
                     v_frag=v_frag, eps=eps, dt_coll=2 * math.pi / om, dt_fn_max=2 * math.pi / om,
                     box_x=L, box_y=L, seed=seed, **extra)
    return dict(params=P, x=x, y=y, z=z, s=s, M=M)


def _lognormal_diameters(rng, n, median_um, sigma_ln, s_min):
    s = 2e-4 * median_um * np.exp(sigma_ln * rng.normal(size=n))
    bad = s < s_min
    while bad.any():                     # truncate below s_min by resampling
        s[bad] = 2e-4 * median_um * np.exp(sigma_ln * rng.normal(size=int(bad.sum())))
        bad = s < s_min
    return s


def disk_instance(n, seed=1, K=32, alpha=1e-3, v_frag=100.0, sizes=("mono", 1.0),
                  R_in_au=5.0, R_out_au=100.0, sigma_1au=1700.0, T_1au=280.0, rho_s=1.67,
                  d2g=0.01, eps=0.08, velocities=False, **extra):
    """One global 3D disk (configurations 1, 2 and 4)."""
    rng = np.random.default_rng(seed)
    R = rng.uniform(R_in_au * AU, R_out_au * AU, n)
    phi = rng.uniform(0.0, 2 * math.pi, n)
    if sizes[0] == "mono":
        s = np.full(n, 2e-4 * sizes[1])
    else:
        s = _lognormal_diameters(rng, n, sizes[1], sizes[2], S_MIN)
    T = T_1au * (R / AU) ** -0.5
    sig = sigma_1au * (R / AU) ** -1.0
    cs = np.sqrt(_KB * T / (_MU * _MH))
    om = np.sqrt(_G * MSUN / R ** 3)
    Hg = cs / om
    St = math.pi * rho_s * s / (4.0 * sig)
    Hd = Hg * np.sqrt(alpha / (alpha + St))
    z = rng.normal(size=n) * Hd
    x, y = R * np.cos(phi), R * np.sin(phi)
    Mdust = d2g * 2 * math.pi * sigma_1au * AU * (R_out_au - R_in_au) * AU
    M = np.full(n, Mdust / n)
    om5 = math.sqrt(_G * MSUN / (R_in_au * AU) ** 3)
    P = _base_params(geometry=DISK, K=K, r0=AU, sigma0=sigma_1au, T0=T_1au, alpha=alpha,
                     rho_s=rho_s, v_frag=v_frag, eps=eps, dt_coll=2 * math.pi / om5,
                     dt_fn_max=2 * math.pi / om5, R_in=R_in_au * AU, R_out=R_out_au * AU,
                     seed=seed, **extra)
    out = dict(params=P, x=x, y=y, z=z, s=s, M=M)
    if velocities:
        # start at the gas velocity: v_r = l_theta = 0, l_phi = R v_g,phi
        # (Sect. 2.2, the analytic azimuthal gas velocity).
        h = Hg / R
        r = np.sqrt(R * R + z * z)
        eta = -0.5 * ((-1.0 - 0.25 - 1.5) * h * h - 0.5 * (1.0 - R / r))
        out["vr"] = np.zeros(n)
        out["lth"] = np.zeros(n)
        out["lph"] = np.sqrt(1.0 - 2.0 * eta) * om * R * R
    return out


def coag_instance(n, K=32, mode=CONSTANT, seed=1, eps=0.08, dt_coll=1.0, **extra):
    """Appendix A coagulation test: periodic unit box, V_i = 1, m_0 = t_0 = 1."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-0.5, 0.5, n)
    y = rng.uniform(-0.5, 0.5, n)
    z = rng.uniform(-0.5, 0.5, n)
    rho_s = 6.0 / math.pi                # s = m^(1/3) in these units
    if mode == LINEAR:
        m = rng.gamma(2.0, 1.0, n)
    else:
        m = np.ones(n)
    s = np.cbrt(6.0 * m / (math.pi * rho_s))
    M = np.full(n, 1.0 / n)
    P = _base_params(geometry=PATCH, kernel_mode=mode, K=K, r0=AU, sigma0=1.0, T0=100.0,
                     rho_s=rho_s, s_min=1e-30, v_frag=1e30, eps=eps, dt_coll=dt_coll,
                     dt_fn_max=dt_coll, box_x=1.0, box_y=1.0, t0=1.0, m0=1.0, seed=seed,
                     **extra)
    return dict(params=P, x=x, y=y, z=z, s=s, M=M)


def ring_params(chi=1, seed=1):
    """Parameters of the diffusion ring test (Sect. 3.2), code units."""
    return _base_params(geometry=DISK, r0=1.0, p=-1.0, diff_mode=DIFF_RING, diff_chi=chi, D0=1e-4,
                        R_in=0.0, R_out=1e3, seed=seed, dt_coll=1.0, dt_fn_max=1.0)


def ring_instance(n, chi=1, seed=1, K=16):
    """Diffusion ring test: ln(R/R_0) ~ N(0, 0.05^2), phi uniform, z = 0."""
    rng = np.random.default_rng(seed)
    lnR = rng.normal(0.0, 0.05, n)
    ph = rng.uniform(0.0, 2 * math.pi, n)
    R = np.exp(lnR)
    P = ring_params(chi=chi, seed=seed)
    P["K"] = K
    return dict(params=P, x=R * np.cos(ph), y=R * np.sin(ph), z=np.zeros(n), s=np.full(n, 1e-4),
                M=np.full(n, 1.0 / n))


# ---------------------------------------------------------------- configurations

def config0(n=4096, K=32):
    """Plain FP64 local patch at 10 au, 4096 particles, seed 1, 100 intervals."""
    return [patch_instance(n, r_au=10.0, sigma=10.0, T=50.0, alpha=1e-3, v_frag=100.0,
                           seed=1, K=K)]


def config1(n=1 << 20, K=32, seed=1):
    """Global disk, 2^20 particles, a = 1 um, K = 32, v_frag = 1 m/s."""
    return [disk_instance(n, seed=seed, K=K, alpha=1e-3, v_frag=100.0, sizes=("mono", 1.0))]


def config2(n=1 << 22, K=32, seed=1):
    """Same disk, 2^22 particles, log-normal sizes (median 10 um, sigma_ln = 1)."""
    return [disk_instance(n, seed=seed, K=K, alpha=1e-3, v_frag=100.0,
                          sizes=("lognormal", 10.0, 1.0))]


def config3(n_patches=256, K=32, seed0=1000, log2_min=10.0, log2_max=16.0):
    """Independent patches of uneven size and parameters (seed_b = seed0 + b)."""
    meta = np.random.default_rng(seed0 - 1)
    out = []
    for b in range(n_patches):
        n = int(math.floor(2.0 ** meta.uniform(log2_min, log2_max)))
        alpha = 10.0 ** meta.uniform(-4.0, -2.0)
        v_frag = meta.uniform(100.0, 1000.0)
        r_au = meta.uniform(5.0, 50.0)
        sigma = 10.0 * (r_au / 10.0) ** -1.0
        T = 50.0 * (r_au / 10.0) ** -0.5
        out.append(patch_instance(max(n, K), r_au=r_au, sigma=sigma, T=T, alpha=alpha,
                                  v_frag=v_frag, seed=seed0 + b, K=K))
    return out


def config4(n=1 << 24, K=48, seed=1):
    """Large disk: 2^24 particles, log-normal (median 1 um, sigma_ln 0.5), K = 48."""
    return [disk_instance(n, seed=seed, K=K, alpha=3e-3, v_frag=500.0,
                          sizes=("lognormal", 1.0, 0.5), velocities=True)]


def concat(instances):
    """CSR concatenation of instances: (offsets[n+1], arrays..., list of params)."""
    offs = np.zeros(len(instances) + 1, dtype=np.int64)
    for b, ins in enumerate(instances):
        offs[b + 1] = offs[b] + len(ins["x"])
    cat = {k: np.concatenate([ins[k] for ins in instances])
           for k in ("x", "y", "z", "s", "M")}
    for k in ("vr", "lth", "lph"):
        if all(k in ins for ins in instances):
            cat[k] = np.concatenate([ins[k] for ins in instances])
    cat["offsets"] = offs
    cat["params"] = [ins["params"] for ins in instances]
    return cat

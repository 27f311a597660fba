"""ctypes wrapper of the plain FP64 CPU oracle (oracle/gdo.c).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import this module.  It imports
nothing from the CUDA package; inputs come from the seeded generators in
paper_2609_35967_gb300.workloads (which hold none of the method's arithmetic).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gdo.c")
_LIB = os.path.join(_HERE, "libgdo.so")
_lock = threading.Lock()
_lib = None

PATCH, DISK = 0, 1
PHYSICAL, CONSTANT, LINEAR, PRODUCT = 0, 1, 2, 3
NFINE = 96


def build(force: bool = False) -> str:
    """Compile gdo.c with gcc (-O2, no FP contraction) into oracle/libgdo.so."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(os.path.join(_HERE, "gdo.h")))):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("geometry", C.c_int32), ("kernel_mode", C.c_int32), ("K", C.c_int32),
                ("audit", C.c_int32),
                ("r0", C.c_double), ("sigma0", C.c_double), ("p", C.c_double),
                ("T0", C.c_double), ("q", C.c_double), ("alpha", C.c_double),
                ("M_star", C.c_double), ("rho_s", C.c_double), ("s_min", C.c_double),
                ("v_frag", C.c_double), ("eps", C.c_double), ("dt_coll", C.c_double),
                ("dt_fn_max", C.c_double), ("R_in", C.c_double), ("R_out", C.c_double),
                ("box_x", C.c_double), ("box_y", C.c_double), ("t0", C.c_double),
                ("m0", C.c_double), ("seed", C.c_uint64), ("max_events", C.c_int64),
                ("diff_mode", C.c_int32), ("diff_chi", C.c_int32), ("Sc_R", C.c_double),
                ("Sc_Z", C.c_double), ("Sc_phi", C.c_double), ("D0", C.c_double),
                ("model", C.c_int32), ("pad_model", C.c_int32),
                ("beta0", C.c_double), ("kappa0", C.c_double), ("rad_s0", C.c_double),
                ("t_beta", C.c_double), ("rad_pr", C.c_int32), ("tau_geom", C.c_int32),
                ("tau_nr", C.c_int32), ("tau_nmu", C.c_int32), ("tau_nphi", C.c_int32),
                ("pad_tau", C.c_int32), ("tau_rmin", C.c_double), ("tau_rmax", C.c_double),
                ("tau_mu", C.c_double)]


class State(C.Structure):
    _fields_ = [("C", C.c_double), ("dt_remain", C.c_double), ("dt_exe", C.c_double),
                ("dt_req", C.c_double), ("remain_ticks", C.c_int64), ("interval", C.c_int64), ("events", C.c_int64),
                ("near_draw", C.c_int64), ("near_dt", C.c_int64), ("near_audit", C.c_int64),
                ("status", C.c_int64), ("n_groups", C.c_int32), ("pad", C.c_int32)]


MAXG = 64


class Groups(C.Structure):
    _fields_ = [("n_groups", C.c_int32), ("pad", C.c_int32), ("t", C.c_int64),
                ("rounds", C.c_int64), ("delayed", C.c_int64), ("breaks", C.c_int64),
                ("level", C.c_int32 * MAXG), ("k_req", C.c_int32 * MAXG),
                ("active", C.c_int32 * MAXG), ("pad2", C.c_int32),
                ("members", C.c_int64 * MAXG), ("intervals", C.c_int64 * MAXG),
                ("inter", C.c_uint64 * MAXG), ("st", State * MAXG)]


class Gas(C.Structure):
    _fields_ = [(k, C.c_double) for k in
                ("R", "Z", "r", "Om", "T", "cs", "H", "h", "Sigma", "rho_g", "eta", "Re", "gst")]


class Pair(C.Structure):
    _fields_ = [("dvR", C.c_double), ("dvZ", C.c_double), ("dvphi", C.c_double),
                ("dvB", C.c_double), ("dvt", C.c_double), ("dv", C.c_double),
                ("Kij", C.c_double), ("lam", C.c_double), ("psi", C.c_double),
                ("ncoll", C.c_double), ("outcome", C.c_int32), ("pad", C.c_int32),
                ("c", C.c_double * 2), ("J1", C.c_double * 2), ("J2", C.c_double * 2)]


class Outputs(C.Structure):
    _fields_ = [("nbr", C.c_void_p), ("d", C.c_void_p), ("V", C.c_void_p),
                ("lam", C.c_void_p), ("mA", C.c_void_p), ("mB", C.c_void_p),
                ("chan", C.c_void_p), ("ev_count", C.c_void_p), ("ev_hash", C.c_void_p),
                ("near", C.c_void_p), ("jsum", C.c_void_p), ("A_b", C.c_void_p),
                ("B_b", C.c_void_p)]


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            vp, i64, dbl = C.c_void_p, C.c_int64, C.c_double
            L.gdo_philox4x32_10.argtypes = [vp, vp, vp]
            L.gdo_u01.argtypes = [C.c_uint32, C.c_uint32]
            L.gdo_u01.restype = dbl
            L.gdo_gas_at.argtypes = [vp, dbl, dbl, dbl, vp]
            L.gdo_knn_one.argtypes = [vp, i64, vp, vp, vp, i64, vp, vp]
            L.gdo_volume.argtypes = [vp, dbl, dbl]
            L.gdo_volume.restype = dbl
            L.gdo_grain_mass.argtypes = [vp, dbl]
            L.gdo_grain_mass.restype = dbl
            L.gdo_frag_moments.argtypes = [dbl, dbl, vp, vp]
            L.gdo_turb_dv2.argtypes = [dbl, dbl, dbl, dbl]
            L.gdo_turb_dv2.restype = dbl
            L.gdo_pair.argtypes = [vp, vp, dbl, dbl, dbl, dbl, dbl, dbl, vp]
            L.gdo_fine_bin.argtypes = [dbl]
            L.gdo_fine_bin.restype = C.c_int
            L.gdo_choose_interval.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
            L.gdo_choose_interval_ab.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
            L.gdo_audit.argtypes = [vp, i64, vp, vp, vp, C.c_int32, vp]
            L.gdo_interval_step.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp]
            L.gdo_rates_subset.argtypes = [vp, i64, vp, vp, vp, vp, vp, i64, vp, vp, vp,
                                           vp, vp, vp, vp]
            L.gdo_sample_subset.argtypes = [vp, i64, vp, vp, vp, vp, vp, i64, vp, vp, vp,
                                            dbl, i64, vp, vp, vp, vp, vp, vp]
            L.gdo_push_one.argtypes = [vp, C.c_int32, dbl, vp, vp, vp, vp, vp, vp, dbl]
            L.gdo_push.argtypes = [vp, C.c_int32, dbl, i64, vp, vp, vp, vp, vp, vp, vp]
            L.gdo_params_size.argtypes = []
            L.gdo_params_size.restype = i64
            assert L.gdo_params_size() == C.sizeof(Params), "gdo_params layout differs"
            L.gdo_rad_beta.argtypes = [vp, dbl]
            L.gdo_rad_beta.restype = dbl
            L.gdo_rad_kappa.argtypes = [vp, dbl]
            L.gdo_rad_kappa.restype = dbl
            L.gdo_rad_taper.argtypes = [vp, dbl]
            L.gdo_rad_taper.restype = dbl
            L.gdo_tau_size.argtypes = [vp]
            L.gdo_tau_size.restype = i64
            L.gdo_tau_grid.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
            L.gdo_tau_at.argtypes = [vp, vp, dbl, dbl, dbl]
            L.gdo_tau_at.restype = dbl
            L.gdo_push_rad.argtypes = [vp, C.c_int32, dbl, dbl, i64, vp, vp, vp, vp, vp, vp, vp, vp,
                                       vp, vp]
            L.gdo_diff_coeffs.argtypes = [vp, dbl, dbl, dbl, vp]
            L.gdo_diffuse.argtypes = [vp, dbl, i64, i64, vp, vp, vp, vp, vp, vp, vp]
            L.gdo_local_dt.argtypes = [vp, vp, dbl, dbl, dbl, dbl, vp]
            L.gdo_local_dt.restype = dbl
            L.gdo_timestep.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
            L.gdo_timestep.restype = dbl
            L.gdo_group_of.argtypes = [vp, C.c_int32, dbl, dbl]
            L.gdo_group_of.restype = C.c_int32
            L.gdo_groups_reset.argtypes = [vp, C.c_int32, vp]
            L.gdo_groups_assign.argtypes = [vp, i64, vp, vp, vp, vp, vp]
            L.gdo_schedule.argtypes = [C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp]
            L.gdo_group_round.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            L.gdo_group_round.restype = C.c_int
            L.gdo_collide_groups.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, C.c_int32]
            L.gdo_collide_groups.restype = C.c_int
            _lib = L
    return _lib


_PARAM_KEYS = [f for f, _ in Params._fields_]


def params(d: dict) -> Params:
    """Oracle parameter struct from an instance dict (extra keys are ignored)."""
    P = Params()
    for k in _PARAM_KEYS:
        if k in d:
            setattr(P, k, d[k])
    if "max_events" not in d:
        P.max_events = 1 << 20
    for k in ("Sc_R", "Sc_Z", "Sc_phi"):
        if k not in d:
            setattr(P, k, 1.0)
    if "diff_chi" not in d:
        P.diff_chi = 1
    return P


def new_state(P: Params) -> State:
    st = State()
    st.C = 1.0
    st.dt_remain = P.dt_coll
    st.remain_ticks = 1 << 60
    st.interval = 0
    return st


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().gdo_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def u01(a: int, b: int) -> float:
    return lib().gdo_u01(a, b)


def gas(P: Params, x: float, y: float, z: float) -> dict:
    g = Gas()
    lib().gdo_gas_at(C.byref(P), x, y, z, C.byref(g))
    return {k: getattr(g, k) for k, _ in Gas._fields_}


def gas_struct(P: Params, x: float, y: float, z: float) -> Gas:
    g = Gas()
    lib().gdo_gas_at(C.byref(P), x, y, z, C.byref(g))
    return g


def knn(P: Params, x, y, z, queries) -> tuple[np.ndarray, np.ndarray]:
    """Brute-force lists for the given query indices: ([nq, K] int32, [nq] d)."""
    x, y, z = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z))
    q = np.asarray(queries, dtype=np.int64)
    nbr = np.zeros((len(q), P.K), dtype=np.int32)
    d = np.zeros(len(q), dtype=np.float64)
    L = lib()
    dv = C.c_double()
    for t, i in enumerate(q):
        rc = L.gdo_knn_one(C.byref(P), len(x), _p(x), _p(y), _p(z), int(i),
                           nbr[t].ctypes.data_as(C.c_void_p), C.byref(dv))
        if rc != 0:
            raise ValueError("instance holds fewer than K particles")
        d[t] = dv.value
    return nbr, d


def volume(P: Params, d: float, R: float) -> float:
    return lib().gdo_volume(C.byref(P), d, R)


def grain_mass(P: Params, s: float) -> float:
    return lib().gdo_grain_mass(C.byref(P), s)


def frag_moments(s_i: float, s_min: float) -> tuple[float, float]:
    a, b = C.c_double(), C.c_double()
    lib().gdo_frag_moments(s_i, s_min, C.byref(a), C.byref(b))
    return a.value, b.value


def turb_dv2(sa, sb, vg2, re) -> float:
    return lib().gdo_turb_dv2(sa, sb, vg2, re)


def pair(P: Params, g: Gas, s_i, m_i, s_j, m_j, N_j, V_i) -> dict:
    o = Pair()
    lib().gdo_pair(C.byref(P), C.byref(g), s_i, m_i, s_j, m_j, N_j, V_i, C.byref(o))
    r = {k: getattr(o, k) for k, _ in Pair._fields_ if k not in ("c", "J1", "J2", "pad")}
    r["c"] = list(o.c)
    r["J1"] = list(o.J1)
    r["J2"] = list(o.J2)
    return r


def fine_bin(s: float) -> int:
    return lib().gdo_fine_bin(s)


def choose_interval(P: Params, st: State, s, M, mA, mB, moments=False):
    """Interval choice of one instance; returns the controller bin of each particle, and
    with moments=True also (A_b, B_b) of the first st.n_groups bins."""
    s, M, mA, mB = (np.ascontiguousarray(a, dtype=np.float64) for a in (s, M, mA, mB))
    grp = np.zeros(len(s), dtype=np.int32)
    A = np.zeros(NFINE)
    B = np.zeros(NFINE)
    lib().gdo_choose_interval_ab(C.byref(P), len(s), _p(s), _p(M), _p(mA), _p(mB),
                                 C.byref(st), _p(grp), _p(A), _p(B))
    if moments:
        return grp, A[:st.n_groups], B[:st.n_groups]
    return grp


def audit(P: Params, st: State, M, jsum, grp, n_groups):
    M, jsum = (np.ascontiguousarray(a, dtype=np.float64) for a in (M, jsum))
    grp = np.ascontiguousarray(grp, dtype=np.int32)
    lib().gdo_audit(C.byref(P), len(M), _p(M), _p(jsum), _p(grp), n_groups, C.byref(st))


def interval_step(P: Params, st: State, x, y, z, s, M, want=("nbr", "d", "V", "lam",
                  "ev_count", "ev_hash", "near")) -> dict:
    """One whole interval of one instance; s (float64 array) is updated in place."""
    x, y, z, M = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, M))
    assert s.dtype == np.float64 and s.flags.c_contiguous
    n, K = len(x), P.K
    shapes = {"nbr": ((n, K), np.int32), "d": (n, np.float64), "V": (n, np.float64),
              "lam": (n, np.float64), "mA": (n, np.float64), "mB": (n, np.float64),
              "chan": ((n, K, 2), np.float64), "ev_count": (n, np.int32),
              "ev_hash": (n, np.uint32), "near": (n, np.int32), "jsum": (n, np.float64),
              "A_b": (NFINE, np.float64), "B_b": (NFINE, np.float64)}
    res = {k: np.zeros(*shapes[k]) for k in want}
    out = Outputs(**{k: _p(v) for k, v in res.items()})
    rc = lib().gdo_interval_step(C.byref(P), n, _p(x), _p(y), _p(z), _p(s), _p(M),
                                 C.byref(st), C.byref(out))
    if rc != 0:
        raise ValueError("oracle interval failed (instance smaller than K?)")
    return res


def rates_subset(P: Params, x, y, z, s, M, queries, nbr, d, chan=False) -> dict:
    x, y, z, s, M = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, s, M))
    q = np.ascontiguousarray(queries, dtype=np.int64)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    d = np.ascontiguousarray(d, dtype=np.float64)
    nq = len(q)
    lam, mA, mB = np.zeros(nq), np.zeros(nq), np.zeros(nq)
    ch = np.zeros((nq, P.K, 2)) if chan else None
    lib().gdo_rates_subset(C.byref(P), len(x), _p(x), _p(y), _p(z), _p(s), _p(M), nq, _p(q),
                           _p(nbr), _p(d), _p(lam), _p(mA), _p(mB), _p(ch))
    r = {"lam": lam, "mA": mA, "mB": mB}
    if chan:
        r["chan"] = ch
    return r


def sample_subset(P: Params, x, y, z, s0, M, queries, nbr, d, dt_exe, interval) -> dict:
    x, y, z, s0, M = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, s0, M))
    q = np.ascontiguousarray(queries, dtype=np.int64)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    d = np.ascontiguousarray(d, dtype=np.float64)
    nq = len(q)
    s_q = np.zeros(nq)
    ec = np.zeros(nq, dtype=np.int32)
    eh = np.zeros(nq, dtype=np.uint32)
    nn = np.zeros(nq, dtype=np.int32)
    js = np.zeros(nq)
    status = C.c_int64(0)
    lib().gdo_sample_subset(C.byref(P), len(x), _p(x), _p(y), _p(z), _p(s0), _p(M), nq, _p(q),
                            _p(nbr), _p(d), dt_exe, interval, _p(s_q), _p(ec), _p(eh), _p(nn),
                            _p(js), C.byref(status))
    return {"s": s_q, "ev_count": ec, "ev_hash": eh, "near": nn, "jsum": js,
            "status": status.value}


def push(P: Params, x, y, z, vr, lth, lph, s, dt, drag=True):
    """One staggered semi-analytic step of every particle, in place (float64 arrays)."""
    for arr in (x, y, z, vr, lth, lph):
        assert arr.dtype == np.float64 and arr.flags.c_contiguous
    s = np.ascontiguousarray(s, dtype=np.float64)
    lib().gdo_push(C.byref(P), 1 if drag else 0, dt, len(x), _p(x), _p(y), _p(z), _p(vr),
                   _p(lth), _p(lph), _p(s))


def rad_beta(P: Params, s: float) -> float:
    """beta(s) of Sect. 2.3.2."""
    return lib().gdo_rad_beta(C.byref(P), s)


def rad_kappa(P: Params, s: float) -> float:
    """kappa(s) of Sect. 2.3.2."""
    return lib().gdo_rad_kappa(C.byref(P), s)


def rad_taper(P: Params, t: float) -> float:
    """The taper xi^2 (3 - 2 xi) of the radiation forces at time t."""
    return lib().gdo_rad_taper(C.byref(P), t)


def tau_grid(P: Params, x, y, z, s, M) -> np.ndarray:
    """Optical depth at the radial faces of every grid column, T[column, face]
    (column = j * nphi + k), from the particles at (x, y, z)."""
    n = len(x)
    size = lib().gdo_tau_size(C.byref(P))
    T = np.zeros(max(size, 1))
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, s, M)]
    lib().gdo_tau_grid(C.byref(P), n, *[_p(a) for a in arrs], _p(T))
    return T[:size]


def tau_at(P: Params, T, x: float, y: float, z: float) -> float:
    """tau at one point, interpolated from the face grid T."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    return lib().gdo_tau_at(C.byref(P), _p(T), x, y, z)


def push_rad(P: Params, x, y, z, vr, lth, lph, s, M, dt, t, drag=True):
    """One staggered step with radiation forces, in place; returns the grid T built at
    the first drift's midpoints and those midpoints (r, theta, phi) as a [3, n] array."""
    for arr in (x, y, z, vr, lth, lph):
        assert arr.dtype == np.float64 and arr.flags.c_contiguous
    n = len(x)
    s = np.ascontiguousarray(s, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64)
    T = np.zeros(max(lib().gdo_tau_size(C.byref(P)), 1))
    mid = np.zeros(3 * max(n, 1))
    lib().gdo_push_rad(C.byref(P), 1 if drag else 0, dt, t, n, _p(x), _p(y), _p(z), _p(vr),
                       _p(lth), _p(lph), _p(s), _p(M), _p(T), _p(mid))
    return T[:lib().gdo_tau_size(C.byref(P))], mid[:3 * n].reshape(3, n)


def diff_coeffs(P: Params, R: float, Z: float, s: float) -> np.ndarray:
    """D_R, D_Z, D_phi, the R and Z drift coefficients, dln rho_g/dR, dln rho_g/dZ."""
    out = np.zeros(7)
    lib().gdo_diff_coeffs(C.byref(P), R, Z, s, _p(out))
    return out


def diffuse(P: Params, dt, step, x, y, z, s, vr=None, lth=None, lph=None):
    """One Euler-Maruyama diffusion step of every particle of one instance, in place."""
    for arr in (x, y, z):
        assert arr.dtype == np.float64 and arr.flags.c_contiguous
    s = np.ascontiguousarray(s, dtype=np.float64)
    v = (vr, lth, lph)
    ptrs = [_p(a) if a is not None else None for a in v]
    lib().gdo_diffuse(C.byref(P), dt, step, len(x), _p(x), _p(y), _p(z), *ptrs, _p(s))


class DtRule(C.Structure):
    _fields_ = [("dt_max", C.c_double), ("dt_out", C.c_double), ("f_orb", C.c_double),
                ("dx_H", C.c_double), ("c_adv", C.c_double), ("c_diff", C.c_double)]


def dt_rule(dt_max, dt_out=math.inf, f_orb=0.0, dx_H=0.0, c_adv=0.0, c_diff=0.0) -> DtRule:
    return DtRule(dt_max, dt_out, f_orb, dx_H, c_adv, c_diff)


def local_dt(P: Params, rule: DtRule, x, y, z, s, v=None) -> float:
    """Delta t_i of one particle (Sect. 2.6); v = (v_r, l_theta, l_phi) or None."""
    vv = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    return lib().gdo_local_dt(C.byref(P), C.byref(rule), x, y, z, s, None if vv is None else _p(vv))


def timestep(P: Params, rule: DtRule, x, y, z, s, vr=None, lth=None, lph=None):
    """Delta t = min(dt_max, dt_out, min_i Delta t_i) over one instance, and every Delta t_i."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, s)]
    vs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (vr, lth, lph)]
    dti = np.zeros(len(arrs[0]))
    dt = lib().gdo_timestep(C.byref(P), C.byref(rule), len(dti), *[_p(a) for a in arrs],
                            *[None if a is None else _p(a) for a in vs], _p(dti))
    return dt, dti


# ---------------------------------------------------------------- spatial groups
def group_of(P: Params, G: int, x: float, y: float) -> int:
    return lib().gdo_group_of(C.byref(P), G, x, y)


def new_groups(P: Params, G: int) -> Groups:
    assert 1 <= G <= MAXG
    S = Groups()
    lib().gdo_groups_reset(C.byref(P), G, C.byref(S))
    return S


def schedule(G, inter, members, active, k_req, k_fit, level):
    """Levels of the active groups (gdo_schedule); level is updated in place and
    (delayed, breaks) returned."""
    inter = np.ascontiguousarray(inter, dtype=np.uint64)
    members = np.ascontiguousarray(members, dtype=np.int64)
    active, k_req, k_fit = (np.ascontiguousarray(a, dtype=np.int32) for a in (active, k_req, k_fit))
    assert level.dtype == np.int32 and level.flags.c_contiguous
    d = C.c_int64(0)
    b = C.c_int64(0)
    lib().gdo_schedule(G, _p(inter), _p(members), _p(active), _p(k_req), _p(k_fit), _p(level),
                       C.byref(d), C.byref(b))
    return d.value, b.value


class GroupRun:
    """Rounds of one instance split into spatial groups: lists, measures and gas once
    (positions are frozen in a collision step), live sizes s and the partner snapshot s0."""

    def __init__(self, P: Params, G: int, x, y, z, s, M, S: Groups | None = None):
        self.P = P
        self.x, self.y, self.z, self.M = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, M))
        self.s = np.array(s, dtype=np.float64)
        self.s0 = self.s.copy()
        n, K = len(self.x), P.K
        self.nbr, d = knn(P, self.x, self.y, self.z, np.arange(n))
        self.nbr = np.ascontiguousarray(self.nbr, dtype=np.int32)
        self.gas = (Gas * n)()
        L = lib()
        for i in range(n):
            L.gdo_gas_at(C.byref(P), self.x[i], self.y[i], self.z[i], C.byref(self.gas[i]))
        self.V = np.array([volume(P, d[i], self.gas[i].R) if P.kernel_mode == PHYSICAL else 1.0
                           for i in range(n)])
        self.S = S if S is not None else new_groups(P, G)
        self.grp = np.zeros(n, dtype=np.int32)
        L.gdo_groups_assign(C.byref(P), n, _p(self.x), _p(self.y), _p(self.nbr), _p(self.grp),
                            C.byref(self.S))

    def round(self, want=("ev_count", "ev_hash", "near")) -> dict:
        n = len(self.x)
        shapes = {"lam": (n, np.float64), "ev_count": (n, np.int32), "ev_hash": (n, np.uint32),
                  "near": (n, np.int32), "jsum": (n, np.float64)}
        res = {k: np.zeros(*shapes[k]) for k in want}
        out = Outputs(**{k: _p(v) for k, v in res.items()})
        res["new_step"] = lib().gdo_group_round(C.byref(self.P), n, _p(self.nbr), _p(self.V), self.gas,
                                                _p(self.s), _p(self.s0), _p(self.M), _p(self.grp),
                                                C.byref(self.S), C.byref(out))
        return res

    def done(self) -> bool:
        S = self.S
        return all(S.members[g] == 0 or S.st[g].remain_ticks == 0 for g in range(S.n_groups))


def collide_groups(P: Params, G: int, x, y, z, s, M, S: Groups | None = None, max_rounds=1 << 20):
    """A whole collision step of one instance in G spatial groups; s (float64) is updated
    in place.  Returns (rounds, groups state)."""
    x, y, z, M = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, M))
    assert s.dtype == np.float64 and s.flags.c_contiguous
    S = S if S is not None else new_groups(P, G)
    rc = lib().gdo_collide_groups(C.byref(P), len(x), _p(x), _p(y), _p(z), _p(s), _p(M), C.byref(S),
                                  max_rounds)
    if rc < 0:
        raise ValueError("oracle collision step failed (%d)" % rc)
    return rc, S

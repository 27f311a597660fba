"""GPU common transport timestep (Sect. 2.6) against the oracle.

* FP64 form: every particle's local limit dt_i within 1e-12 relative (both sides FP64;
  they differ only in the last bits of pow, exp and sqrt), +infinity at the same
  particles, and the global dt within 1e-12 of the oracle's minimum over the instances,
  for a disk with velocities, local patches and the ring model in one context.
* Mixed form (FP32 limits): 2e-5 relative, plus 1e-13 of the Keplerian speed over |u_i|
  for the deterministic limit (its l_phi / R - v_K is formed from an FP64 difference of
  squares, so only the rounding of the inputs remains); where the oracle has no
  deterministic limit (u_i = 0) the FP32 one must not bind.
* The bounds dt_max and dt_out, the limits switched off, the argument checks, and a
  particle at R = 0 (no finite limit) reported as GD_ERR_NONFINITE.
* The full-size bench disk (2^22 particles): dt_i on a sample against the oracle and dt
  equal to the minimum of the returned dt_i.
"""
import math

import numpy as np
import pytest

from paper_2609_35967_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RULE = dict(f_orb=0.05, dx_H=0.1, c_adv=0.5, c_diff=0.5)


def _oracle_dt(oracle, insts, rule, velocities):
    dts, dtis = [], []
    for ins in insts:
        P = oracle.params(ins["params"])
        v = [ins[k] for k in ("vr", "lth", "lph")] if velocities else [None, None, None]
        dt, dti = oracle.timestep(P, oracle.dt_rule(**rule), ins["x"], ins["y"], ins["z"], ins["s"], *v)
        dts.append(dt)
        dtis.append(dti)
    return min(dts), np.concatenate(dtis)


def _mixed_context():
    disk = W.disk_instance(3000, seed=81, sizes=("lognormal", 10.0, 1.0), velocities=True, alpha=1e-2)
    # velocities off the gas motion, so the deterministic limit binds somewhere
    rng = np.random.default_rng(5)
    disk["vr"] = rng.normal(0.0, 3e3, 3000)
    disk["lth"] = rng.normal(0.0, 3e3, 3000) * np.sqrt(disk["x"] ** 2 + disk["y"] ** 2)
    p1 = W.patch_instance(700, seed=82, alpha=1e-3)
    p2 = W.patch_instance(900, seed=83, r_au=30.0, alpha=1e-2)
    for p in (p1, p2):
        p["vr"], p["lth"], p["lph"] = np.zeros(len(p["x"])), np.zeros(len(p["x"])), np.zeros(len(p["x"]))
    ring = W.ring_instance(800, chi=1, seed=84)
    ring["vr"], ring["lth"] = np.zeros(800), np.zeros(800)
    # sub-Keplerian by 0.1-0.2% (an exact Kepler orbit has u_i at the rounding level)
    ring["lph"] = np.sqrt(6.674e-8 * W.MSUN * np.hypot(ring["x"], ring["y"])) * (1.0 - 1e-3 * (1.0 + rng.random(800)))
    return [disk, p1, p2, ring]


def _speed_ratio(insts, velocities):
    """v_K / |u_i| of every particle (0 where the deterministic limit does not apply)."""
    out = []
    GM = 6.674e-8 * W.MSUN
    for ins in insts:
        n = len(ins["x"])
        if not velocities or ins["params"]["geometry"] != W.DISK:
            out.append(np.zeros(n))
            continue
        R = np.hypot(ins["x"], ins["y"])
        r = np.hypot(R, ins["z"])
        vK = np.sqrt(GM / R)
        u = np.sqrt(ins["vr"] ** 2 + (ins["lth"] / r) ** 2 + (ins["lph"] / R - vK) ** 2)
        out.append(vK / np.maximum(u, 1e-300 * vK))
    return np.concatenate(out)


def _compare(dti, odti, tol):
    inf = np.isinf(odti)
    fin = ~inf
    assert np.all(np.abs(dti[fin] / odti[fin] - 1.0) <= tol[fin]), \
        np.max(np.abs(dti[fin] / odti[fin] - 1.0) / tol[fin])
    if inf.any():
        # no limit in the oracle: none, or one that cannot bind, on the GPU
        floor = np.median(odti[fin]) * 1e3 if fin.any() else 0.0
        assert np.all(dti[inf] > floor)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("velocities", [False, True])
def test_timestep_parity(gd, oracle, precision, velocities):
    insts = _mixed_context()
    sess = gd.Session(insts, precision=precision, velocities=velocities)
    ratio = _speed_ratio(insts, velocities)
    base = np.full(len(ratio), 1e-12 if precision == 0 else 2e-5)
    rule = dict(dt_max=1e30, **RULE)
    dt, dti = sess.timestep(**rule, want=True)
    dti = dti.cpu().numpy()
    odt, odti = _oracle_dt(oracle, insts, rule, velocities)
    tol_adv = base + (0.0 if precision == 0 else 1e-13) * np.minimum(ratio, 1e18)
    _compare(dti, odti, tol_adv)
    if precision == 0:
        assert np.array_equal(np.isinf(dti), np.isinf(odti))
    assert abs(dt / odt - 1.0) < (1e-12 if precision == 0 else 1e-4)
    assert dt == dti.min()
    # each limit alone
    for one in (dict(f_orb=0.05), dict(dx_H=0.1, c_adv=0.5), dict(dx_H=0.1, c_diff=0.5)):
        r1 = dict(dt_max=1e30, **one)
        d1, t1 = sess.timestep(**r1, want=True)
        o1, ot1 = _oracle_dt(oracle, insts, r1, velocities)
        t1 = t1.cpu().numpy()
        _compare(t1, ot1, tol_adv if "c_adv" in one else base)
        if precision == 0:
            assert np.array_equal(np.isfinite(t1), np.isfinite(ot1))
            assert d1 == o1 or abs(d1 / o1 - 1.0) < 1e-12
    # the timestep drives a split step
    assert sess.step(min(dt, 1e6)) >= 1
    assert sess.stats()["status"] == 0
    sess.close()


def test_timestep_bounds_and_errors(gd, oracle):
    insts = _mixed_context()
    sess = gd.Session(insts, precision=1, velocities=True)
    dt = sess.timestep(1e30, **RULE)
    assert sess.timestep(0.5 * dt, **RULE) == 0.5 * dt
    assert sess.timestep(1e30, dt_out=0.25 * dt, **RULE) == 0.25 * dt
    assert sess.timestep(2.0 * dt, **RULE) == dt
    assert sess.timestep(123.0) == 123.0                  # every limit off
    for bad in (dict(dt_max=0.0), dict(dt_max=-1.0), dict(dt_max=math.nan), dict(dt_max=1.0, dt_out=0.0),
                dict(dt_max=1.0, c_diff=0.5), dict(dt_max=1.0, dx_H=math.inf, c_adv=0.5),
                dict(dt_max=1.0, f_orb=math.nan)):
        with pytest.raises(gd.GDError) as e:
            sess.timestep(**bad)
        assert e.value.code == gd.GD_ERR_ARG
    # a disk particle at R = 0 has no finite limit
    import torch
    sess.t["x"][0] = 0.0
    sess.t["y"][0] = 0.0
    torch.cuda.synchronize()
    with pytest.raises(gd.GDError) as e:
        sess.timestep(1e30, f_orb=0.05)
    assert e.value.code == gd.GD_ERR_NONFINITE
    sess.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_timestep_full_size(gd, oracle, precision):
    ins = W.disk_instance(1 << 22, seed=1, K=32, sizes=("lognormal", 10.0, 1.0), velocities=True)
    sess = gd.Session([ins], precision=precision, velocities=True)
    rule = dict(dt_max=1e30, **RULE)
    dt, dti = sess.timestep(**rule, want=True)
    dti = dti.cpu().numpy()
    sess.close()
    assert dt == dti.min()
    q = np.arange(0, len(dti), 4099)
    q = np.append(q, int(np.argmin(dti)))
    P = oracle.params(ins["params"])
    r = oracle.dt_rule(**rule)
    ratio = _speed_ratio([ins], True)
    for i in q:
        o = oracle.local_dt(P, r, ins["x"][i], ins["y"][i], ins["z"][i], ins["s"][i],
                            (ins["vr"][i], ins["lth"][i], ins["lph"][i]))
        tol = 1e-12 if precision == 0 else 2e-5 + 1e-13 * min(ratio[i], 1e18)
        assert abs(dti[i] / o - 1.0) < tol, (i, dti[i], o)

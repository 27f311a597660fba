"""GPU common transport timestep (Sect. 2.6) against the oracle.

* Every particle's local limit dt_i within 1e-12 relative (both sides FP64; they differ
  only in the last bits of pow, exp and sqrt), +infinity at the same particles, and the
  global dt within 1e-12 of the oracle's minimum over the instances, for a disk with
  velocities, local patches and the ring model in one context, in both precision forms.
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
    ring["lph"] = np.sqrt(6.674e-8 * W.MSUN * np.hypot(ring["x"], ring["y"]))
    return [disk, p1, p2, ring]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("velocities", [False, True])
def test_timestep_parity(gd, oracle, precision, velocities):
    insts = _mixed_context()
    sess = gd.Session(insts, precision=precision, velocities=velocities)
    rule = dict(dt_max=1e30, **RULE)
    dt, dti = sess.timestep(**rule, want=True)
    dti = dti.cpu().numpy()
    odt, odti = _oracle_dt(oracle, insts, rule, velocities)
    inf = np.isinf(odti)
    assert np.array_equal(np.isinf(dti), inf)
    assert np.abs(dti[~inf] / odti[~inf] - 1.0).max() < 1e-12
    assert abs(dt / odt - 1.0) < 1e-12
    assert dt == dti.min()
    # each limit alone
    for one in (dict(f_orb=0.05), dict(dx_H=0.1, c_adv=0.5), dict(dx_H=0.1, c_diff=0.5)):
        r1 = dict(dt_max=1e30, **one)
        d1, t1 = sess.timestep(**r1, want=True)
        o1, ot1 = _oracle_dt(oracle, insts, r1, velocities)
        t1 = t1.cpu().numpy()
        fin = np.isfinite(ot1)
        assert np.array_equal(np.isfinite(t1), fin)
        if fin.any():
            assert np.abs(t1[fin] / ot1[fin] - 1.0).max() < 1e-12
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


def test_timestep_full_size(gd, oracle):
    ins = W.disk_instance(1 << 22, seed=1, K=32, sizes=("lognormal", 10.0, 1.0), velocities=True)
    sess = gd.Session([ins], precision=1, velocities=True)
    rule = dict(dt_max=1e30, **RULE)
    dt, dti = sess.timestep(**rule, want=True)
    dti = dti.cpu().numpy()
    sess.close()
    assert dt == dti.min()
    q = np.arange(0, len(dti), 4099)
    q = np.append(q, int(np.argmin(dti)))
    P = oracle.params(ins["params"])
    r = oracle.dt_rule(**rule)
    for i in q:
        o = oracle.local_dt(P, r, ins["x"][i], ins["y"][i], ins["z"][i], ins["s"][i],
                            (ins["vr"][i], ins["lth"][i], ins["lph"][i]))
        assert abs(dti[i] / o - 1.0) < 1e-12, (i, dti[i], o)

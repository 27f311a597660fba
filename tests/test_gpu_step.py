"""Bounded collision steps and the symmetric split timestep (Sect. 2.5.3, 2.6) against
the oracle driven the same way.

The oracle runs frozen-neighbour intervals with dt_coll = tau until the exact tick
count of the step is used up (its controller restarts the count there); diffusion
and the push use the oracle's own step functions.  Per instance:
* gd_collide: the same number of intervals, the same diameters (FP64 form: 1e-12
  where no near tie was flagged), whatever the other instances of the context do
  (an instance that finishes first idles);
* gd_step: C(dt/2) D(dt/2) T(dt) D(dt/2) C(dt/2), positions, velocities and diameters
  after two steps, the second reusing the lists of the first one's last C.
"""
import math

import numpy as np
import pytest

from paper_2609_35967_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _oracle_collide(oracle, params, st, tau, x, y, z, s, M):
    P = oracle.params(dict(params, dt_coll=tau))
    st.remain_ticks = 1 << 60
    st.dt_remain = tau
    n, near = 0, 0
    while True:
        oracle.interval_step(P, st, x, y, z, s, M, want=())
        n += 1
        near += st.near_draw + st.near_dt + st.near_audit
        if st.remain_ticks == 1 << 60:
            return n, near


def test_collide_matches_oracle_per_instance(gd, oracle):
    # three patches with very different collision rates in one context
    insts = [W.patch_instance(n, r_au=r, alpha=a, v_frag=v, seed=70 + b)
             for b, (n, r, a, v) in enumerate(((1500, 8.0, 1e-2, 500.0), (900, 20.0, 1e-4, 100.0),
                                               (2200, 12.0, 3e-3, 150.0)))]
    sess = gd.Session(insts, precision=gd.GD_FP64)
    om = math.sqrt(6.674e-8 * W.MSUN / (10 * W.AU) ** 3)
    tau = 2.0 * math.pi / om
    n_gpu = sess.collide(tau)
    st_all = sess.stats()
    s_gpu = sess.t["s"].cpu().numpy()
    off = W.concat(insts)["offsets"]
    n_max = 0
    for b, ins in enumerate(insts):
        P0 = oracle.params(ins["params"])
        st = oracle.new_state(P0)
        s = ins["s"].copy()
        n, near = _oracle_collide(oracle, ins["params"], st, tau, ins["x"], ins["y"], ins["z"], s, ins["M"])
        n_max = max(n_max, n)
        inst = st_all["instances"][b]
        if near + inst["near_draw"] + inst["near_dt"] + inst["near_audit"] == 0:
            assert np.abs(s_gpu[off[b]:off[b + 1]] / s - 1.0).max() < 1e-12, b
            assert inst["C"] == st.C
    # the context ran until its slowest instance was done
    assert n_gpu == n_max
    assert st_all["status"] == 0
    # afterwards the instances are back to open-ended collision steps
    sess.build_neighbors()
    sess.collision_rates()
    sess.sample_collisions()
    assert all(i["dt_exe"] > 0.0 for i in sess.stats()["instances"])
    sess.close()


def test_collide_reuses_lists(gd):
    ins = W.patch_instance(3000, seed=75, alpha=1e-2)
    sess = gd.Session([ins], precision=gd.GD_MIXED, flags=gd.GD_FLAG_TIMING)
    om = math.sqrt(6.674e-8 * W.MSUN / ins["params"]["r0"] ** 3)
    n1 = sess.collide(0.5 / om)
    k1 = sess.stats()["kernel_calls"]["knn"]
    n2 = sess.collide(0.5 / om, reuse_lists=True)
    k2 = sess.stats()["kernel_calls"]["knn"]
    assert n1 >= 1 and n2 >= 1
    assert k1 == 1 and k2 == 1          # one build, kept for the second step
    sess.close()


def test_split_step_matches_oracle(gd, oracle):
    ins = W.disk_instance(3000, seed=76, sizes=("lognormal", 10.0, 1.0), velocities=True, alpha=1e-2)
    ins["params"] = dict(ins["params"], diff_chi=1)
    sess = gd.Session([ins], precision=gd.GD_FP64, velocities=True)
    P = oracle.params(ins["params"])
    st = oracle.new_state(P)
    x, y, z, s = (ins[k].copy() for k in ("x", "y", "z", "s"))
    vr, lth, lph = (ins[k].copy() for k in ("vr", "lth", "lph"))
    om5 = math.sqrt(6.674e-8 * W.MSUN / (5 * W.AU) ** 3)
    dt = 0.2 / om5
    near = 0
    n_or = 0
    for k in range(2):
        n, nr = _oracle_collide(oracle, ins["params"], st, 0.5 * dt, x, y, z, s, ins["M"])
        n_or += n
        near += nr
        oracle.diffuse(P, 0.5 * dt, 2 * k, x, y, z, s, vr, lth, lph)
        oracle.push(P, x, y, z, vr, lth, lph, s, dt)
        oracle.diffuse(P, 0.5 * dt, 2 * k + 1, x, y, z, s, vr, lth, lph)
        n, nr = _oracle_collide(oracle, ins["params"], st, 0.5 * dt, x, y, z, s, ins["M"])
        n_or += n
        near += nr
    n_gpu = sess.step(dt) + sess.step(dt, reuse_lists=True)
    stg = sess.stats()
    got = {k: sess.t[k].cpu().numpy() for k in sess.t}
    sess.close()
    assert stg["status"] == 0
    assert n_gpu == n_or
    R = np.sqrt(x * x + y * y).max()
    if near + stg["near_draw"] + stg["near_dt"] + stg["near_audit"] == 0:
        assert np.abs(got["s"] / s - 1.0).max() < 1e-12
        # positions through two pushes and four diffusion steps
        for a, kk in ((x, "x"), (y, "y"), (z, "z")):
            assert np.abs(got[kk] - a).max() < 1e-10 * R
        for a, kk in ((vr, "vr"), (lth, "lth"), (lph, "lph")):
            assert np.abs(got[kk] - a).max() < 1e-9 * np.abs(a).max()

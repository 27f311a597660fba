"""GPU dust diffusion (Sect. 2.4) against the oracle and the ring test of Sect. 3.2.

* Parity: the same Philox draws give the same displacements; positions (and the
  recomputed velocity components) agree to 1e-12 of the radius (1e-10 relative for the
  velocities): the two sides differ only in the last bits of log, sin, cos and atan2.
* Ring test at the paper's 2^20 particles through the CUDA path: the mean and variance of
  ln(R/R_0) at t~ = 0.1 against the analytic values, for both prescriptions.
* The neighbour search after a diffusion step (particles moved away from the radius of
  their previous distance) still gives the oracle's lists.
"""
import math

import numpy as np
import pytest

from paper_2609_35967_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _steps_both(gd, oracle, ins, precision, velocities, n_steps, dt):
    sess = gd.Session([ins], precision=precision, velocities=velocities)
    P = oracle.params(ins["params"])
    x, y, z = ins["x"].copy(), ins["y"].copy(), ins["z"].copy()
    v = [ins[k].copy() for k in ("vr", "lth", "lph")] if velocities else [None, None, None]
    for k in range(n_steps):
        oracle.diffuse(P, dt, k, x, y, z, ins["s"], *v)
        sess.diffuse(dt)
    st = sess.stats()
    got = {k: sess.t[k].cpu().numpy() for k in sess.t}
    sess.close()
    return st, (x, y, z), v, got


@pytest.mark.parametrize("chi", [0, 1])
def test_disk_diffusion_parity(gd, oracle, chi):
    ins = W.disk_instance(5000, seed=12, sizes=("lognormal", 10.0, 1.0), velocities=True)
    ins["params"] = dict(ins["params"], diff_chi=chi, Sc_Z=2.0)
    om5 = math.sqrt(6.674e-8 * W.MSUN / (5 * W.AU) ** 3)
    st, (x, y, z), v, got = _steps_both(gd, oracle, ins, 0, True, 3, 20.0 / om5)
    assert st["status"] == 0
    R = np.sqrt(x * x + y * y)
    for a, g in ((x, got["x"]), (y, got["y"]), (z, got["z"])):
        assert np.abs(g - a).max() < 1e-12 * R.max()
    # the particles did move (by far more than the tolerance)
    assert np.abs(got["z"] - ins["z"]).max() > 1e-6 * R.max()
    for a, k in zip(v, ("vr", "lth", "lph")):
        scale = np.abs(a).max()
        assert np.abs(got[k] - a).max() < 1e-10 * scale


def test_patch_diffusion_parity(gd, oracle):
    ins = W.patch_instance(4000, seed=13, alpha=1e-2)
    om = math.sqrt(6.674e-8 * W.MSUN / ins["params"]["r0"] ** 3)
    st, (x, y, z), _, got = _steps_both(gd, oracle, ins, 0, False, 4, 5.0 / om)
    L = ins["params"]["box_x"]
    for a, g in ((x, got["x"]), (y, got["y"]), (z, got["z"])):
        assert np.abs(g - a).max() < 1e-12 * L
    assert (np.abs(got["x"]) <= 0.5 * L).all() and (np.abs(got["y"]) <= 0.5 * L).all()


@pytest.mark.parametrize("chi", [0, 1])
def test_ring_parity_and_solution(gd, oracle, chi):
    # parity on a small ring
    ins = W.ring_instance(3000, chi=chi, seed=14)
    _, (x, y, z), _, got = _steps_both(gd, oracle, ins, 0, False, 5, 100.0)
    for a, g in ((x, got["x"]), (y, got["y"])):
        assert np.abs(g - a).max() < 1e-12
    # the ring test at 2^20 particles to t~ = 0.1 in 100 steps
    big = W.ring_instance(1 << 20, chi=chi, seed=15)
    sess = gd.Session([big], precision=1, flags=gd.GD_FLAG_TIMING)
    P = big["params"]
    t0 = P["r0"] ** 2 / P["D0"]
    for _ in range(100):
        sess.diffuse(0.1 * t0 / 100)
    st = sess.stats()
    xs, ys = sess.t["x"].cpu().numpy(), sess.t["y"].cpu().numpy()
    sess.close()
    lnR = np.log(np.sqrt(xs * xs + ys * ys) / P["r0"])
    n = len(lnR)
    mu, var = (2.0 + chi * P["p"]) * 0.1, 0.2025
    assert abs(lnR.mean() - mu) < 4 * math.sqrt(var / n) + 1e-3, lnR.mean()
    assert abs(lnR.var() - var) < 4 * var * math.sqrt(2.0 / n) + 1e-3, lnR.var()
    assert st["kernel_calls"]["diffuse"] == 100


def test_neighbours_after_diffusion(gd, oracle):
    ins = W.disk_instance(1 << 14, seed=16, sizes=("lognormal", 10.0, 1.0))
    om5 = math.sqrt(6.674e-8 * W.MSUN / (5 * W.AU) ** 3)
    sess = gd.Session([ins], precision=1)
    sess.build_neighbors()
    sess.collision_rates()
    sess.sample_collisions()
    for _ in range(3):
        sess.diffuse(200.0 / om5)
    nbr, d = sess.build_neighbors(want=True)
    x, y, z = (sess.t[k].cpu().numpy() for k in ("x", "y", "z"))
    assert np.abs(z - ins["z"]).max() > 0.0
    P = oracle.params(ins["params"])
    q = np.arange(0, len(x), 37)
    onbr, od = oracle.knn(P, x, y, z, q)
    assert np.array_equal(nbr.cpu().numpy()[q], onbr)
    assert np.array_equal(d.cpu().numpy()[q], od)
    sess.close()


@pytest.mark.parametrize("geometry", ["disk", "patch", "disk_v"])
def test_mixed_diffusion_close_to_oracle(gd, oracle, geometry):
    """Mixed form: FP32 draws (the FP64 form's uniforms rounded to FP32) and FP32
    coefficients, the step applied to the FP64 positions.  The displacements agree with the
    FP64 oracle's to 1e-4 of their size.  With velocities (disk_v) the FP64 basis change
    from direction cosines gives the oracle's components to 1e-6 of their scale (the two
    sides re-project at positions that differ by the displacement error)."""
    vel = geometry == "disk_v"
    if geometry.startswith("disk"):
        ins = W.disk_instance(5000, seed=17, sizes=("lognormal", 10.0, 1.0), velocities=vel)
        om = math.sqrt(6.674e-8 * W.MSUN / (5 * W.AU) ** 3)
    else:
        ins = W.patch_instance(4000, seed=18, alpha=1e-2)
        om = math.sqrt(6.674e-8 * W.MSUN / ins["params"]["r0"] ** 3)
    st, (x, y, z), v, got = _steps_both(gd, oracle, ins, 1, vel, 1, 20.0 / om)
    if vel:
        # scales: the speed for v_r, r times it for l_theta, R times it for l_phi (the
        # components start at the gas motion, so v_r and l_theta are small themselves)
        Rn = np.hypot(x, y)
        speed = np.abs(v[2] / Rn)
        for a, k, sc in zip(v, ("vr", "lth", "lph"), (speed, speed * np.hypot(Rn, z), speed * Rn)):
            err = np.abs(got[k] - a).max() / sc.max()
            assert err < 1e-6, (k, err)
    L = ins["params"]["box_x"] if geometry == "patch" else 0.0

    def diff(a, b):
        # minimum image across the patch's periodic edges
        return a - b - (L * np.round((a - b) / L) if L > 0.0 else 0.0)

    d = np.sqrt(diff(x, ins["x"]) ** 2 + diff(y, ins["y"]) ** 2 + (z - ins["z"]) ** 2)
    err = np.sqrt(diff(got["x"], x) ** 2 + diff(got["y"], y) ** 2 + (got["z"] - z) ** 2)
    assert np.median(d) > 0.0
    assert (err <= 1e-4 * np.median(d) + 1e-4 * d).all(), (err / np.median(d)).max()

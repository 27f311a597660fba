"""GPU parity of the radiation forces and the optical depth grid (Sect. 2.3.2) against the
oracle.

- gd_optical_depth: the face grid and tau at every particle, both forms, 3D and vertically
  integrated grids, against the oracle's tau_grid / tau_at within 1e-12 (the GPU's cell sums
  are exact 128-bit fixed point, the oracle's sequential FP64); particles inside, beyond
  and above the grid; the sums do not depend on scheduling (two runs, bit for bit).
- The FP64 push with radiation pressure, P-R drag, tau and the taper against the oracle's
  push_rad over five steps (positions within 1e-12 of their scale, velocities 1e-10), the
  taper clock in the instance stats.
- The mixed push against the oracle at the plain mixed push's bars, on particles whose
  first-drift midpoints lie at least 1e-3 cells from every cell edge (so both deposit
  into the same cells).
- A batched context: a 3D-grid disk with radiation, a plain disk and a 2D-grid disk with
  P-R drag, each against its own oracle step; the grid output holds only the gridded
  instances, in order.
- The graph-captured interval loop with a radiation push equals the same calls one by one.
"""
import math

import numpy as np
import pytest

from paper_2609_35967_gb300 import workloads as W

pytestmark = pytest.mark.gpu

AU = W.AU


def rad_disk(n, seed, geom=0, beta0=0.05, pr=1, t_beta=0.0, nr=24, nmu=8, nphi=16, tau_max=3.0,
             oracle=None):
    """A global disk with velocities, log-normal sizes and a grid from 8 to 80 au and
    |z/r| < 0.1 (the disk spans 5-100 au and its small grains follow the gas scale height,
    so particles lie inside, beyond and above the grid); kappa0 puts the largest face of
    the grid near tau_max."""
    ins = W.disk_instance(n, seed=seed, K=16, velocities=True, sizes=("lognormal", 1.0, 0.7))
    rng = np.random.default_rng(seed + 100)
    R0 = np.hypot(ins["x"], ins["y"])
    ins["vr"] = rng.normal(0.0, 3e3, n)
    ins["lth"] = rng.normal(0.0, 3e3, n) * R0
    p = dict(ins["params"], beta0=beta0, kappa0=1.0, rad_s0=2e-4, t_beta=t_beta, rad_pr=pr,
             tau_geom=geom, tau_nr=nr, tau_nmu=nmu, tau_nphi=nphi, tau_rmin=8 * AU, tau_rmax=80 * AU,
             tau_mu=0.1)
    if oracle is not None:
        T = oracle.tau_grid(oracle.params(p), ins["x"], ins["y"], ins["z"], ins["s"], ins["M"])
        p["kappa0"] = tau_max / T.max()
    ins["params"] = p
    return ins


def _faces(p):
    nm = 1 if p["tau_geom"] == 1 else p["tau_nmu"]
    return nm * p["tau_nphi"] * (p["tau_nr"] + 1)


@pytest.mark.parametrize("geom", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_optical_depth_matches_oracle(gd, oracle, geom, precision):
    ins = rad_disk(20000, seed=41 + geom, geom=geom, oracle=oracle)
    P = oracle.params(ins["params"])
    T = oracle.tau_grid(P, ins["x"], ins["y"], ins["z"], ins["s"], ins["M"])
    sess = gd.Session([ins], precision=precision, velocities=True)
    tau, grid = sess.optical_depth(want_grid=True)
    tau, grid = tau.cpu().numpy(), grid.cpu().numpy()
    assert grid.shape == T.shape
    assert np.abs(grid - T).max() <= 1e-12 * T.max()
    ref = np.array([oracle.tau_at(P, T, a, b, c) for a, b, c in zip(ins["x"], ins["y"], ins["z"])])
    assert np.abs(tau - ref).max() <= 1e-12 * T.max()
    # the workload spans every case: inside the grid, inside r_min (tau = 0), beyond r_max
    rad = np.hypot(ins["x"], ins["y"]) if geom else np.sqrt(ins["x"] ** 2 + ins["y"] ** 2 + ins["z"] ** 2)
    assert (rad < 8 * AU).any() and (rad > 80 * AU).any()
    assert np.all(tau[rad < 8 * AU] == 0.0) and (tau > 0.5).sum() > 1000
    if geom == 0:
        assert (np.abs(ins["z"] / rad) > 0.1).any()
    # exact cell sums: a second call gives the same bits
    tau2, grid2 = sess.optical_depth(want_grid=True)
    assert np.array_equal(grid2.cpu().numpy(), grid) and np.array_equal(tau2.cpu().numpy(), tau)
    sess.close()


def _state(ins):
    return [ins[k].copy() for k in ("x", "y", "z", "vr", "lth", "lph")]


def _compare64(got, ref, what):
    x, y, z, vr, lth, lph = ref
    for k, r in (("x", x), ("y", y), ("z", z), ("lph", lph)):
        assert np.abs(got[k] - r).max() <= 1e-12 * np.abs(r).max(), (what, k)
    for k, r in (("vr", vr), ("lth", lth)):
        assert np.abs(got[k] - r).max() <= 1e-10 * np.abs(r).max(), (what, k)


def test_push_rad_fp64_matches_oracle(gd, oracle):
    dt = 3.0e7
    ins = rad_disk(8000, seed=43, beta0=0.05, pr=1, t_beta=8 * dt, oracle=oracle)
    ins["params"]["t_start"] = 2 * dt
    P = oracle.params(ins["params"])
    sess = gd.Session([ins], precision=gd.GD_FP64, velocities=True)
    ref = _state(ins)
    for k in range(5):
        sess.push_staggered(dt)
        sess.stats()
        oracle.push_rad(P, *ref, ins["s"], ins["M"], dt, (2 + k) * dt)
        got = {key: sess.t[key].cpu().numpy() for key in ("x", "y", "z", "vr", "lth", "lph")}
        _compare64(got, ref, k)
    st = sess.stats()
    assert st["instances"][0]["t_rad"] == pytest.approx(7 * dt, rel=1e-15)
    # the radiation forces acted: the same steps without them end elsewhere
    plain = _state(ins)
    for k in range(5):
        oracle.push(P, *plain, ins["s"], dt, drag=True)
    assert np.abs(plain[3] - ref[3]).max() > 1e-3 * np.abs(ref[3]).max()
    sess.close()


def test_push_rad_mixed_close_to_oracle(gd, oracle):
    dt = 3.0e7
    ins = rad_disk(8000, seed=44, beta0=0.05, pr=1, oracle=oracle)
    P = oracle.params(ins["params"])
    # keep the particles whose first-drift midpoints lie at least 1e-3 cells from every edge
    st = _state(ins)
    _, mid = oracle.push_rad(P, *st, ins["s"], ins["M"], dt, 0.0)
    r, th, ph = mid
    p = ins["params"]
    u = (r - p["tau_rmin"]) / ((p["tau_rmax"] - p["tau_rmin"]) / p["tau_nr"])
    w = (np.cos(th) + p["tau_mu"]) / (2 * p["tau_mu"] / p["tau_nmu"])
    v = (np.arctan2(np.sin(ph), np.cos(ph)) + math.pi) / (2 * math.pi / p["tau_nphi"])
    far = lambda a: np.abs(a - np.round(a)) > 1e-3
    keep = far(u) & far(w) & far(v)
    assert keep.mean() > 0.98
    sub = {k: (ins[k][keep] if isinstance(ins[k], np.ndarray) else ins[k]) for k in ins}
    sess = gd.Session([sub], precision=gd.GD_MIXED, velocities=True)
    sess.push_staggered(dt)
    sess.stats()
    ref = _state(sub)
    oracle.push_rad(P, *ref, sub["s"], sub["M"], dt, 0.0)
    got = {k: sess.t[k].cpu().numpy() for k in ("x", "y", "z", "vr", "lth", "lph")}
    sess.close()
    x, y, z, vr, lth, lph = ref
    R = np.hypot(x, y)
    for k, rf in (("x", x), ("y", y), ("z", z)):
        assert np.abs(got[k] - rf).max() <= 1e-7 * R.max(), k
    speed = np.abs(lph / R)
    for k, rf, sc in (("vr", vr, speed), ("lth", lth, speed * np.hypot(R, z)), ("lph", lph, speed * R)):
        err = (np.abs(got[k] - rf) / sc).max()
        assert err < 1e-6, (k, err)


def test_batched_radiation_and_plain(gd, oracle):
    dt = 2.0e7
    a = rad_disk(6000, seed=45, geom=0, beta0=0.05, pr=0, oracle=oracle)
    b = W.disk_instance(3000, seed=46, K=16, velocities=True, sizes=("lognormal", 1.0, 0.7))
    c = rad_disk(5000, seed=47, geom=1, beta0=0.08, pr=1, nr=17, nphi=11, oracle=oracle)
    insts = [a, b, c]
    offs = W.concat(insts)["offsets"]
    sess = gd.Session(insts, K=16, precision=gd.GD_FP64, velocities=True)
    tau, grid = sess.optical_depth(want_grid=True)
    grid = grid.cpu().numpy()
    Ta = oracle.tau_grid(oracle.params(a["params"]), a["x"], a["y"], a["z"], a["s"], a["M"])
    Tc = oracle.tau_grid(oracle.params(c["params"]), c["x"], c["y"], c["z"], c["s"], c["M"])
    assert grid.size == Ta.size + Tc.size == _faces(a["params"]) + _faces(c["params"])
    assert np.abs(grid[:Ta.size] - Ta).max() <= 1e-12 * Ta.max()
    assert np.abs(grid[Ta.size:] - Tc).max() <= 1e-12 * Tc.max()
    assert np.all(tau.cpu().numpy()[offs[1]:offs[2]] == 0.0)
    refs = [_state(i) for i in insts]
    for k in range(3):
        sess.push_staggered(dt)
        sess.stats()
        oracle.push_rad(oracle.params(a["params"]), *refs[0], a["s"], a["M"], dt, k * dt)
        oracle.push(oracle.params(b["params"]), *refs[1], b["s"], dt, drag=True)
        oracle.push_rad(oracle.params(c["params"]), *refs[2], c["s"], c["M"], dt, k * dt)
        for j, ref in enumerate(refs):
            lo, hi = offs[j], offs[j + 1]
            got = {key: sess.t[key].cpu().numpy()[lo:hi] for key in ("x", "y", "z", "vr", "lth", "lph")}
            _compare64(got, ref, (k, j))
    sess.close()


def test_graph_loop_with_radiation_push(gd):
    """gd_run_intervals with a radiation push (captured once, replayed) ends where the same
    calls made one by one end, bit for bit."""
    ins = rad_disk(6000, seed=48, beta0=0.05, pr=1, t_beta=1e9)
    ins["params"]["kappa0"] = 1e-12
    outs = []
    for graph in (True, False):
        sess = gd.Session([ins], precision=gd.GD_MIXED, velocities=True)
        if graph:
            sess.run_intervals(3, push=True)
        else:
            for _ in range(3):
                sess.build_neighbors()
                sess.collision_rates()
                sess.sample_collisions()
                sess.push_staggered(-1.0)
        st = sess.stats()
        assert st["status"] == 0
        outs.append(({k: sess.t[k].cpu().numpy() for k in ("x", "y", "z", "vr", "lth", "lph", "s")},
                     st["instances"][0]["t_rad"]))
        sess.close()
    for k in outs[0][0]:
        assert np.array_equal(outs[0][0][k], outs[1][0][k]), k
    assert outs[0][1] == outs[1][1] > 0.0

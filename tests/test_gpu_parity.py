"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same
seeded inputs.

Bars (from the method's precision split):
* neighbour lists and neighbour distances: bit-exact (both forms);
* FP64 rates: every channel rate lambda*_ij within 1e-12 relative of the oracle's (a zero
  channel exactly zero), and lambda*_i; the controller-bin moments A_b, B_b within 1e-12;
* event sequences: identical per particle (count and channel hash) except where a
  near tie (a draw within 1e-10 of a boundary) was flagged on either side;
* diameters after sampling: within 1e-12 relative (FP64) where the sequences agree;
* represented mass: never written (bitwise), sum N m = sum M within 1e-12;
* mixed form: lists bit-exact; lambda*_i and every channel rate within 1e-4 relative (the
  largest pair-rate error the mixed form accepts without FP64); A_b, B_b within 2e-4; event
  sequences identical to the FP64 ones except flagged near ties -- every FP32 decision is
  certified against its error bound and the particles it cannot certify are replayed in
  FP64 -- so the same bar as the FP64 form applies, with diameters within 1e-12.
"""
import math

import numpy as np
import pytest

from paper_2609_35967_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _step_both(gd, oracle, sess, P, st, ins, s_or):
    ref = oracle.interval_step(P, st, ins["x"], ins["y"], ins["z"], s_or, ins["M"],
                               want=("nbr", "d", "V", "lam", "chan", "ev_count", "ev_hash", "near",
                                     "A_b", "B_b"))
    nbr, d = sess.build_neighbors(want=True)
    lam, chan = sess.collision_rates(want=True, chan=True)
    A_b, B_b = sess.controller_bins(0)
    ec, eh, nn = sess.sample_collisions(want=True)
    return ref, dict(nbr=nbr.cpu().numpy(), d=d.cpu().numpy(), lam=lam.cpu().numpy(),
                     chan=chan.cpu().numpy(), A_b=np.array(A_b), B_b=np.array(B_b),
                     ev_count=ec.cpu().numpy(), ev_hash=eh.cpu().numpy().view(np.uint32),
                     near=nn.cpu().numpy())


def _check_channels(ref, got, tol):
    """Every channel rate lambda*_ij of every slot against the oracle's: zeros exactly zero,
    the rest within tol relative."""
    rc, gc = ref["chan"], got["chan"]
    assert np.array_equal(rc == 0.0, gc == 0.0), "a zero channel differs"
    nz = rc != 0.0
    rel = np.abs(gc[nz] / rc[nz] - 1.0)
    assert rel.max() < tol, rel.max()
    return rel.max()


def _check_bins(ref, got, st, tol):
    """Controller-bin moments A_b, B_b of the interval choice against the oracle's."""
    n = st.n_groups
    assert len(got["A_b"]) == n
    for k in ("A_b", "B_b"):
        r, g = ref[k][:n], got[k]
        assert np.array_equal(r == 0.0, g == 0.0), k
        nz = r != 0.0
        if nz.any():
            assert np.abs(g[nz] / r[nz] - 1.0).max() < tol, (k, np.abs(g[nz] / r[nz] - 1.0).max())


def _compare_events(ref, got, allow_frac=1e-3):
    same = (ref["ev_count"] == got["ev_count"]) & (ref["ev_hash"] == got["ev_hash"])
    flagged = (ref["near"] > 0) | (got["near"] > 0)
    bad = ~same & ~flagged
    assert bad.sum() == 0, f"{bad.sum()} particles differ without a near tie"
    return same


@pytest.mark.parametrize("precision", [0, 1])
def test_patch_interval_parity(gd, oracle, precision):
    ins = W.patch_instance(2048, K=32, seed=5)
    sess = gd.Session([ins], precision=precision)
    P = oracle.params(ins["params"])
    st = oracle.new_state(P)
    s_or = ins["s"].copy()
    for it in range(3):
        ref, got = _step_both(gd, oracle, sess, P, st, ins, s_or)
        assert np.array_equal(got["nbr"], ref["nbr"])
        assert np.array_equal(got["d"], ref["d"])
        rel = np.abs(got["lam"] / ref["lam"] - 1.0)
        if precision == 0:
            assert rel.max() < 1e-12
            _check_channels(ref, got, 1e-12)
            _check_bins(ref, got, st, 1e-12)
        else:
            assert rel.max() < 1e-4, rel.max()
            _check_channels(ref, got, 1e-4)
            _check_bins(ref, got, st, 2e-4)
        stats = sess.stats()
        inst = stats["instances"][0]
        s_gpu = sess.t["s"].cpu().numpy()
        if inst["dt_exe"] != st.dt_exe:
            # only a flagged near tie of the interval or audit rule may change the interval
            assert inst["near_dt"] + inst["near_audit"] + st.near_dt + st.near_audit > 0
        else:
            same = _compare_events(ref, got)
            assert np.abs(s_gpu[same] / s_or[same] - 1.0).max() < 1e-12
        # keep both sides on the same state for the next interval
        import torch
        sess.t["s"].copy_(torch.as_tensor(s_or, device=sess.device))
        torch.cuda.synchronize()
    assert stats["status"] == 0
    sess.close()


def test_patch_hundred_intervals(gd, oracle):
    """Configuration 0 shape (4096 particles, K = 32, seed 1): 100 intervals, FP64.  Every
    interval: each particle's event count and channel sequence equal the oracle's unless a
    near tie was flagged for it, the interval and C are the same, and the flagged near ties
    stay below 1e-6 of the events.  After a flagged tie both sides continue from the
    oracle's sizes, so later intervals are compared from the same state."""
    import torch
    ins = W.config0(n=4096)[0]
    sess = gd.Session([ins], precision=gd.GD_FP64)
    P = oracle.params(ins["params"])
    st = oracle.new_state(P)
    s_or = ins["s"].copy()
    n_int = 100
    events = near_total = 0
    for _ in range(n_int):
        ref = oracle.interval_step(P, st, ins["x"], ins["y"], ins["z"], s_or, ins["M"],
                                   want=("ev_count", "ev_hash", "near"))
        sess.build_neighbors()
        sess.collision_rates()
        ec, eh, nn = sess.sample_collisions(want=True)
        got = dict(ev_count=ec.cpu().numpy(), ev_hash=eh.cpu().numpy().view(np.uint32), near=nn.cpu().numpy())
        inst = sess.stats()["instances"][0]
        assert inst["dt_exe"] == st.dt_exe or inst["near_dt"] + st.near_dt > 0
        same = _compare_events(ref, got)
        events += int(ref["ev_count"].sum())
        flagged = int(((ref["near"] > 0) | (got["near"] > 0)).sum())
        near_total += flagged
        s_gpu = sess.t["s"].cpu().numpy()
        assert np.abs(s_gpu[same] / s_or[same] - 1.0).max() < 1e-12
        if flagged or inst["near_dt"] + inst["near_audit"] > 0:
            sess.t["s"].copy_(torch.as_tensor(s_or, device=sess.device))
            torch.cuda.synchronize()
    stats = sess.stats()
    assert stats["intervals"] == n_int
    assert stats["status"] == 0
    assert events > 0
    assert near_total <= 1e-6 * events, (near_total, events)
    inst = stats["instances"][0]
    assert inst["C"] == st.C
    # the size spectrum of gd_stats: M summed per fine log-size bin of the current diameters,
    # against the same sums formed here with the oracle's bins, and against the oracle's run
    s_gpu = sess.t["s"].cpu().numpy()
    bins = np.array([oracle.fine_bin(v) for v in s_gpu])
    want = np.bincount(bins, weights=ins["M"], minlength=96)
    got = np.array(inst["spectrum"])
    assert np.array_equal(got == 0.0, want == 0.0)
    nz = want > 0
    assert np.abs(got[nz] / want[nz] - 1.0).max() < 1e-13
    assert got.sum() == pytest.approx(ins["M"].sum(), rel=1e-14)
    bins_or = np.array([oracle.fine_bin(v) for v in s_or])
    assert np.array_equal(np.bincount(bins_or, weights=ins["M"], minlength=96) > 0, got > 0)
    # represented mass is never written; sum N m = sum M
    assert np.array_equal(sess.t["M"].cpu().numpy(), ins["M"])
    m = math.pi * P.rho_s * s_gpu ** 3 / 6.0
    assert abs((ins["M"] / m * m).sum() - ins["M"].sum()) <= 1e-12 * ins["M"].sum()
    assert inst["sum_M"] == pytest.approx(ins["M"].sum(), rel=1e-14)
    sess.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_runs_are_bitwise_reproducible(gd, precision):
    """No float atomics on a parity-checked quantity: two contexts over the same inputs give
    bit-identical intervals, safety factors, bin moments and diameters."""
    ins = W.disk_instance(1 << 15, seed=23, K=32, sizes=("lognormal", 10.0, 1.0))
    out = []
    for _ in range(2):
        sess = gd.Session([ins], precision=precision)
        rec = []
        for _ in range(4):
            sess.build_neighbors()
            sess.collision_rates()
            rec.append(sess.controller_bins(0))
            sess.sample_collisions()
            inst = sess.stats()["instances"][0]
            rec.append((inst["dt_exe"], inst["C"], inst["events"]))
        rec.append(sess.t["s"].cpu().numpy().tobytes())
        out.append(rec)
        sess.close()
    assert out[0] == out[1]


def test_batched_patches(gd, oracle):
    """Several independent patches of uneven size and parameters in one context."""
    rng = np.random.default_rng(9)
    insts = []
    for b in range(6):
        n = int(rng.integers(200, 3000))
        insts.append(W.patch_instance(n, r_au=float(rng.uniform(5, 50)), alpha=10 ** rng.uniform(-4, -2),
                                      v_frag=float(rng.uniform(100, 1000)), seed=1000 + b, K=16))
    sess = gd.Session(insts, precision=gd.GD_FP64)
    Ps = [oracle.params(i["params"]) for i in insts]
    sts = [oracle.new_state(P) for P in Ps]
    s_or = [i["s"].copy() for i in insts]
    offs = W.concat(insts)["offsets"]
    for it in range(3):
        refs = [oracle.interval_step(P, st, i["x"], i["y"], i["z"], s, i["M"], want=("nbr", "lam"))
                for P, st, i, s in zip(Ps, sts, insts, s_or)]
        nbr, _ = sess.build_neighbors(want=True)
        lam, _ = sess.collision_rates(want=True)
        sess.sample_collisions()
        nbr = nbr.cpu().numpy()
        lam = lam.cpu().numpy()
        for b, ref in enumerate(refs):
            lo, hi = offs[b], offs[b + 1]
            assert np.array_equal(nbr[lo:hi] - lo, ref["nbr"])
            assert np.abs(lam[lo:hi] / ref["lam"] - 1.0).max() < 1e-12
    stats = sess.stats()
    s_gpu = sess.t["s"].cpu().numpy()
    for b in range(len(insts)):
        inst = stats["instances"][b]
        if inst["near_draw"] == 0 and sts[b].near_draw == 0:
            assert np.abs(s_gpu[offs[b]:offs[b + 1]] / s_or[b] - 1.0).max() < 1e-12
        assert inst["dt_exe"] == sts[b].dt_exe or inst["near_dt"] > 0
    sess.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_disk_sampled_queries(gd, oracle, precision):
    """Global disk (radial caps, flared density): lists and rates of sampled particles."""
    ins = W.disk_instance(1 << 15, seed=2, K=32, sizes=("lognormal", 10.0, 1.0))
    sess = gd.Session([ins], precision=precision)
    nbr, d = sess.build_neighbors(want=True)
    lam, _ = sess.collision_rates(want=True)
    sess.stats()
    P = oracle.params(ins["params"])
    q = np.random.default_rng(4).choice(len(ins["x"]), 300, replace=False)
    onbr, od = oracle.knn(P, ins["x"], ins["y"], ins["z"], q)
    assert np.array_equal(nbr.cpu().numpy()[q], onbr)
    assert np.array_equal(d.cpu().numpy()[q], od)
    r = oracle.rates_subset(P, ins["x"], ins["y"], ins["z"], ins["s"], ins["M"], q, onbr, od)
    rel = np.abs(lam.cpu().numpy()[q] / r["lam"] - 1.0)
    assert rel.max() < (1e-12 if precision == 0 else 1e-4), rel.max()
    sess.close()


def test_constant_kernel_mean_mass_gpu(gd):
    """Appendix A constant kernel on the GPU: mass-weighted mean mass = 1 + t (5 sigma)."""
    devs, ses = [], []
    for seed in (21, 22):
        ins = W.coag_instance(4096, K=16, mode=W.CONSTANT, seed=seed)
        sess = gd.Session([ins], precision=gd.GD_FP64)
        t = 0.0
        while t < 4.0 - 1e-12:
            sess.build_neighbors()
            sess.collision_rates()
            sess.sample_collisions()
            t += sess.stats()["instances"][0]["dt_exe"]
        s = sess.t["s"].cpu().numpy()
        m = math.pi * ins["params"]["rho_s"] * s ** 3 / 6.0
        devs.append(m.mean() - (1.0 + t))
        ses.append(m.std() / math.sqrt(len(m)))
        sess.close()
    se = math.sqrt(sum(x * x for x in ses)) / len(ses)
    assert abs(np.mean(devs)) < 5 * se


def test_graph_replay_matches_calls(gd):
    ins = W.patch_instance(3000, K=32, seed=8)
    a = gd.Session([ins], precision=gd.GD_MIXED)
    b = gd.Session([ins], precision=gd.GD_MIXED)
    for _ in range(4):
        a.build_neighbors()
        a.collision_rates()
        a.sample_collisions()
    b.run_intervals(4)
    sa, sb = a.stats(), b.stats()
    assert sa["intervals"] == sb["intervals"] == 4
    assert np.array_equal(a.t["s"].cpu().numpy(), b.t["s"].cpu().numpy())
    assert sa["events"] == sb["events"]
    a.close()
    b.close()


def test_mixed_push_close_to_oracle(gd, oracle):
    """Mixed form of the push: the drifts as rotations by FP32 angle increments applied to
    the FP64 position, the forces in FP64, the gas disk and the drag factor in FP32.  The
    positions agree with the oracle's to 1e-7 of the radius, the velocities to 1e-6 of the
    speed scale (v_r), r times it (l_theta) and R times it (l_phi)."""
    ins = W.disk_instance(4096, seed=6, K=32, velocities=True, sizes=("lognormal", 1.0, 0.5))
    rng = np.random.default_rng(3)
    R0 = np.hypot(ins["x"], ins["y"])
    ins["vr"] = rng.normal(0.0, 3e3, 4096)
    ins["lth"] = rng.normal(0.0, 3e3, 4096) * R0
    sess = gd.Session([ins], precision=gd.GD_MIXED, velocities=True)
    dt = 3.0e7
    sess.push_staggered(dt)
    sess.stats()
    P = oracle.params(ins["params"])
    x, y, z = ins["x"].copy(), ins["y"].copy(), ins["z"].copy()
    vr, lth, lph = ins["vr"].copy(), ins["lth"].copy(), ins["lph"].copy()
    oracle.push(P, x, y, z, vr, lth, lph, ins["s"], dt, drag=True)
    got = {k: sess.t[k].cpu().numpy() for k in ("x", "y", "z", "vr", "lth", "lph")}
    sess.close()
    R = np.hypot(x, y)
    for k, ref in (("x", x), ("y", y), ("z", z)):
        assert np.abs(got[k] - ref).max() <= 1e-7 * R.max(), k
    speed = np.abs(lph / R)
    for k, ref, sc in (("vr", vr, speed), ("lth", lth, speed * np.hypot(R, z)), ("lph", lph, speed * R)):
        err = (np.abs(got[k] - ref) / sc).max()
        assert err < 1e-6, (k, err)
    # the particles did move and the velocities changed
    assert np.abs(got["x"] - ins["x"]).max() > 1e3 * 1e-7 * R.max()
    assert np.abs(got["vr"] - ins["vr"]).max() > 1e-3 * np.abs(ins["vr"]).max()


def test_push_matches_oracle(gd, oracle):
    ins = W.disk_instance(4096, seed=6, K=32, velocities=True, sizes=("lognormal", 1.0, 0.5))
    sess = gd.Session([ins], precision=gd.GD_FP64, velocities=True)
    dt = 3.0e7
    sess.push_staggered(dt)
    sess.stats()
    P = oracle.params(ins["params"])
    x, y, z = ins["x"].copy(), ins["y"].copy(), ins["z"].copy()
    vr, lth, lph = ins["vr"].copy(), ins["lth"].copy(), ins["lph"].copy()
    oracle.push(P, x, y, z, vr, lth, lph, ins["s"], dt, drag=True)
    for k, ref in (("x", x), ("y", y), ("z", z), ("lph", lph)):
        got = sess.t[k].cpu().numpy()
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-12 * scale, k
    # velocities pass through acos/atan2/sin/cos/exp/expm1 (CUDA vs libm differ by a few
    # ulp) and the 1 - R/r cancellation of the vertical gas factor: 1e-10 of their scale
    for k, ref in (("vr", vr), ("lth", lth)):
        got = sess.t[k].cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), k
    sess.close()


def test_sequencing_errors(gd):
    ins = W.patch_instance(256, K=16, seed=1)
    sess = gd.Session([ins])
    with pytest.raises(gd.GDError) as e:
        gd.gd_collision_rates(sess.ctx)
    assert e.value.code == gd.GD_ERR_STATE
    with pytest.raises(gd.GDError):
        gd.gd_sample_collisions(sess.ctx)
    with pytest.raises(gd.GDError):
        gd.gd_push_staggered(sess.ctx, 1.0)     # no velocities configured
    sess.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_full_size_disk_sampled(gd, oracle, precision):
    """The benchmark workload at full size (2^22 particles, log-normal sizes, K = 32) in
    the launch configuration bench.py times: lists, distances and rates of sampled
    particles against the oracle's brute force, and two whole intervals without any
    status bit (no failed search, no event cap, no non-finite rate)."""
    ins = W.config2()[0]
    sess = gd.Session([ins], precision=precision, flags=gd.GD_FLAG_TIMING)
    nbr, d = sess.build_neighbors(want=True)
    lam, _ = sess.collision_rates(want=True)
    sess.sample_collisions()
    sess.build_neighbors()
    sess.collision_rates()
    sess.sample_collisions()
    st = sess.stats(check=False)
    assert st["status"] == 0, st["status"]
    P = oracle.params(ins["params"])
    rng = np.random.default_rng(17)
    q = rng.choice(len(ins["x"]), 48, replace=False)
    # include the innermost and the highest particles (densest / sparsest regions)
    R = np.hypot(ins["x"], ins["y"])
    q = np.concatenate([q, [int(np.argmin(R)), int(np.argmax(np.abs(ins["z"])))]])
    onbr, od = oracle.knn(P, ins["x"], ins["y"], ins["z"], q)
    assert np.array_equal(nbr.cpu().numpy()[q], onbr)
    assert np.array_equal(d.cpu().numpy()[q], od)
    r = oracle.rates_subset(P, ins["x"], ins["y"], ins["z"], ins["s"], ins["M"], q, onbr, od)
    rel = np.abs(lam.cpu().numpy()[q] / r["lam"] - 1.0)
    assert rel.max() < (1e-12 if precision == 0 else 1e-4), rel.max()
    sess.close()


def test_autotune_keeps_lists_exact(gd, oracle):
    ins = W.disk_instance(1 << 14, seed=31, K=32, sizes=("lognormal", 10.0, 1.0))
    sess = gd.Session([ins], precision=gd.GD_MIXED)
    f, xs = sess.autotune()
    assert 0.35 < f < 1.5 and xs in (1, 2, 4)
    nbr, d = sess.build_neighbors(want=True)
    P = oracle.params(ins["params"])
    q = np.arange(0, len(ins["x"]), 97)
    onbr, od = oracle.knn(P, ins["x"], ins["y"], ins["z"], q)
    assert np.array_equal(nbr.cpu().numpy()[q], onbr)
    assert np.array_equal(d.cpu().numpy()[q], od)
    sess.close()

"""GPU parity at the full sizes of the five workload shapes, in the launch configuration
bench.py times, on sampled outputs the oracle computes one by one.

Sampled particles are checked against the oracle's brute force (lists and distances
bit-exact, rates within the form's bound) and, for the first interval, their whole event
sequence is replayed by the oracle with the GPU's interval length (particles are
independent inside an interval, so this is an exact check of the sampled ones).
"""
import numpy as np
import pytest

from paper_2609_35967_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RATE_TOL = {0: 1e-12, 1: 1e-4}


def _sample(n, k, seed, extra=()):
    q = np.random.default_rng(seed).choice(n, k, replace=False)
    return np.unique(np.concatenate([q, np.asarray(extra, dtype=np.int64)]))


def _check_subset(oracle, P, ins, q, nbr, d, lam, precision, events=None, interval=0, chan=None):
    onbr, od = oracle.knn(P, ins["x"], ins["y"], ins["z"], q)
    assert np.array_equal(nbr[q], onbr)
    assert np.array_equal(d[q], od)
    r = oracle.rates_subset(P, ins["x"], ins["y"], ins["z"], ins["s"], ins["M"], q, onbr, od,
                            chan=chan is not None)
    rel = np.abs(lam[q] / r["lam"] - 1.0)
    assert rel.max() < RATE_TOL[precision], rel.max()
    if chan is not None:
        # every channel rate of every slot: zeros exactly zero, the rest within the bound
        rc, gc = r["chan"], chan[q]
        assert np.array_equal(rc == 0.0, gc == 0.0)
        nz = rc != 0.0
        assert np.abs(gc[nz] / rc[nz] - 1.0).max() < RATE_TOL[precision]
    if events is None:
        return 0
    ec, eh, nn, dt_exe = events
    o = oracle.sample_subset(P, ins["x"], ins["y"], ins["z"], ins["s"], ins["M"], q, onbr, od,
                             dt_exe, interval)
    same = (o["ev_count"] == ec[q]) & (o["ev_hash"] == eh[q])
    flagged = (o["near"] > 0) | (nn[q] > 0)
    bad = int((~same & ~flagged).sum())
    assert bad == 0, bad
    return int(o["ev_count"].sum())


def _extremes(ins):
    R = np.hypot(ins["x"], ins["y"])
    return [int(np.argmin(R)), int(np.argmax(R)), int(np.argmax(np.abs(ins["z"])))]


def test_config1_disk_2p20_fp64(gd, oracle):
    """Global disk of 2^20 equal 1 um grains, K = 32, plain FP64 form."""
    ins = W.config1()[0]
    sess = gd.Session([ins], precision=gd.GD_FP64)
    nbr, d = sess.build_neighbors(want=True)
    lam, chan = sess.collision_rates(want=True, chan=True)
    ec, eh, nn = sess.sample_collisions(want=True)
    st = sess.stats()
    P = oracle.params(ins["params"])
    q = _sample(len(ins["x"]), 256, 21, _extremes(ins))
    _check_subset(oracle, P, ins, q, nbr.cpu().numpy(), d.cpu().numpy(), lam.cpu().numpy(), 0,
                  (ec.cpu().numpy(), eh.cpu().numpy().view(np.uint32), nn.cpu().numpy(),
                   st["instances"][0]["dt_exe"]), chan=chan.cpu().numpy())
    del chan
    for _ in range(2):
        sess.build_neighbors()
        sess.collision_rates()
        sess.sample_collisions()
    st = sess.stats(check=False)
    assert st["status"] == 0 and st["intervals"] == 3
    sess.close()


def test_config2_events_of_sampled_particles(gd, oracle):
    """The bench workload (2^22, log-normal sizes, mixed form): first-interval events of
    sampled particles replayed by the oracle."""
    ins = W.config2()[0]
    sess = gd.Session([ins], precision=gd.GD_MIXED)
    sess.autotune()
    nbr, d = sess.build_neighbors(want=True)
    lam, _ = sess.collision_rates(want=True)
    ec, eh, nn = sess.sample_collisions(want=True)
    st = sess.stats()
    P = oracle.params(ins["params"])
    ecn = ec.cpu().numpy()
    # half of the sample from particles that had events, so the replay is not vacuous
    busy = np.flatnonzero(ecn > 0)
    rng = np.random.default_rng(5)
    q = np.unique(np.concatenate([_sample(len(ins["x"]), 128, 6, _extremes(ins)),
                                  rng.choice(busy, min(128, len(busy)), replace=False)]))
    n_ev = _check_subset(oracle, P, ins, q, nbr.cpu().numpy(), d.cpu().numpy(), lam.cpu().numpy(), 1,
                         (ecn, eh.cpu().numpy().view(np.uint32), nn.cpu().numpy(),
                          st["instances"][0]["dt_exe"]))
    assert n_ev > 0
    sess.close()


def test_config2_mixed_reproduces_fp64(gd):
    """The bench workload at full size, one interval in each form: every one of the 2^22
    particles has the same event count and channel sequence in the mixed form as in the FP64
    form unless a near tie was flagged (the mixed form certifies each FP32 decision against
    its error bound and replays the rest in FP64), the flagged particles stay below 1e-6 of
    the events, and the diameters agree to 1e-12 where the sequences do.  Among them are the
    heavy particles whose open time decisions the deferred FP64 pass settled from their
    logged events (some every interval on this workload)."""
    ins = W.config2()[0]
    res = {}
    for prec in (0, 1):
        sess = gd.Session([ins], precision=prec)
        sess.build_neighbors()
        sess.collision_rates()
        ec, eh, nn = sess.sample_collisions(want=True)
        st = sess.stats()
        res[prec] = (ec.cpu().numpy(), eh.cpu().numpy().view(np.uint32), nn.cpu().numpy(),
                     sess.t["s"].cpu().numpy(), st)
        sess.close()
    (e64, h64, n64, s64, st64), (e32, h32, n32, s32, st32) = res[0], res[1]
    i64, i32 = st64["instances"][0], st32["instances"][0]
    print(f"events {st64['events']} / {st32['events']}; near ties {st64['near_draw']} / {st32['near_draw']}; "
          f"mixed FP64 redo: rates {st32['rate_redo']}, sampling {st32['sample_redo']} "
          f"(deferred {st32['sample_deferred']})")
    assert st64["status"] == 0 and st32["status"] == 0
    assert st32["sample_deferred"] >= 1 and st64["sample_deferred"] == 0
    assert i64["dt_exe"] == i32["dt_exe"] or i32["near_dt"] + i64["near_dt"] > 0
    if i64["dt_exe"] == i32["dt_exe"]:
        same = (e64 == e32) & (h64 == h32)
        flagged = (n64 > 0) | (n32 > 0)
        assert int((~same & ~flagged).sum()) == 0
        assert int(flagged.sum()) <= 1e-6 * st64["events"], (int(flagged.sum()), st64["events"])
        assert np.abs(s32[same] / s64[same] - 1.0).max() < 1e-12


def test_config3_batched_patches_graph(gd, oracle):
    """256 independent patches of log-uniform sizes 2^10-2^16 and their own parameters in
    one context (mixed form, autotuned cells): sampled queries of every patch, whole
    first-interval events of the three smallest patches, then graph-replayed intervals."""
    insts = W.config3()
    offs = W.concat(insts)["offsets"]
    sess = gd.Session(insts, precision=gd.GD_MIXED)
    sess.autotune()
    nbr, d = sess.build_neighbors(want=True)
    lam, _ = sess.collision_rates(want=True)
    ec, eh, nn = sess.sample_collisions(want=True)
    st = sess.stats()
    nbr, d, lam = nbr.cpu().numpy(), d.cpu().numpy(), lam.cpu().numpy()
    ec, eh, nn = ec.cpu().numpy(), eh.cpu().numpy().view(np.uint32), nn.cpu().numpy()
    sizes = np.diff(offs)
    small = set(np.argsort(sizes)[:3].tolist())
    rng = np.random.default_rng(33)
    for b, ins in enumerate(insts):
        lo, hi = offs[b], offs[b + 1]
        P = oracle.params(ins["params"])
        n = hi - lo
        if b in small:
            # the whole patch: lists, rates and events of every particle
            q = np.arange(n)
            ev = (ec[lo:hi], eh[lo:hi], nn[lo:hi], st["instances"][b]["dt_exe"])
        else:
            q = rng.choice(n, 3, replace=False)
            ev = None
        _check_subset(oracle, P, ins, q, nbr[lo:hi] - lo, d[lo:hi], lam[lo:hi], 1, ev)
    M0 = [float(np.sum(i["M"])) for i in insts]
    sess.run_intervals(3)
    st = sess.stats(check=False)
    assert st["status"] == 0 and st["intervals"] == 4
    for b in range(len(insts)):
        assert st["instances"][b]["sum_M"] == pytest.approx(M0[b], rel=1e-12)
    assert np.array_equal(sess.t["M"].cpu().numpy(), W.concat(insts)["M"])
    sess.close()


def test_config4_disk_2p24_k48_push(gd, oracle):
    """Global disk of 2^24 particles, K = 48, mixed form, staggered push after each
    interval: sampled lists/rates/events, then the mixed push of sampled particles against
    the oracle's (1e-7 of the radius, 1e-6 of the velocity scales), then a further interval
    on the pushed positions."""
    ins = W.config4()[0]
    sess = gd.Session([ins], precision=gd.GD_MIXED, velocities=True)
    nbr, d = sess.build_neighbors(want=True)
    lam, _ = sess.collision_rates(want=True)
    ec, eh, nn = sess.sample_collisions(want=True)
    st = sess.stats()
    dt = st["instances"][0]["dt_exe"]
    P = oracle.params(ins["params"])
    q = _sample(len(ins["x"]), 160, 44, _extremes(ins))
    _check_subset(oracle, P, ins, q, nbr.cpu().numpy(), d.cpu().numpy(), lam.cpu().numpy(), 1,
                  (ec.cpu().numpy(), eh.cpu().numpy().view(np.uint32), nn.cpu().numpy(), dt))
    del nbr, d, lam, ec, eh, nn
    s_now = sess.t["s"].cpu().numpy()[q]
    sess.push_staggered(-1.0)
    sess.stats()
    arrs = {k: np.ascontiguousarray(ins[k][q]) for k in ("x", "y", "z", "vr", "lth", "lph")}
    oracle.push(P, arrs["x"], arrs["y"], arrs["z"], arrs["vr"], arrs["lth"], arrs["lph"], s_now, dt,
                drag=True)
    # the mixed push: FP32 angle increments and gas, FP64 positions and forces
    R = np.hypot(arrs["x"], arrs["y"])
    for k in ("x", "y", "z"):
        got = sess.t[k].cpu().numpy()[q]
        assert np.abs(got - arrs[k]).max() <= 1e-7 * R.max(), k
    speed = np.abs(arrs["lph"] / R)
    for k, sc in (("vr", speed), ("lth", speed * np.hypot(R, arrs["z"])), ("lph", speed * R)):
        got = sess.t[k].cpu().numpy()[q]
        assert (np.abs(got - arrs[k]) / sc).max() < 1e-6, k
    sess.build_neighbors()
    sess.collision_rates()
    sess.sample_collisions()
    sess.push_staggered(-1.0)
    st = sess.stats(check=False)
    assert st["status"] == 0 and st["intervals"] == 2
    sess.close()

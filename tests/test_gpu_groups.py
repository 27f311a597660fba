"""GPU parity of spatial groups (Sect. 2.5.3) against the oracle's rounds, and the interval
count of eight groups against one group on the full-size bench disk.

Each round both sides take the groups whose interval ends first: the same groups, levels,
requests, C and interval counters, every particle's event count and channel sequence
(idle groups' particles: none), and the diameters within 1e-12.  A flagged near tie ends
the comparison at that round (both sides are right there; they may part afterwards).
"""
import numpy as np
import pytest

from paper_2609_35967_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FULL = 1 << 60


def dense_inner_disk(n, seed, K=16, factor=100.0, R_au=40.0, G=2):
    """A disk whose particles inside R_au carry factor times the mass, so that the inner
    groups request much shorter intervals and the ratio-16 rule binds."""
    ins = W.disk_instance(n, seed=seed, K=K, sizes=("lognormal", 1.0, 0.7))
    M = ins["M"].copy()
    M[np.hypot(ins["x"], ins["y"]) < R_au * W.AU] *= factor
    ins["M"] = M
    ins["params"] = dict(ins["params"], spatial_groups=G)
    return ins


def _rounds(gd, oracle, ins, G, precision, max_rounds, min_compared):
    P = oracle.params(ins["params"])
    run = oracle.GroupRun(P, G, ins["x"], ins["y"], ins["z"], ins["s"], ins["M"])
    S = run.S
    sess = gd.Session([ins], precision=precision)
    compared = 0
    steps = 0
    delayed = refined = 0
    for r in range(max_rounds):
        sess.build_neighbors()      # every interval call starts with a build (positions are unchanged)
        sess.collision_rates()
        ec, eh, nn = sess.sample_collisions(want=True)
        o = run.round(want=("ev_count", "ev_hash", "near"))
        gs = sess.group_stats(0)
        ec, eh, nn = ec.cpu().numpy(), eh.cpu().numpy().view(np.uint32), nn.cpu().numpy()
        near_audit = sess.stats(check=False)["near_audit"]
        near = bool((nn > 0).any() or (o["near"] > 0).any() or near_audit > 0
                    or any(g["near_dt"] for g in gs) or any(S.st[g].near_dt for g in range(G))
                    or any(S.st[g].near_audit for g in range(G)))
        if near:
            break
        if r == 0:
            for g in range(G):
                assert gs[g]["members"] == S.members[g]
                assert gs[g]["interacts"] == int(S.inter[g]), (g, gs[g]["interacts"], int(S.inter[g]))
        assert gs[0]["round_clock"] == S.t and gs[0]["rounds"] == S.rounds
        for g in range(G):
            a = bool(S.active[g])
            assert bool(gs[g]["active"]) == a, (r, g)
            assert gs[g]["level"] == S.level[g], (r, g, gs[g]["level"], S.level[g])
            assert gs[g]["intervals"] == S.intervals[g]
            assert gs[g]["clock"] == FULL - S.st[g].remain_ticks, (r, g)
            assert gs[g]["C"] == S.st[g].C, (r, g)
            if a:
                assert gs[g]["k_req"] == S.k_req[g]
                assert gs[g]["dt_exe"] == S.st[g].dt_exe
                refined += gs[g]["level"] > gs[g]["k_req"]
            else:
                assert gs[g]["dt_exe"] == 0.0
        assert np.array_equal(ec, o["ev_count"]), r
        assert np.array_equal(eh, o["ev_hash"]), r
        s_gpu = sess.t["s"].cpu().numpy()
        assert np.abs(s_gpu / run.s - 1.0).max() < 1e-12, r
        assert gs[0]["delayed"] == S.delayed and gs[0]["breaks"] == S.breaks
        compared += 1
        if run.done():
            steps += 1
    st = sess.stats(check=False)
    assert st["status"] == 0
    sess.close()
    assert compared >= min_compared, compared
    return compared, steps, S.delayed, refined


@pytest.mark.parametrize("precision", [0, 1])
def test_two_groups_match_oracle(gd, oracle, precision):
    ins = dense_inner_disk(3000, seed=31, G=2)
    # about 580 rounds a collision step: the comparison runs past the first step's end
    compared, steps, delayed, refined = _rounds(gd, oracle, ins, 2, precision, 620, 500)
    assert steps >= 1 and refined > 0


def test_eight_groups_match_oracle(gd, oracle):
    # the dense region inside the first annulus: group 0 requests 2^5-2^6 times shorter
    # intervals than group 1 (about 1160 rounds a step)
    ins = dense_inner_disk(6000, seed=32, R_au=16.0, G=8)
    compared, steps, delayed, refined = _rounds(gd, oracle, ins, 8, gd.GD_FP64, 1200, 1000)
    assert steps >= 1 and refined > 0 and delayed > 0


def test_collide_groups_ends_every_group(gd):
    """gd_collide on a grouped disk completes its step (no timeout) in as many rounds as
    its groups' distinct interval ends, twice in a row; the rounds equal those of the
    same step driven by single interval calls."""
    ins = dense_inner_disk(5000, seed=33, G=4)
    sess = gd.Session([ins], precision=gd.GD_MIXED)
    before = [0] * 4
    for _ in range(2):
        n = sess.collide(ins["params"]["dt_coll"])
        gs = sess.group_stats(0)
        iv = [g["intervals"] - b for g, b in zip(gs, before)]
        assert max(iv) <= n <= sum(iv) and min(iv) >= 1, (n, iv)
        before = [g["intervals"] for g in gs]
    assert sess.stats()["status"] == 0
    sess.close()
    # the same step by single interval calls: rounds until every group reached the end
    sess = gd.Session([ins], precision=gd.GD_MIXED)
    rounds = 0
    while True:
        sess.build_neighbors()
        sess.collision_rates()
        sess.sample_collisions()
        rounds += 1
        gs = sess.group_stats(0)
        if all(g["clock"] == FULL for g in gs if g["members"] > 0):
            break
        assert rounds < 100000
    assert sess.stats()["status"] == 0
    sess.close()


def test_disk22_eight_groups_fewer_updates(gd):
    """The 2^22 bench disk, one collision step with one group and with eight radial groups
    (mixed form): the inner group needs about as many intervals as the single group, the
    outer ones far fewer, so the particle-interval updates drop."""
    ins = W.config2()[0]
    res = {}
    for G in (1, 8):
        i2 = dict(ins, params=dict(ins["params"], spatial_groups=G))
        sess = gd.Session([i2], precision=gd.GD_MIXED)
        rounds = sess.collide(ins["params"]["dt_coll"])
        gs = sess.group_stats(0)
        upd = sum(g["members"] * g["intervals"] for g in gs)
        res[G] = (rounds, [g["intervals"] for g in gs], upd, gs[0]["delayed"], gs[0]["breaks"])
        assert sess.stats()["status"] == 0
        sess.close()
    print("one group: %d intervals, %d updates; eight groups: %d rounds, intervals %s, %d updates, "
          "delayed %d, breaks %d" % (res[1][0], res[1][2], res[8][0], res[8][1], res[8][2], res[8][3], res[8][4]))
    assert res[8][2] < res[1][2]
    assert max(res[8][1]) >= res[1][1][0] // 2


def test_batched_grouped_and_plain_instances(gd, oracle):
    """One context with a three-group disk, a plain patch and a two-slab patch: each instance
    advances by its own rounds (the plain one by intervals) and matches its own oracle run;
    the units of the later instances sit behind the first instance's groups."""
    disk = dense_inner_disk(2000, seed=34, G=3)
    plain = W.patch_instance(900, K=16, seed=35)
    slabs = W.patch_instance(1200, K=16, seed=36)
    slabs["params"] = dict(slabs["params"], spatial_groups=2)
    insts = [disk, plain, slabs]
    Gs = [3, 1, 2]
    runs = [oracle.GroupRun(oracle.params(i["params"]), G, i["x"], i["y"], i["z"], i["s"], i["M"])
            for i, G in zip(insts, Gs)]
    offs = W.concat(insts)["offsets"]
    sess = gd.Session(insts, K=16, precision=gd.GD_FP64)
    compared = 0
    for r in range(60):
        sess.build_neighbors()
        sess.collision_rates()
        ec, eh, nn = sess.sample_collisions(want=True)
        ec, eh, nn = ec.cpu().numpy(), eh.cpu().numpy().view(np.uint32), nn.cpu().numpy()
        s_gpu = sess.t["s"].cpu().numpy()
        outs = [run.round(want=("ev_count", "ev_hash", "near")) for run in runs]
        if (nn > 0).any() or any((o["near"] > 0).any() for o in outs):
            break
        for b, (run, o, G) in enumerate(zip(runs, outs, Gs)):
            lo, hi = offs[b], offs[b + 1]
            assert np.array_equal(ec[lo:hi], o["ev_count"]), (r, b)
            assert np.array_equal(eh[lo:hi], o["ev_hash"]), (r, b)
            assert np.abs(s_gpu[lo:hi] / run.s - 1.0).max() < 1e-12, (r, b)
            gs = sess.group_stats(b)
            assert len(gs) == G
            for g in range(G):
                assert gs[g]["level"] == run.S.level[g] and gs[g]["C"] == run.S.st[g].C, (r, b, g)
                assert gs[g]["clock"] == FULL - run.S.st[g].remain_ticks or G == 1, (r, b, g)
        compared += 1
    assert compared >= 40, compared
    assert sess.stats()["status"] == 0
    sess.close()

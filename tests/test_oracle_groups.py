"""Pins of the oracle's spatial groups (Sect. 2.5.3): each group keeps its own
frozen-neighbour intervals, interacting groups stay within a ratio of 16, and a
scheduled interval is kept, so a refinement may wait.

* the scheduling rule on hand-worked cases (levels k: intervals dt_coll 2^-k);
* one group is the single-group interval loop, bit for bit;
* two groups whose lists never meet evolve exactly as each group alone;
* an interacting disk: every group ends the step exactly, no interacting pair is ever more
  than 16 apart, the interaction masks are those of the lists, and the busy inner
  groups take more intervals than the outer ones.
"""
import math

import numpy as np
import pytest

from paper_2609_35967_gb300 import workloads as W

FULL = 1 << 60


def _sched(G, pairs, active, k_req, level, k_fit=None):
    from oracle import gdo
    inter = np.zeros(G, dtype=np.uint64)
    for g, h in pairs:
        inter[g] |= np.uint64(1 << h)
        inter[h] |= np.uint64(1 << g)
    level = np.array(level, dtype=np.int32)
    d, b = gdo.schedule(G, inter, np.ones(G), active, k_req, k_fit if k_fit is not None else [0] * G, level)
    return level.tolist(), d, b


def test_schedule_hand_worked(oracle):
    # step start, both active: the coarse group is refined to within 4 levels of the fine one
    assert _sched(2, [(0, 1)], [1, 1], [9, 0], [-1, -1]) == ([9, 5], 0, 0)
    # group 1 is in the middle of a whole-step interval (level 0): group 0's request for
    # level 9 waits at level 4 (a delayed refinement), its step-end floor 1 is below that
    assert _sched(2, [(0, 1)], [1, 0], [9, 0], [-1, 0], [1, 0]) == ([4, 0], 1, 0)
    # a scheduled fine neighbour (level 10) refines a coarse request to level 6
    assert _sched(2, [(0, 1)], [1, 0], [0, 0], [-1, 10]) == ([6, 10], 0, 0)
    # a chain 0-1-2 (0 and 2 do not interact): 12 -> 8 -> 4
    assert _sched(3, [(0, 1), (1, 2)], [1, 1, 1], [12, 0, 0], [-1] * 3) == ([12, 8, 4], 0, 0)
    # the chain with group 2 scheduled at level 1: group 1 may go no finer than 5 and group 0
    # no finer than 9 (delayed); group 1 is then refined from 3 to 5
    assert _sched(3, [(0, 1), (1, 2)], [1, 1, 0], [12, 3, 0], [-1, -1, 1]) == ([9, 5, 1], 1, 0)
    # groups that do not interact keep their requests
    assert _sched(2, [], [1, 1], [12, 0], [-1, -1]) == ([12, 0], 0, 0)
    # the end of the step wins over the ratio: floor 8 against a neighbour at level 2
    assert _sched(2, [(0, 1)], [1, 0], [8, 0], [-1, 2], [8, 0]) == ([8, 2], 0, 1)


def test_group_of_edges(oracle):
    P = oracle.params(W.disk_instance(64, seed=3)["params"])
    R_in, R_out = P.R_in, P.R_out
    assert oracle.group_of(P, 8, R_in, 0.0) == 0
    assert oracle.group_of(P, 8, 0.0, R_out) == 7          # the outer edge joins the last group
    assert oracle.group_of(P, 8, 0.5 * R_in, 0.0) == 0     # inside R_in: the first group
    assert oracle.group_of(P, 8, 2 * R_out, 0.0) == 7
    assert oracle.group_of(P, 8, math.nan, 0.0) == 0
    # equal widths: the midpoint of annulus g lies in g
    for g in range(8):
        R = R_in + (g + 0.5) * (R_out - R_in) / 8
        assert oracle.group_of(P, 8, R / math.sqrt(2), R / math.sqrt(2)) == g
    Pp = oracle.params(W.patch_instance(64, seed=3)["params"])
    assert oracle.group_of(Pp, 4, -0.5 * Pp.box_x, 0.0) == 0
    assert oracle.group_of(Pp, 4, 0.0, 123.0) == 2
    assert oracle.group_of(Pp, 4, 0.4999 * Pp.box_x, 0.0) == 3


def test_one_group_is_the_interval_loop(oracle):
    ins = W.patch_instance(700, K=16, seed=5)
    P = oracle.params(ins["params"])
    run = oracle.GroupRun(P, 1, ins["x"], ins["y"], ins["z"], ins["s"], ins["M"])
    st = oracle.new_state(P)
    s = np.array(ins["s"], dtype=np.float64)
    for r in range(12):
        o1 = oracle.interval_step(P, st, ins["x"], ins["y"], ins["z"], s, ins["M"],
                                  want=("ev_count", "ev_hash"))
        o2 = run.round()
        g = run.S.st[0]
        assert g.dt_exe == st.dt_exe and g.dt_req == st.dt_req, r
        assert g.C == st.C and g.interval == st.interval and g.events == st.events, r
        assert np.array_equal(o1["ev_count"], o2["ev_count"]) and np.array_equal(o1["ev_hash"], o2["ev_hash"])
        assert np.array_equal(run.s, s), r
    assert run.S.intervals[0] == 12 and run.S.rounds == 12


def _rings(n_each, K, seed, order):
    """Two rings of one disk, R in [10, 12] au and [60, 62] au: the K nearest neighbours of
    every particle lie in its own ring.  order "AB" puts ring A first in index order."""
    ins = W.disk_instance(2 * n_each, seed=seed, K=K, sizes=("lognormal", 1.0, 0.5))
    x, y, z = ins["x"], ins["y"], ins["z"]
    R = np.hypot(x, y)
    rng = np.random.default_rng(seed + 1)
    Rn = np.concatenate([rng.uniform(10, 12, n_each), rng.uniform(60, 62, n_each)]) * W.AU
    f = Rn / R
    out = dict(ins, x=x * f, y=y * f, z=z * f)
    idx = np.arange(2 * n_each) if order == "AB" else np.r_[n_each:2 * n_each, 0:n_each]
    for k in ("x", "y", "z", "s", "M"):
        out[k] = np.ascontiguousarray(out[k][idx])
    return out


def test_groups_apart_evolve_alone(oracle):
    n1, K = 300, 16
    for order, g_first in (("AB", 0), ("BA", 1)):
        both = _rings(n1, K, 21, order)
        P = oracle.params(both["params"])
        s2 = np.array(both["s"])
        rounds, S = oracle.collide_groups(P, 2, both["x"], both["y"], both["z"], s2, both["M"])
        assert S.inter[0] == 0 and S.inter[1] == 0 and S.members[0] == S.members[1] == n1
        # the first n1 particles, alone in an instance of one group
        one = {k: np.ascontiguousarray(both[k][:n1]) for k in ("x", "y", "z", "s", "M")}
        s1 = np.array(one["s"])
        r1, S1 = oracle.collide_groups(P, 1, one["x"], one["y"], one["z"], s1, one["M"])
        assert np.array_equal(s2[:n1], s1)
        assert S.intervals[g_first] == S1.intervals[0] == r1
        assert S.st[g_first].C == S1.st[0].C and S.st[g_first].events == S1.st[0].events
        # each group's own clock: the rounds are the distinct interval ends of both groups
        assert max(S.intervals[0], S.intervals[1]) <= rounds <= S.intervals[0] + S.intervals[1]
    assert S.intervals[0] > S.intervals[1]     # the inner ring collides faster


def dense_inner_disk(n, seed=8, K=16, factor=100.0, R_au=40.0):
    """A disk whose particles inside R_au carry factor times the mass: their partners are
    that much more numerous, so the inner groups request intervals 2^6-2^7 times shorter
    and the ratio-16 rule binds."""
    ins = W.disk_instance(n, seed=seed, K=K, sizes=("lognormal", 1.0, 0.7))
    M = ins["M"].copy()
    M[np.hypot(ins["x"], ins["y"]) < R_au * W.AU] *= factor
    ins["M"] = M
    return ins


def test_interacting_groups_schedule(oracle):
    ins = dense_inner_disk(2500)
    P = oracle.params(ins["params"])
    G = 3
    run = oracle.GroupRun(P, G, ins["x"], ins["y"], ins["z"], ins["s"], ins["M"])
    S = run.S
    # the interaction masks are those of the lists, by brute force
    want = np.zeros((G, G), dtype=bool)
    for i in range(len(run.grp)):
        for j in run.nbr[i]:
            want[run.grp[i], run.grp[j]] = want[run.grp[j], run.grp[i]] = True
    np.fill_diagonal(want, False)
    got = np.array([[(int(S.inter[g]) >> h) & 1 for h in range(G)] for g in range(G)], dtype=bool)
    assert np.array_equal(got, want)
    assert [S.members[g] for g in range(G)] == np.bincount(run.grp, minlength=G).tolist()
    ends = np.zeros(G, dtype=np.int64)
    last_t = -1
    covered = np.zeros(G, dtype=np.int64)
    refined = 0
    while True:
        run.round()
        assert S.t > last_t
        last_t = S.t
        lv = [S.level[g] for g in range(G)]
        for g in range(G):
            if S.active[g]:
                refined += lv[g] > S.k_req[g]
                assert ends[g] == S.t                # a group starts where its last interval ended
                ends[g] += 1 << (60 - lv[g])
                covered[g] += 1 << (60 - lv[g])
                assert S.st[g].dt_exe == math.ldexp(P.dt_coll, -lv[g])
        for g in range(G):
            for h in range(G):
                if got[g, h]:
                    assert abs(lv[g] - lv[h]) <= 4, (S.t, lv)
        if run.done():
            break
    assert np.all(covered == FULL) and np.all(ends == FULL)
    assert S.breaks == 0
    # the rule binds both ways: requests refined for a fine neighbour, refinements delayed
    assert refined > 0 and S.delayed > 0, (refined, S.delayed)
    iv = [S.intervals[g] for g in range(G)]
    assert iv[0] >= iv[-1] and iv[0] > 1, iv
    assert S.rounds >= max(iv)
    # the next call starts a new step at clock 0 with every group active
    run.round()
    assert S.t == 0 and all(S.active[g] for g in range(G))


def test_schedule_invariants_random(oracle):
    """The scheduling rule on 3000 random cases (up to 10 groups, random interactions, active
    sets, scheduled levels within 4 of each other where they interact, requests and step-end
    floors): every active group ends inside the step (level >= floor); every interacting pair
    with an active member ends within 4 levels unless a break is counted; a group is coarser
    than its request only when a scheduled neighbour holds it (a delay is counted) and finer
    only for a floor or a neighbour; and the result does not depend on the groups' order."""
    rng = np.random.default_rng(77)
    for case in range(3000):
        G = int(rng.integers(2, 11))
        inter = np.zeros((G, G), dtype=bool)
        for g in range(G):
            for h in range(g + 1, G):
                if rng.random() < 0.4:
                    inter[g, h] = inter[h, g] = True
        active = rng.random(G) < 0.5
        # scheduled levels of the inactive groups: a consistent state (interacting ones within 4)
        level = np.full(G, -1, dtype=np.int32)
        base = int(rng.integers(0, 30))
        for g in range(G):
            if not active[g]:
                level[g] = base + int(rng.integers(0, 3))
        k_req = rng.integers(0, 45, G).astype(np.int32)
        k_fit = np.minimum(rng.integers(0, 6, G), k_req).astype(np.int32)
        masks = [sum(1 << h for h in range(G) if inter[g, h]) for g in range(G)]
        lv = level.copy()
        d, b = _sched_raw(oracle, G, masks, active, k_req, k_fit, lv)
        for g in range(G):
            if not active[g]:
                assert lv[g] == level[g]
                continue
            assert lv[g] >= k_fit[g]
            if lv[g] < k_req[g]:
                # held back by an inactive interacting group within 4 levels of it, or by a chain
                assert any(inter[g, h] for h in range(G)), case
        n_far = sum(1 for g in range(G) for h in range(g + 1, G)
                    if inter[g, h] and (active[g] or active[h]) and abs(int(lv[g]) - int(lv[h])) > 4)
        assert n_far == b, (case, n_far, b)
        assert d == sum(1 for g in range(G) if active[g] and lv[g] < k_req[g])
        # the same case with the groups in reverse order gives the reversed levels
        rev = list(range(G))[::-1]
        masks_r = [sum(1 << rev.index(h) for h in range(G) if inter[g, h]) for g in rev]
        lv_r = level[rev].copy()
        _sched_raw(oracle, G, masks_r, active[rev], k_req[rev], k_fit[rev], lv_r)
        assert np.array_equal(lv_r[::-1], lv), case


def _sched_raw(oracle, G, masks, active, k_req, k_fit, level):
    from oracle import gdo
    inter = np.array(masks, dtype=np.uint64)
    return gdo.schedule(G, inter, np.ones(G), np.asarray(active, dtype=np.int32), k_req, k_fit, level)

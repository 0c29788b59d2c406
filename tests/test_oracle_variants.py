"""Pins of the oracle's reduction variants (rules SE and FE of Section 3.1,
the "MD+SE" and KernelGPU-FE variants of Section 5.1).

Each expected value comes from something other than the oracle: the f = 1
special case (SE is Weihe's W2 there), the matrix form of Algorithms 1-3
with the SE test, FE applied to all full hyperedges at once, brute force
over vertex subsets, hand-derived small cases, and invariants the rules fix.
"""
import numpy as np
import pytest

import pins
from oracle import oracle as O
from paper_2109_06042_gb300 import instances as I


def _as_lists(r):
    return {k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in r.items()}


# ---------------------------------------------------------------- SE (MD+SE)

def test_se_is_weihe_for_unit_demands():
    """With f = 1, SE (subset, f_i >= f_j) is W2, the same test as DP."""
    for seed in range(120):
        rng = np.random.default_rng(30_000 + seed)
        n = int(rng.integers(1, 30))
        m = int(rng.integers(0, 40))
        inst = I.uniform_random(n, m, 1, min(6, n), 1, 0, 30_000 + seed)
        if seed % 3 == 0 and m >= 2:
            edges = inst.edges()
            edges[-1] = list(edges[0])
            inst = I.from_edges(n, edges, [1] * m)
        v, e, r = pins.fone_kernelize(inst)
        res = O.reduce_variant(inst, "se")
        assert res["vertices"].tolist() == v and res["edges"].tolist() == e, seed
        assert res["rounds"] == r, seed


@pytest.mark.parametrize("block", range(3))
def test_se_matrix_formulation(block):
    """Algorithm 3 in matrix form with D_ij = [I^E_ij = I^E_ii and f_i >= f_j]."""
    for seed in range(block * 100, block * 100 + 100):
        inst = I.tiny_random(seed, nmax=24, mmax=30) if seed % 2 else \
            I.uniform_random(30, 50, 1, 8, 3, 0, 40_000 + seed)
        mv, me, mr, _ = pins.matrix_kernelize(inst, rule="se")
        for prune in (False, True):
            res = O.reduce_variant(inst, "se", prune=prune)
            assert res["vertices"].tolist() == np.nonzero(mv)[0].tolist(), seed
            assert res["edges"].tolist() == np.nonzero(me)[0].tolist(), seed
            assert res["rounds"] == mr, seed
            assert res["demands"].tolist() == [int(inst.demand[i]) for i in res["edges"]]


@pytest.mark.parametrize("block", range(3))
def test_se_brute_force_minimum_preserved(block):
    """SE and MD are safe rules: same minimum (None = infeasible)."""
    for seed in range(block * 200, block * 200 + 200):
        inst = I.tiny_random(seed)
        edges = inst.edges()
        before = pins.min_mhs_size(inst.n, edges, inst.demand)
        r = O.reduce_variant(inst, "se")
        kern = [edges[i] for i in r["edges"]]
        assert before == pins.min_mhs_size(inst.n, kern, r["demands"], allowed=r["vertices"])


def test_se_fixpoint_and_weaker_than_dp():
    """At the end no alive e_i lies inside another alive e_j with
    f_i >= f_j; and an SE deletion is a DP deletion on the same pair, so
    where DP finds nothing to delete in round 1, SE does not either."""
    for seed in range(200):
        inst = I.tiny_random(seed, nmax=24, mmax=30)
        r = O.reduce_variant(inst, "se")
        V = set(r["vertices"].tolist())
        live = {i: set(inst.edges()[i]) & V for i in r["edges"].tolist()}
        f = {i: int(inst.demand[i]) for i in live}
        for i, ei in live.items():
            for j, ej in live.items():
                assert i == j or not (ei <= ej and f[i] >= f[j]), (seed, i, j)
        av, ae = np.ones(inst.n, bool), np.ones(inst.m, bool)
        if not O.dp_pass(inst, av, ae).any():
            one = O.reduce_variant(inst, "se", max_rounds=1)
            assert len(one["edges"]) == inst.m, seed


def test_se_keeps_what_only_dp_deletes():
    """Section 3.1: e_0 = {0,1,2,3} with f = 3 pushes 3 - 1 = 2 >= 2 units
    into e_1 = {1,2,3,4}, so DP deletes e_1; e_0 is no subset of e_1, so
    the SE pass of the first round keeps both."""
    inst = I.from_edges(5, [[0, 1, 2, 3], [1, 2, 3, 4]], [3, 2])
    dp = O.reduce_variant(inst, "dp", max_rounds=1)
    se = O.reduce_variant(inst, "se", max_rounds=1)
    assert 1 not in dp["edges"].tolist()
    assert se["edges"].tolist() == [0, 1]


# ---------------------------------------------------------- FE, KernelGPU-FE

def test_fe_hand_single_full_edge():
    """e_0 = {0,1,2}, f = 3, n = 4, k = 5.  Round 1: DP nothing (one
    hyperedge); MD deletes the isolated v_3; v_0, v_1, v_2 are twins with
    0, 1, 2 lower-index dominators < 3.  Round 2 changes nothing.  FE: e_0
    is full, so v_0..v_2 join the solution and k = 2.  Algorithm 3 on the
    empty rest: one round.  FE again: nothing."""
    inst = I.from_edges(4, [[0, 1, 2]], [3], k=5)
    for rule in ("dp", "se"):
        r = _as_lists(O.reduce_variant(inst, rule, full_edges=True))
        assert r["vertices"] == [] and r["edges"] == [] and r["forced"] == [0, 1, 2]
        assert r["k"] == 2 and r["rounds"] == 3 and r["fe_passes"] == 2


def test_fe_hand_overlapping_full_edges():
    """e_0 = {0,1}, f = 2; e_1 = {1,2,3}, f = 2; k = 5.  Round 1: DP nothing
    (2 - 1 < 2 both ways); MD: v_3 has v_1 (superset) and its twin v_2
    (lower index) as dominators, 2 >= 2, deleted; v_0 and v_2 have one.
    Round 2 changes nothing.  FE: e_0 = {0,1} and e_1 = {1,2} are full;
    S = {0,1,2}, k = 2.  Then one empty round and a last FE pass."""
    inst = I.from_edges(4, [[0, 1], [1, 2, 3]], [2, 2], k=5)
    r = _as_lists(O.reduce_variant(inst, "dp", full_edges=True))
    assert r["vertices"] == [] and r["edges"] == [] and r["forced"] == [0, 1, 2]
    assert r["k"] == 2 and r["rounds"] == 3 and r["fe_passes"] == 2


def test_fe_hand_demand_reaches_zero():
    """Under SE: e_0 = {0,1}, f = 2; e_1 = {1,2,3}, f = 1 (DP would delete
    e_1: 2 - 1 >= 1; SE does not, e_0 is no subset).  Round 1 MD deletes
    v_2 (dominator v_1) and v_3 (v_1 and its lower twin v_2), C >= 1.
    Round 2: e_1 = {1}, f = 1: SE needs f_1 >= f_0, no.  FE: e_0 is full,
    S = {0,1}; e_1 loses v_1 and its demand reaches 0, so it goes too."""
    inst = I.from_edges(4, [[0, 1], [1, 2, 3]], [2, 1], k=3)
    r = _as_lists(O.reduce_variant(inst, "se", full_edges=True))
    assert r["vertices"] == [] and r["edges"] == [] and r["forced"] == [0, 1]
    assert r["k"] == 1 and r["rounds"] == 3 and r["fe_passes"] == 2


@pytest.mark.parametrize("rule", ["dp", "se"])
def test_fe_one_at_a_time_equals_all_at_once(rule):
    """The oracle applies FE per hyperedge as the rule states; the pin
    applies it to all full hyperedges at once, in matrix form."""
    for seed in range(300):
        inst = I.tiny_random(seed, nmax=24, mmax=30) if seed % 3 else \
            I.uniform_random(40, 60, 1, 6, 4, 20, 50_000 + seed)
        p = pins.matrix_kernelize_fe(inst, rule)
        o = _as_lists(O.reduce_variant(inst, rule, full_edges=True))
        for key in ("vertices", "edges", "demands", "forced", "k", "rounds", "fe_passes"):
            assert o[key] == p[key], (seed, key)


@pytest.mark.parametrize("rule", ["dp", "se"])
def test_fe_brute_force_and_invariants(rule):
    """FE is safe: min MHS of the input = |forced| + min MHS of the result
    (with its lowered demands); infeasible stays infeasible.  k drops by
    |forced|, surviving demands are >= 1, and no full hyperedge is left."""
    for seed in range(400):
        inst = I.tiny_random(seed)
        edges = inst.edges()
        before = pins.min_mhs_size(inst.n, edges, inst.demand)
        r = O.reduce_variant(inst, rule, full_edges=True)
        kern = [edges[i] for i in r["edges"]]
        after = pins.min_mhs_size(inst.n, kern, r["demands"], allowed=r["vertices"])
        if before is None:
            assert after is None, seed
        else:
            assert after is not None and before == len(r["forced"]) + after, seed
        assert r["k"] == inst.k - len(r["forced"])
        assert not set(r["forced"].tolist()) & set(r["vertices"].tolist())
        V = set(r["vertices"].tolist())
        for i, f in zip(r["edges"].tolist(), r["demands"].tolist()):
            assert f >= 1 and len(set(edges[i]) & V) != f, seed


def test_fe_without_full_edges_is_algorithm3():
    """Where FE finds no full hyperedge after the first fixpoint, the result
    is Algorithm 3's, with one FE pass."""
    for seed in range(100):
        inst = I.uniform_random(20, 30, 2, 5, 1, 0, 60_000 + seed)
        a = O.reduce(inst)
        b = O.reduce_variant(inst, "dp", full_edges=True)
        if b["forced"].size == 0:
            assert a["vertices"].tolist() == b["vertices"].tolist()
            assert a["edges"].tolist() == b["edges"].tolist()
            assert a["rounds"] == b["rounds"] and b["fe_passes"] == 1

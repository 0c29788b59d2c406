"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each expected value comes
from the paper's worked example, a closed form, a special case that reduces
to Weihe's textbook rules, brute force, or an invariant from the paper's
correctness proofs.
"""
import json
import os

import numpy as np
import pytest

import pins
from oracle import oracle as O
from paper_2109_06042_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _appendix():
    with open(os.path.join(GOLDEN, "appendix_counterexample.json")) as fh:
        g = json.load(fh)
    inst = I.from_edges(g["n"], g["edges"], g["demand"], k=g["k"])
    return g, inst


def test_appendix_example_kernel():
    """Appendix A example, reduced by hand under Algorithms 1-3."""
    g, inst = _appendix()
    exp = g["hand_derived_under_algorithms_1_to_3"]
    for prune in (False, True):
        r = O.reduce(inst, prune=prune)
        assert r["vertices"].tolist() == exp["vertices"]
        assert r["edges"].tolist() == exp["edges"]
        assert r["demands"].tolist() == exp["demands"]
        assert r["rounds"] == exp["rounds"]
        assert r["k"] == g["k"]
    _, _, _, _, trace = O.reduce_state(inst, trace_cap=8)
    assert trace.tolist() == exp["trace_dp_deleted_md_deleted_alive_edges_alive_vertices"]


def test_appendix_example_solution_sizes():
    """The paper's printed sizes: 3 before, 4 after the faulty deletion of v3,
    and the kernel keeps the optimum at 3 (MD must not delete v3)."""
    g, inst = _appendix()
    pv = g["paper_values"]
    assert pins.min_mhs_size(inst.n, inst.edges(), inst.demand) == pv["min_mhs_size"]
    keep = [v for v in range(inst.n) if v != 2]
    assert pins.min_mhs_size(inst.n, inst.edges(), inst.demand, allowed=keep) == \
        pv["min_mhs_size_after_deleting_v3"]
    r = O.reduce(inst)
    assert 2 in r["vertices"].tolist()
    kern_edges = [inst.edges()[i] for i in r["edges"]]
    assert pins.min_mhs_size(inst.n, kern_edges, r["demands"], allowed=r["vertices"]) == \
        pv["min_mhs_size"]


@pytest.mark.parametrize("n", [1, 2, 7, 64])
def test_singleton_family_irreducible(n):
    """Section 3.2 tightness example: n hyperedges {v_i}; nothing reducible."""
    inst = I.from_edges(n, [[i] for i in range(n)], [1] * n)
    r = O.reduce(inst)
    assert r["vertices"].tolist() == list(range(n))
    assert r["edges"].tolist() == list(range(n))
    assert r["rounds"] == 1


def test_empty_and_edge_free_instances():
    """No hyperedges: every vertex has max demand 0 and is deleted (Algorithm 2,
    the conjunction over an empty set holds); no vertices: nothing to do."""
    r = O.reduce(I.from_edges(4, [], []))
    assert r["vertices"].size == 0 and r["edges"].size == 0 and r["rounds"] == 2
    r = O.reduce(I.from_edges(0, [], []))
    assert r["rounds"] == 1


def test_equal_edges_keep_lowest_index():
    """Identical hyperedges with equal demand supersede each other; the
    tie-break of Algorithm 1 keeps the lowest index."""
    inst = I.from_edges(3, [[0, 1, 2], [0, 1, 2], [0, 1, 2]], [2, 2, 2])
    av, ae = np.ones(3, bool), np.ones(3, bool)
    assert O.dp_pass(inst, av, ae).tolist() == [False, True, True]
    # higher demand supersedes lower demand even at a higher index
    inst = I.from_edges(3, [[0, 1, 2], [0, 1, 2]], [1, 2])
    assert O.dp_pass(inst, np.ones(3, bool), np.ones(2, bool)).tolist() == [True, False]


def test_twin_vertices_keep_lowest_index():
    """Vertices with equal hyperedge sets: Algorithm 2 orients the tie from
    the lower to the higher index, so with max demand 1 only the lowest
    survives."""
    inst = I.from_edges(4, [[0, 1, 2, 3]], [1])
    dv, cnt, mxf = O.md_pass(inst, np.ones(4, bool), np.ones(1, bool))
    assert dv.tolist() == [False, True, True, True]
    assert cnt.tolist() == [0, 1, 2, 3]
    assert mxf.tolist() == [1, 1, 1, 1]


def test_demand_pushing_beyond_inclusion():
    """DP deletes e_j that is not a superset of e_i (Section 3.1, the rule
    generalises SE): f(e_i) - |e_i \\ e_j| = 3 - 1 >= 2 = f(e_j)."""
    inst = I.from_edges(5, [[0, 1, 2, 3], [1, 2, 3, 4]], [3, 2])
    de = O.dp_pass(inst, np.ones(5, bool), np.ones(2, bool))
    assert de.tolist() == [False, True]


def _rand_small(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    m = int(rng.integers(0, 60))
    return I.uniform_random(n, m, 1, min(8, n), int(rng.integers(1, 5)), 0, seed)


@pytest.mark.parametrize("block", range(4))
def test_matrix_formulation_agrees(block):
    """The paper's matrix form (Eq. (1), Eq. (2), Algorithms 1-3) agrees with
    the oracle's explicit set tests round by round."""
    for seed in range(block * 60, block * 60 + 60):
        inst = _rand_small(seed) if seed % 2 else I.tiny_random(seed, nmax=24, mmax=30)
        mv, me, mr, mtrace = pins.matrix_kernelize(inst)
        for prune in (False, True):
            av, ae, r, ch, tr = O.reduce_state(inst, prune=prune, trace_cap=64)
            assert r == mr, seed
            assert np.array_equal(av, mv), seed
            assert np.array_equal(ae, me), seed
            assert np.array_equal(tr, mtrace), seed


def test_matrix_formulation_uniform_workload():
    """Same on the plain 200 x 400 workload (several seeds)."""
    for seed in range(3):
        inst = I.config_uniform(seed)
        mv, me, mr, mtrace = pins.matrix_kernelize(inst)
        av, ae, r, _, tr = O.reduce_state(inst, trace_cap=64)
        assert r == mr and np.array_equal(av, mv) and np.array_equal(ae, me)
        assert np.array_equal(tr, mtrace)


def test_f_one_reduces_to_weihe():
    """With f = 1, DP is W2 and MD is W1 (Section 1 vs Section 3.1)."""
    for seed in range(150):
        rng = np.random.default_rng(10_000 + seed)
        n = int(rng.integers(1, 30))
        m = int(rng.integers(0, 40))
        inst = I.uniform_random(n, m, 1, min(6, n), 1, 0, 10_000 + seed)
        if seed % 3 == 0 and m >= 2:  # force duplicates and twins
            edges = inst.edges()
            edges[-1] = list(edges[0])
            inst = I.from_edges(n, edges, [1] * m)
        v, e, r = pins.fone_kernelize(inst)
        res = O.reduce(inst)
        assert res["vertices"].tolist() == v, seed
        assert res["edges"].tolist() == e, seed
        assert res["rounds"] == r, seed


@pytest.mark.parametrize("block", range(5))
def test_brute_force_minimum_preserved(block):
    """Lemmas for Algorithms 1 and 2: the kernel has the same minimum
    multiple hitting set size (None = infeasible) as the input; 1000
    instances in total, n <= 16."""
    for seed in range(block * 200, block * 200 + 200):
        inst = I.tiny_random(seed)
        edges = inst.edges()
        before = pins.min_mhs_size(inst.n, edges, inst.demand)
        r = O.reduce(inst)
        kern = [edges[i] for i in r["edges"]]
        after = pins.min_mhs_size(inst.n, kern, r["demands"], allowed=r["vertices"])
        assert before == after, seed
        assert r["demands"].tolist() == [int(inst.demand[i]) for i in r["edges"]]
        assert r["k"] == inst.k


def test_rounds_bounded_by_matching_number():
    """The proof of the parallel kernelization theorem (Section 4.1) bounds
    the iterations of Algorithm 3 that change the hypergraph by nu(I(H)) + 1.
    The round count here also includes the final pass that changes nothing,
    so rounds - 1 <= nu + 1."""
    for seed in range(300):
        inst = I.tiny_random(seed, nmax=24, mmax=30) if seed % 2 else _rand_small(seed)
        r = O.reduce(inst)
        assert r["rounds"] - 1 <= pins.matching_number(inst) + 1, seed
    for seed in range(3):
        inst = I.config_uniform(seed)
        assert O.reduce(inst)["rounds"] - 1 <= pins.matching_number(inst) + 1


def test_idempotent():
    """The output is exhaustively reduced: reducing it again changes nothing
    and takes one round (Lemmas for Algorithms 1 and 2, part (iii))."""
    for seed in range(200):
        inst = I.tiny_random(seed, nmax=24, mmax=30) if seed % 2 else _rand_small(seed)
        av, ae, _, _, _ = O.reduce_state(inst)
        av2, ae2, r2, ch2, _ = O.reduce_state(inst, alive_v=av, alive_e=ae)
        assert r2 == 1 and not ch2
        assert np.array_equal(av, av2) and np.array_equal(ae, ae2)


def test_pass_invariants():
    """Proof of the lemma for Algorithm 1: every hyperedge a DP pass deletes
    is superseded by a hyperedge that survives the pass.  Proof of the lemma
    for Algorithm 2: every deleted vertex keeps at least max f dominators
    among the vertices that survive the pass.  Checked with set algebra."""
    for seed in range(200):
        inst = I.tiny_random(seed, nmax=24, mmax=30) if seed % 2 else _rand_small(seed)
        edges = [set(e) for e in inst.edges()]
        f = inst.demand
        av = np.ones(inst.n, bool)
        ae = np.ones(inst.m, bool)
        for _ in range(50):
            de = O.dp_pass(inst, av, ae)
            alive_vs = set(np.nonzero(av)[0].tolist())
            cur = [e & alive_vs for e in edges]
            surv = ae & ~de
            for j in np.nonzero(de)[0]:
                assert any(pins.supersedes_sets(cur[i], cur[j], f[i], f[j])
                           for i in np.nonzero(surv)[0] if i != j), (seed, j)
            ae = surv
            dv, _, mxf = O.md_pass(inst, av, ae)
            Ev = {v: {i for i in np.nonzero(ae)[0] if v in edges[i]} for v in range(inst.n)}
            survv = av & ~dv
            for j in np.nonzero(dv)[0]:
                doms = [i for i in np.nonzero(survv)[0] if i != j and Ev[j] <= Ev[i]]
                need = max((int(f[e]) for e in Ev[j]), default=0)
                assert mxf[j] == need
                assert len(doms) >= need, (seed, j)
            av = survv
            if not de.any() and not dv.any():
                break


def test_pruned_equals_unpruned_medium():
    """The exact candidate pruning never changes the result."""
    for seed in range(20):
        inst = I.uniform_random(300, 600, 1, 10, 4, 0, 777 + seed)
        a = O.reduce(inst, prune=True)
        b = O.reduce(inst, prune=False)
        for key in ("vertices", "edges", "rounds"):
            assert np.array_equal(a[key], b[key])

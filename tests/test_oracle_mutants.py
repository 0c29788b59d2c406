"""Planted mistakes in the oracle must each fail at least one pin.

Every variant is the oracle compiled with one ``ORACLE_MUTANT_*`` define
(a transposed set difference, a dropped demand term, a reversed or missing
tie-break, strict instead of non-strict comparison, demands taken over
hyperedges already deleted in the round, passes run in the wrong order,
isolated vertices kept, a superedge test without its demand condition, FE
without its demand decrement, ...).  This runs on the CPU only.
"""
import json
import os

import numpy as np
import pytest

import pins
from oracle import oracle as O
from paper_2109_06042_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _same(res, v, e, r):
    return res["vertices"].tolist() == list(v) and res["edges"].tolist() == list(e) \
        and res["rounds"] == r


def _first_failing_pin(mutant):
    with open(os.path.join(GOLDEN, "appendix_counterexample.json")) as fh:
        g = json.load(fh)
    inst = I.from_edges(g["n"], g["edges"], g["demand"], k=g["k"])
    exp = g["hand_derived_under_algorithms_1_to_3"]
    if not _same(O.reduce(inst, mutant=mutant), exp["vertices"], exp["edges"], exp["rounds"]):
        return "appendix"
    for n in (1, 5):
        inst = I.from_edges(n, [[i] for i in range(n)], [1] * n)
        if not _same(O.reduce(inst, mutant=mutant), range(n), range(n), 1):
            return "singleton"
    inst = I.from_edges(4, [], [])
    if O.reduce(inst, mutant=mutant)["vertices"].size != 0:
        return "edge-free"
    for seed in range(40):
        inst = I.uniform_random(12, 16, 1, 6, 1, 0, 20_000 + seed)
        v, e, r = pins.fone_kernelize(inst)
        if not _same(O.reduce(inst, mutant=mutant), v, e, r):
            return "f=1"
    for seed in range(80):
        inst = I.tiny_random(seed, nmax=24, mmax=30)
        mv, me, mr, _ = pins.matrix_kernelize(inst)
        res = O.reduce(inst, mutant=mutant)
        if not _same(res, np.nonzero(mv)[0], np.nonzero(me)[0], mr):
            return "matrix"
    for seed in range(200):
        inst = I.tiny_random(seed)
        edges = inst.edges()
        before = pins.min_mhs_size(inst.n, edges, inst.demand)
        r = O.reduce(inst, mutant=mutant)
        kern = [edges[i] for i in r["edges"]]
        if before != pins.min_mhs_size(inst.n, kern, r["demands"], allowed=r["vertices"]):
            return "brute-force"
    return None


def _first_failing_variant_pin(mutant):
    """Pins of the SE and FE variants (see test_oracle_variants.py)."""
    for seed in range(40):
        inst = I.uniform_random(12, 16, 1, 6, 1, 0, 20_000 + seed)
        v, e, r = pins.fone_kernelize(inst)
        if not _same(O.reduce_variant(inst, "se", mutant=mutant), v, e, r):
            return "se f=1"
    for seed in range(80):
        inst = I.tiny_random(seed, nmax=24, mmax=30)
        mv, me, mr, _ = pins.matrix_kernelize(inst, rule="se")
        if not _same(O.reduce_variant(inst, "se", mutant=mutant), np.nonzero(mv)[0],
                     np.nonzero(me)[0], mr):
            return "se matrix"
    for seed in range(150):
        inst = I.tiny_random(seed, nmax=24, mmax=30)
        for rule in ("dp", "se"):
            p = pins.matrix_kernelize_fe(inst, rule)
            o = O.reduce_variant(inst, rule, full_edges=True, mutant=mutant)
            got = {k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in o.items()}
            if any(got[k] != p[k] for k in ("vertices", "edges", "demands", "forced", "k",
                                             "rounds", "fe_passes")):
                return "fe at once"
    for seed in range(200):
        inst = I.tiny_random(seed)
        edges = inst.edges()
        before = pins.min_mhs_size(inst.n, edges, inst.demand)
        r = O.reduce_variant(inst, "dp", full_edges=True, mutant=mutant)
        kern = [edges[i] for i in r["edges"]]
        after = pins.min_mhs_size(inst.n, kern, r["demands"], allowed=r["vertices"])
        if (before is None) != (after is None) or \
                (before is not None and before != len(r["forced"]) + after):
            return "fe brute-force"
        if r["k"] != inst.k - len(r["forced"]) or any(f < 1 for f in r["demands"]):
            return "fe invariants"
    return None


def test_unmutated_oracle_passes_the_same_pins():
    assert _first_failing_pin(None) is None
    assert _first_failing_variant_pin(None) is None


@pytest.mark.parametrize("mutant", O.MUTANTS)
def test_mutant_is_caught(mutant):
    assert (_first_failing_pin(mutant) or _first_failing_variant_pin(mutant)) is not None, mutant

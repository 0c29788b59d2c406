"""The paper's sequential design (Section 4.2, Algorithms 4-6) against the
pairwise oracle (Algorithms 1-3) and against the pins.

The sequential design tests only candidate pairs (P^E, P^V) and keeps
explicit count matrices; Algorithms 1-3 test every pair every round.  Each
pass removes the same set in both (a pair not in the candidate lists cannot
have changed its outcome), so survivors and the number of passes agree.
"""
import json
import os

import numpy as np
import pytest

import pins
from oracle import kernelcpu as KC
from oracle import oracle as O
from paper_2109_06042_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _same(a, b):
    assert a["vertices"].tolist() == b["vertices"].tolist()
    assert a["edges"].tolist() == b["edges"].tolist()
    assert a["demands"].tolist() == b["demands"].tolist()
    assert a["rounds"] == b["rounds"]


def test_appendix_example():
    with open(os.path.join(GOLDEN, "appendix_counterexample.json")) as fh:
        g = json.load(fh)
    inst = I.from_edges(g["n"], g["edges"], g["demand"], k=g["k"])
    r = KC.reduce(inst)
    exp = g["hand_derived_under_algorithms_1_to_3"]
    assert r["vertices"].tolist() == exp["vertices"]
    assert r["edges"].tolist() == exp["edges"]
    assert r["rounds"] == exp["rounds"]


@pytest.mark.parametrize("block", range(4))
def test_tiny_against_oracle_and_matrix_pin(block):
    for seed in range(block * 250, (block + 1) * 250):
        inst = I.tiny_random(seed, nmax=24, mmax=30)
        r = KC.reduce(inst)
        _same(r, O.reduce(inst))
        if seed % 5 == 0:
            av, ae, rounds, _ = pins.matrix_kernelize(inst)
            assert r["vertices"].tolist() == np.nonzero(av)[0].tolist()
            assert r["edges"].tolist() == np.nonzero(ae)[0].tolist()
            assert r["rounds"] == rounds


def test_uniform_workload_threads():
    for seed in range(6):
        inst = I.config_uniform(seed)
        ref = O.reduce(inst)
        _same(KC.reduce(inst, threads=1), ref)
        _same(KC.reduce(inst, threads=4), ref)


def test_medium_uniform_and_loose():
    for seed in range(4):
        inst = I.uniform_random(400, 800, 1, 10, 4, 0, 900 + seed)
        _same(KC.reduce(inst, threads=2), O.reduce(inst))
    # demands above |e| (infeasible hyperedges) change which zero counts matter
    inst = I.from_edges(6, [[0, 1], [1, 2, 3], [3, 4], [4, 5], [0, 5]], [3, 2, 1, 1, 2])
    _same(KC.reduce(inst), O.reduce(inst))


def test_degenerate():
    _same(KC.reduce(I.from_edges(0, [], [])), O.reduce(I.from_edges(0, [], [])))
    _same(KC.reduce(I.from_edges(5, [], [])), O.reduce(I.from_edges(5, [], [])))
    inst = I.from_edges(3, [[0, 1, 2]] * 4, [2, 2, 1, 3])
    _same(KC.reduce(inst), O.reduce(inst))
    inst = I.from_edges(8, [[i] for i in range(8)], [1] * 8)
    _same(KC.reduce(inst), O.reduce(inst))


def test_refuses_oversized_matrices():
    inst = I.config_uniform(0)
    with pytest.raises(MemoryError):
        KC.reduce(inst, max_bytes=1000)

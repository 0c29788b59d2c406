"""Bit-exact parity of the reduction variants on the GPU (through the C ABI)
with the oracle: the superedge rule SE in place of DP ("MD+SE") and the
alternation with the full-edge rule FE (KernelGPU-FE), Section 5.1.

Compared: surviving vertex and hyperedge ids, current demands, k, rounds,
and with FE the vertices FE put into the solution and the FE pass count.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_06042_gb300 import instances as I

pytestmark = pytest.mark.gpu

MODES = ("fp8", "popcount")
VARIANTS = (("se", False), ("dp", True), ("se", True))


@pytest.fixture(scope="module")
def mhs():
    from paper_2109_06042_gb300 import build
    build.build()
    from paper_2109_06042_gb300 import mhs as M
    return M


def _same(gpu, ref, fe, ctx=""):
    for key in ("vertices", "edges", "demands"):
        assert gpu[key].tolist() == ref[key].tolist(), f"{key} differ {ctx}"
    assert gpu["k"] == ref["k"], f"k {gpu['k']} != {ref['k']} {ctx}"
    assert gpu["rounds"] == ref["rounds"], f"rounds {gpu['rounds']} != {ref['rounds']} {ctx}"
    if fe:
        assert gpu["forced"].tolist() == ref["forced"].tolist(), f"forced differ {ctx}"
        assert gpu["fe_passes"] == ref["fe_passes"], ctx


def _run(mhs, inst, mode, rule, fe, **kw):
    return mhs.kernelize(inst, contraction=mode, rule=rule, full_edges=fe, **kw)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("rule,fe", VARIANTS)
def test_uniform_and_tiny(mhs, mode, rule, fe):
    for seed in range(40):
        inst = I.config_uniform(seed)
        _same(_run(mhs, inst, mode, rule, fe), O.reduce_variant(inst, rule, fe), fe,
              f"uniform {seed}")
    for seed in range(200):
        inst = I.tiny_random(seed, nmax=24, mmax=30)
        _same(_run(mhs, inst, mode, rule, fe), O.reduce_variant(inst, rule, fe), fe,
              f"tiny {seed}")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("rule,fe", VARIANTS)
@pytest.mark.parametrize("n,m", [(129, 257), (257, 640), (700, 1500)])
def test_ragged_sizes(mhs, mode, rule, fe, n, m):
    """Several tiles per side with ragged tails; demands up to 4 make many
    hyperedges full once MD shrinks them."""
    for seed in range(2):
        inst = I.uniform_random(n, m, 1, 8, 4, n // 4, 80_000 + 31 * n + seed)
        _same(_run(mhs, inst, mode, rule, fe), O.reduce_variant(inst, rule, fe), fe,
              f"seed {seed}")


@pytest.mark.parametrize("rule,fe", VARIANTS)
def test_edge_cases(mhs, rule, fe):
    cases = [
        I.from_edges(0, [], []),
        I.from_edges(5, [], []),
        I.from_edges(3, [[], [0]], [1, 1]),            # an empty (infeasible) hyperedge
        I.from_edges(4, [[0, 1, 2]], [3], k=5),         # one full hyperedge
        I.from_edges(4, [[0, 1], [1, 2, 3]], [2, 2], k=5),
        I.from_edges(4, [[0, 1], [1, 2, 3]], [2, 1], k=3),
        I.from_edges(4, [[0, 1, 2, 3]] * 5, [1, 2, 2, 1, 2]),
        I.from_edges(6, [[0, 1, 2, 3, 4, 5]], [7]),     # f > |e|: never full
        I.from_edges(300, [[i] for i in range(300)], [1] * 300),  # all full
    ]
    for mode in MODES:
        for c, inst in enumerate(cases):
            _same(_run(mhs, inst, mode, rule, fe), O.reduce_variant(inst, rule, fe), fe,
                  f"{mode} case {c}")


@pytest.mark.parametrize("sparsity", ["skip", "dense"])
def test_se_empty_hyperedge_zero_tiles(mhs, sparsity):
    """Under SE an empty hyperedge lies within every other one: with f = 3 it
    deletes every hyperedge with f <= 3 it shares nothing with (count 0), so
    tiles without a shared K block must be tested."""
    rng = np.random.default_rng(9)
    n, m = 1000, 2100
    edges = [[]] + [sorted(rng.choice(np.arange(n), size=int(rng.integers(2, 9)),
                                      replace=False).tolist()) for _ in range(m - 1)]
    dem = [2] + [int(rng.integers(1, 4)) for _ in range(m - 1)]
    inst = I.from_edges(n, edges, dem)
    for fe in (False, True):
        ref = O.reduce_variant(inst, "se", fe)
        for mode in MODES:
            _same(_run(mhs, inst, mode, "se", fe, sparsity=sparsity), ref, fe,
                  f"{mode} {sparsity} fe={fe}")


@pytest.mark.parametrize("rule,fe", VARIANTS)
def test_powerlaw_full_size(mhs, rule, fe):
    """n=20,000, m=40,000 power-law workload, tcgen05 path."""
    inst = I.config_powerlaw(0)
    _same(_run(mhs, inst, "fp8", rule, fe), O.reduce_variant(inst, rule, fe), fe)


def test_interval_medium_layouts(mhs):
    for layout in ("input", "sorted", "degree"):
        for rule, fe in VARIANTS:
            inst = I.config_interval(2, n=6000, m=12000)
            _same(_run(mhs, inst, "fp8", rule, fe, layout=layout),
                  O.reduce_variant(inst, rule, fe), fe, f"{layout} {rule} {fe}")


def test_batch_with_variants(mhs):
    """A batch mixes instances that finish at different FE passes."""
    insts = [I.config_batch_one(4300 + i) for i in range(16)]
    insts += [I.from_edges(0, [], []), I.from_edges(4, [[0, 1, 2]], [3], k=5), I.tiny_random(3)]
    for rule, fe in VARIANTS:
        refs = [O.reduce_variant(i, rule, fe) for i in insts]
        for mode in MODES:
            with mhs.Instance.load_batch(insts, contraction=mode, rule=rule, full_edges=fe) as h:
                h.kernelize()
                for b in range(len(insts)):
                    got = h.result(b)
                    if fe:
                        got["forced"], got["fe_passes"] = h.forced(b)
                    _same(got, refs[b], fe, f"{mode} {rule} instance {b}")


def test_round_by_round_with_fe(mhs):
    """One round per call; FE runs right after a fixpoint round, and the
    final state equals the oracle's."""
    inst = I.uniform_random(300, 600, 1, 6, 4, 50, 91_000)
    ref = O.reduce_variant(inst, "dp", True)
    with mhs.Instance.load(inst, contraction="fp8", full_edges=True) as h:
        for _ in range(10_000):
            st = h.reduce_round()
            if st["rounds"] == ref["rounds"] and h.forced()[1] == ref["fe_passes"]:
                break
        got = h.result()
        got["forced"], got["fe_passes"] = h.forced()
        _same(got, ref, True)
        assert h.reduce_round()["rounds"] == ref["rounds"]  # finished: nothing runs


def test_fe_rejects_max_rounds(mhs):
    with pytest.raises(mhs.MhsError) as ei:
        mhs.kernelize(I.config_uniform(0), max_rounds=2, full_edges=True)
    assert ei.value.status == mhs.MHS_EINVAL


@pytest.mark.parametrize("rule,fe", VARIANTS)
def test_server_variants(mhs, rule, fe):
    insts = [I.config_stream_one(7000 + i) for i in range(6)] + \
            [I.config_uniform(s) for s in range(10)]
    with mhs.Server(max_slots=8, contraction="fp8", rule=rule, full_edges=fe) as srv:
        tickets = [srv.submit(i) for i in insts]
        for t, inst in zip(tickets, insts):
            got = srv.poll(t, timeout_us=120_000_000)
            assert got is not None
            ref = O.reduce_variant(inst, rule, fe)
            _same(got, ref, False, f"{rule} ticket {t}")
            if fe:  # the server reports the vertices FE took, not its pass count
                assert got["forced"].tolist() == ref["forced"].tolist(), t

"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

Results are integer sets, so the bar is exact equality of the surviving
vertex ids, hyperedge ids, demands, k and the round count.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_06042_gb300 import instances as I

pytestmark = pytest.mark.gpu

MODES = ("fp8", "popcount")


@pytest.fixture(scope="module")
def mhs():
    from paper_2109_06042_gb300 import build
    build.build()
    from paper_2109_06042_gb300 import mhs as M
    return M


def _same(gpu, ref, ctx=""):
    assert gpu["vertices"].tolist() == ref["vertices"].tolist(), f"vertices differ {ctx}"
    assert gpu["edges"].tolist() == ref["edges"].tolist(), f"edges differ {ctx}"
    assert gpu["demands"].tolist() == ref["demands"].tolist(), f"demands differ {ctx}"
    assert gpu["k"] == ref["k"], ctx
    assert gpu["rounds"] == ref["rounds"], f"rounds {gpu['rounds']} != {ref['rounds']} {ctx}"


@pytest.mark.parametrize("mode", MODES)
def test_uniform_workload_100_seeds(mhs, mode):
    """The plain 200 x 400 workload, seeds 0..99."""
    for seed in range(100):
        inst = I.config_uniform(seed)
        _same(mhs.kernelize(inst, contraction=mode), O.reduce(inst), f"seed {seed}")


@pytest.mark.parametrize("mode", MODES)
def test_tiny_and_degenerate(mhs, mode):
    """Tiny instances with duplicate hyperedges, twin vertices and infeasible demands."""
    for seed in range(300):
        inst = I.tiny_random(seed, nmax=24, mmax=30)
        _same(mhs.kernelize(inst, contraction=mode), O.reduce(inst), f"seed {seed}")


@pytest.mark.parametrize("mode", MODES)
def test_edge_cases(mhs, mode):
    cases = [
        I.from_edges(0, [], []),
        I.from_edges(5, [], []),                      # no hyperedges: all vertices go
        I.from_edges(3, [[], [0]], [1, 1]),           # an empty (infeasible) hyperedge
        I.from_edges(1, [[0]], [1]),
        I.from_edges(300, [[i] for i in range(300)], [1] * 300),   # irreducible family
        I.from_edges(5, [[0, 1], [1, 2, 3], [1, 2, 4]], [2, 2, 2], k=3),  # Appendix A
        I.from_edges(4, [[0, 1, 2, 3]] * 5, [1, 2, 2, 1, 2]),    # equal hyperedges
        I.from_edges(6, [[0, 1, 2, 3, 4, 5]], [6]),    # a full hyperedge
    ]
    for c, inst in enumerate(cases):
        _same(mhs.kernelize(inst, contraction=mode), O.reduce(inst), f"case {c}")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,m", [(127, 129), (128, 256), (129, 257), (255, 383), (257, 640),
                                 (513, 1100), (700, 1500)])
def test_ragged_tile_boundaries(mhs, mode, n, m):
    """Sizes around the 64 / 128 / 256 tile edges, several tiles per side."""
    for seed in range(3):
        inst = I.uniform_random(n, m, 1, 12, 3, n // 10, 50_000 + 97 * n + seed)
        _same(mhs.kernelize(inst, contraction=mode), O.reduce(inst), f"seed {seed}")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,m", [(1024, 1024), (1025, 1024), (1000, 2049), (3073, 1023),
                                 (2048, 4100)])
def test_compaction_chunk_boundaries(mhs, mode, n, m):
    """A single instance compacts with one block per 1024 ids (a chained
    scan across blocks): id ranges on, just past and well past the chunk
    edges, with n and m on different sides of them, plus the round-by-round
    path, whose graphs launch the same kernels."""
    for seed in range(2):
        inst = I.uniform_random(n, m, 1, 10, 3, n // 8, 61_000 + 7 * n + m + seed)
        ref = O.reduce(inst)
        _same(mhs.kernelize(inst, contraction=mode), ref, f"seed {seed}")
    with mhs.Instance.load(inst, contraction=mode) as h:
        r = 0
        while True:
            st = h.reduce_round()
            r += 1
            ref = O.reduce(inst, max_rounds=r)
            _same(h.result(), ref, f"round {r}")
            if not ref["changed"]:
                assert st["changed"] == 0
                break


@pytest.mark.parametrize("mode", MODES)
def test_round_by_round(mhs, mode):
    """mhs_reduce_round after each round equals the oracle's state after as many rounds."""
    for seed in range(5):
        inst = I.uniform_random(400, 900, 1, 10, 3, 0, 70_000 + seed)
        with mhs.Instance.load(inst, contraction=mode) as h:
            r = 0
            while True:
                st = h.reduce_round()
                r += 1
                got = h.result()
                ref = O.reduce(inst, max_rounds=r)
                _same(got, ref, f"seed {seed} round {r}")
                if not ref["changed"]:
                    assert st["changed"] == 0
                    break
                assert st["changed"] == 1


@pytest.mark.parametrize("mode", MODES)
def test_powerlaw_full_size(mhs, mode):
    """n=20,000, m=40,000, power-law sizes, Zipf(1.1) vertices, bit-exact."""
    inst = I.config_powerlaw(0)
    _same(mhs.kernelize(inst, contraction=mode), O.reduce(inst))


@pytest.mark.parametrize("mode", MODES)
def test_interval_full_size(mhs, mode):
    """n=50,000, m=100,000 interval hyperedges with noise, bit-exact."""
    inst = I.config_interval(0)
    _same(mhs.kernelize(inst, contraction=mode), O.reduce(inst))


def test_fp8_and_popcount_agree_on_medium(mhs):
    for seed in range(4):
        inst = I.config_powerlaw(seed, n=3000, m=6000)
        a = mhs.kernelize(inst, contraction="fp8")
        b = mhs.kernelize(inst, contraction="popcount")
        for key in ("vertices", "edges", "rounds"):
            assert np.array_equal(a[key], b[key])


def test_groups_beyond_the_sector_table(mhs):
    """Hyperedges of 30-60 vertices: a group of 32 rows holds more incidences
    than the operand passes' shared-memory table (512), so those groups set
    their bytes with atomics instead; mixed with groups that use the table
    (sizes 2-6), and with a few dominated hyperedges so that rounds go on."""
    big = I.uniform_random(1500, 900, 30, 60, 3, 150, seed=31)
    mixed = I.uniform_random(1200, 1600, 2, 6, 2, 120, seed=32)
    edges = big.edges() + [e[:3] for e in big.edges()[:64]] + mixed.edges()
    dem = np.concatenate([big.demand, np.ones(64, np.int32), mixed.demand]).tolist()
    inst = I.from_edges(1500, edges, dem, k=150)
    assert max(len(e) for e in edges) >= 30 and inst.nnz > 40_000
    ref = O.reduce(inst)
    _same(mhs.kernelize(inst, contraction="fp8"), ref, "fp8 sector table overflow")
    _same(mhs.kernelize(inst, contraction="fp8", layout="input"), ref, "input layout")


def test_large_counts_exact(mhs):
    """Counts up to 2^20 stay exact with E4M3 0/1 operands and FP32 accumulation.

    Hyperedges {0, 1, a, b} over all pairs a < b of the other vertices, f = 1.
    Closed form under Algorithms 1-3: no DP deletion in round 1 (distinct
    hyperedges of equal size); MD deletes v1 (same hyperedges as v0, higher
    index) and every v_a (strictly dominated by v0 and v1) -- this needs the
    pair count I_01 = m to equal deg(v1) = m exactly; round 2 keeps the first
    of the now identical hyperedges {0}; round 3 changes nothing.
    """
    nb = 1450
    pairs = np.array([(a, b) for a in range(2, nb + 2) for b in range(a + 1, nb + 2)],
                     dtype=np.int32)[: (1 << 20) + 5]
    m = pairs.shape[0]
    vtx = np.empty((m, 4), np.int32)
    vtx[:, 0] = 0
    vtx[:, 1] = 1
    vtx[:, 2:] = pairs
    inst = I.Instance(n=nb + 2, m=m, edge_ptr=np.arange(0, 4 * m + 1, 4, dtype=np.int32),
                      edge_vtx=vtx.reshape(-1), demand=np.ones(m, np.int32), k=1)
    for mode in MODES:
        r = mhs.kernelize(inst, contraction=mode)
        assert r["vertices"].tolist() == [0], mode
        assert r["edges"].tolist() == [0], mode
        assert r["rounds"] == 3, mode


def test_batch_matches_single(mhs):
    """A batch of uneven instances reduced together equals each reduced alone
    and the oracle."""
    insts = [I.config_batch_one(4000 + i) for i in range(24)]
    insts += [I.from_edges(0, [], []), I.from_edges(3, [], []), I.tiny_random(5)]
    for mode in MODES:
        with mhs.Instance.load_batch(insts, contraction=mode) as h:
            assert h.count == len(insts)
            h.kernelize()
            for b, inst in enumerate(insts):
                _same(h.result(b), O.reduce(inst), f"{mode} instance {b}")


def test_load_device_and_masks(mhs):
    import torch
    inst = I.config_uniform(3)
    dev = torch.device("cuda:0")
    ptr = torch.from_numpy(inst.edge_ptr).to(dev)
    vtx = torch.from_numpy(inst.edge_vtx).to(dev)
    dem = torch.from_numpy(inst.demand).to(dev)
    ref = O.reduce(inst)
    for mode in MODES:
        with mhs.Instance.load_device(inst.n, inst.m, ptr, vtx, dem, inst.k, contraction=mode) as h:
            h.kernelize()
            _same(h.result(), ref, mode)
            av = torch.zeros(inst.n, dtype=torch.uint8, device=dev)
            ae = torch.zeros(inst.m, dtype=torch.uint8, device=dev)
            h.result_device(av, ae)
            torch.cuda.synchronize()
            assert np.nonzero(av.cpu().numpy())[0].tolist() == ref["vertices"].tolist()
            assert np.nonzero(ae.cpu().numpy())[0].tolist() == ref["edges"].tolist()


def test_export_and_resume(mhs):
    """A post-round state re-loaded through mhs_export reaches the same fixpoint."""
    inst = I.config_uniform(7, n=300, m=700)
    full = O.reduce(inst)
    with mhs.Instance.load(inst) as h:
        h.reduce_round()
        n, ptr, vtx, dem = h.export()
        part = h.result()
    sub = I.Instance(n=n, m=len(dem), edge_ptr=ptr, edge_vtx=vtx, demand=dem, k=inst.k)
    res = mhs.kernelize(sub)
    # map renumbered ids back
    assert part["vertices"][res["vertices"]].tolist() == full["vertices"].tolist()
    assert part["edges"][res["edges"]].tolist() == full["edges"].tolist()
    assert res["rounds"] + 1 == full["rounds"] or (res["rounds"] == 1 and full["rounds"] == 1)


def test_invalid_inputs_rejected(mhs):
    import torch
    bad = [
        I.Instance(n=3, m=1, edge_ptr=np.array([0, 2], np.int32),
                   edge_vtx=np.array([0, 3], np.int32), demand=np.array([1], np.int32), k=0),
        I.Instance(n=3, m=1, edge_ptr=np.array([0, 2], np.int32),
                   edge_vtx=np.array([1, 1], np.int32), demand=np.array([1], np.int32), k=0),
        I.Instance(n=3, m=1, edge_ptr=np.array([0, 2], np.int32),
                   edge_vtx=np.array([0, 1], np.int32), demand=np.array([0], np.int32), k=0),
    ]
    for inst in bad:
        with pytest.raises(mhs.MhsError) as ei:
            mhs.Instance.load(inst)
        assert ei.value.status == mhs.MHS_EINVAL
    dev = torch.device("cuda:0")
    inst = bad[0]
    with pytest.raises(mhs.MhsError) as ei:
        mhs.Instance.load_device(3, 1, torch.from_numpy(inst.edge_ptr).to(dev),
                                 torch.from_numpy(inst.edge_vtx).to(dev),
                                 torch.from_numpy(inst.demand).to(dev), 0)
    assert ei.value.status == mhs.MHS_EINVAL


def test_invalid_large_instance_rejected(mhs):
    """Above 128k incidences the host checks run on several threads while the
    inputs are copied to the device; an error anywhere is still found, with
    the single-threaded check's message, and a valid load afterwards works."""
    base = I.config_powerlaw(0)  # 160k incidences
    assert base.nnz >= 1 << 17

    def variant(edit):
        ptr, vtx, dem = base.edge_ptr.copy(), base.edge_vtx.copy(), base.demand.copy()
        edit(ptr, vtx, dem)
        return I.Instance(n=base.n, m=base.m, edge_ptr=ptr, edge_vtx=vtx, demand=dem, k=base.k)

    last = int(base.m) - 1
    wide = next(e for e in range(last, 0, -1) if base.edge_ptr[e + 1] - base.edge_ptr[e] >= 2)

    def dup(ptr, vtx, dem):
        vtx[ptr[wide] + 1] = vtx[ptr[wide]]

    def decrease(ptr, vtx, dem):  # hyperedge m/2 ends before it starts (the first error)
        ptr[base.m // 2 + 1] = ptr[base.m // 2] - 1

    cases = [(lambda p, v, d: v.__setitem__(-1, base.n), "outside"),
             (dup, "twice"),
             (lambda p, v, d: d.__setitem__(last, 0), "demand"),
             (decrease, "decreases")]
    for edit, frag in cases:
        with pytest.raises(mhs.MhsError) as ei:
            mhs.Instance.load(variant(edit), contraction="fp8")
        assert ei.value.status == mhs.MHS_EINVAL and frag in str(ei.value), str(ei.value)
    with mhs.Instance.load(base, contraction="fp8") as h:
        st = h.kernelize()
    assert st["rounds"] >= 2 and st["m_alive"] < base.m


def test_deterministic_repeats(mhs):
    inst = I.config_powerlaw(1, n=4000, m=8000)
    first = mhs.kernelize(inst)
    for _ in range(5):
        again = mhs.kernelize(inst)
        for key in ("vertices", "edges", "rounds"):
            assert np.array_equal(first[key], again[key])


def _concat(insts):
    nnz = np.array([i.nnz for i in insts], np.int64)
    base = np.concatenate([[0], np.cumsum(nnz)])
    m_tot = sum(i.m for i in insts)
    ptr = np.zeros(m_tot + 1, np.int64)
    e0 = 0
    for b, i in enumerate(insts):
        ptr[e0:e0 + i.m + 1] = i.edge_ptr.astype(np.int64) + base[b]
        e0 += i.m
    vtx = np.concatenate([i.edge_vtx for i in insts] + [np.zeros(1, np.int32)])
    dem = np.concatenate([i.demand for i in insts] + [np.zeros(1, np.int32)])
    return ptr, vtx, dem


def _oracle_trace_rows(inst):
    """(hyperedges into DP, vertices into DP, hyperedges after DP) per round,
    from the oracle's per-round deletion counts."""
    _, _, _, _, tr = O.reduce_state(inst, trace_cap=64)
    rows, m, n = [], inst.m, inst.n
    for de, dv, am, an in tr.tolist():
        rows.append([m, n, m - de])
        m, n = am, an
    return rows


def test_batch_device_load_masks_and_trace(mhs):
    import torch
    insts = [I.config_batch_one(4100 + i) for i in range(20)]
    insts += [I.from_edges(0, [], []), I.tiny_random(7), I.from_edges(4, [], [])]
    ptr, vtx, dem = _concat(insts)
    dev = torch.device("cuda:0")
    n = np.array([i.n for i in insts], np.int32)
    m = np.array([i.m for i in insts], np.int32)
    k = np.array([i.k for i in insts], np.int64)
    tp, tv, td = (torch.from_numpy(x).to(dev) for x in (ptr, vtx, dem))
    refs = [O.reduce(i) for i in insts]
    for mode in MODES:
        with mhs.Instance.load_batch_device(n, m, k, tp, tv, td, contraction=mode) as h:
            h.kernelize()
            av = torch.zeros(int(n.sum()) + 1, dtype=torch.uint8, device=dev)
            ae = torch.zeros(int(m.sum()) + 1, dtype=torch.uint8, device=dev)
            h.result_batch_device(av, ae)
            av, ae = av.cpu().numpy(), ae.cpu().numpy()
            vb = eb = 0
            for b, inst in enumerate(insts):
                ref = refs[b]
                _same(h.result(b), ref, f"{mode} instance {b}")
                assert np.nonzero(av[vb:vb + inst.n])[0].tolist() == ref["vertices"].tolist()
                assert np.nonzero(ae[eb:eb + inst.m])[0].tolist() == ref["edges"].tolist()
                vb += inst.n
                eb += inst.m
                rows, rounds = h.trace(b)
                assert rounds == ref["rounds"]
                assert rows.tolist() == _oracle_trace_rows(inst)[:32], (mode, b)


def test_batch_device_rejects_malformed(mhs):
    import torch
    insts = [I.config_batch_one(4200 + i) for i in range(5)]
    insts[3].demand[2] = 0  # demand < 1 in instance 3
    ptr, vtx, dem = _concat(insts)
    dev = torch.device("cuda:0")
    n = np.array([i.n for i in insts], np.int32)
    m = np.array([i.m for i in insts], np.int32)
    k = np.array([i.k for i in insts], np.int64)
    tp, tv, td = (torch.from_numpy(x).to(dev) for x in (ptr, vtx, dem))
    with pytest.raises(mhs.MhsError) as ei:
        mhs.Instance.load_batch_device(n, m, k, tp, tv, td)
    assert ei.value.status == mhs.MHS_EINVAL and "instance 3" in str(ei.value)
    insts[3].demand[2] = 1
    insts[1].edge_vtx[5] = insts[1].n  # vertex id out of range in instance 1
    ptr, vtx, dem = _concat(insts)
    tp, tv, td = (torch.from_numpy(x).to(dev) for x in (ptr, vtx, dem))
    with pytest.raises(mhs.MhsError) as ei:
        mhs.Instance.load_batch_device(n, m, k, tp, tv, td)
    assert "instance 1" in str(ei.value)


def test_bounded_wait_times_out_and_context_survives(mhs):
    """A wait that nothing satisfies ends after its limit with the timeout
    status; the context then still runs a full kernelization."""
    status, waited = mhs.selftest_bounded_wait(20_000_000)
    assert status == 4
    assert 20_000_000 <= waited < 2_000_000_000
    inst = I.config_uniform(11)
    _same(mhs.kernelize(inst), O.reduce(inst), "after timeout")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("layout", ["input", "sorted", "degree"])
def test_layouts_and_tie_breaks(mhs, mode, layout):
    """Rows in input order, hyperedges sorted by smallest vertex, or vertices
    grouped by degree class: the lowest-index tie-breaks compare input ids,
    so the result is the same either way.  Tiny instances carry duplicate
    hyperedges and twin vertices; the power-law ones skewed degrees."""
    for seed in range(300):
        inst = I.tiny_random(seed, nmax=24, mmax=30)
        _same(mhs.kernelize(inst, contraction=mode, layout=layout), O.reduce(inst),
              f"{layout} seed {seed}")
    for seed in range(3):
        inst = I.config_interval(seed, n=3000, m=6000)
        _same(mhs.kernelize(inst, contraction=mode, layout=layout), O.reduce(inst),
              f"{layout} interval {seed}")
        inst = I.config_powerlaw(seed, n=3000, m=6000)
        _same(mhs.kernelize(inst, contraction=mode, layout=layout), O.reduce(inst),
              f"{layout} powerlaw {seed}")


@pytest.mark.parametrize("sparsity", ["skip", "dense"])
def test_zero_tiles_with_loose_hyperedge(mhs, sparsity):
    """A hyperedge with f > |e| supersedes hyperedges it shares no vertex
    with (count 0): tiles with no shared K block must still be tested in DP
    then.  e_0 = {0} with f = 3 pushes 3 - 1 = 2 units of demand to every
    other hyperedge, so every hyperedge with f <= 2 goes."""
    rng = np.random.default_rng(5)
    n, m = 1200, 2500
    edges = [[0]] + [sorted(rng.choice(np.arange(300, n), size=int(rng.integers(2, 9)),
                                       replace=False).tolist()) for _ in range(m - 1)]
    dem = [3] + [int(rng.integers(1, 4)) for _ in range(m - 1)]
    inst = I.from_edges(n, edges, dem)
    ref = O.reduce(inst)
    for mode in MODES:
        _same(mhs.kernelize(inst, contraction=mode, sparsity=sparsity), ref, f"{mode} {sparsity}")
    # and a feasible instance whose blocks are mostly disjoint (interval layout)
    inst = I.config_interval(4, n=6000, m=12000)
    _same(mhs.kernelize(inst, sparsity=sparsity), O.reduce(inst), f"interval {sparsity}")


def test_skip_and_dense_agree_and_skip_does_less(mhs):
    inst = I.config_interval(1, n=8000, m=16000)
    with mhs.Instance.load(inst, contraction="fp8", sparsity="dense") as h:
        h.kernelize()
        dense = h.result()
        kb_dense, t_dense = h.work_stats()
    with mhs.Instance.load(inst, contraction="fp8", sparsity="skip") as h:
        h.kernelize()
        skip = h.result()
        kb_skip, t_skip = h.work_stats()
    for key in ("vertices", "edges", "demands", "rounds"):
        assert np.array_equal(np.asarray(dense[key]), np.asarray(skip[key]))
    assert 0 < kb_skip < kb_dense and 0 < t_skip <= t_dense


def test_reused_operand_regions(mhs):
    """Dense operand regions return to a zero-state cache when an instance is
    freed and are reused by later loads without a memset: results must not
    depend on what used the region before (full runs, runs stopped after one
    round, other sizes, both contractions)."""
    insts = [I.config_powerlaw(7, n=3000, m=6000), I.config_uniform(12),
             I.config_interval(3, n=3000, m=6000)]
    refs = [O.reduce(i) for i in insts]
    for rep in range(3):
        for inst, ref in zip(insts, refs):
            _same(mhs.kernelize(inst, contraction="fp8"), ref, f"rep {rep}")
            with mhs.Instance.load(inst, contraction="fp8") as h:
                h.reduce_round()  # freed between rounds
            with mhs.Instance.load(inst, contraction="fp8", full_edges=True) as h:
                h.kernelize()
            _same(mhs.kernelize(inst, contraction="popcount"), ref, f"rep {rep} popcount")


@pytest.mark.parametrize("graphs", [True, False])
@pytest.mark.parametrize("mode", MODES)
def test_timing_mode(mhs, graphs, mode):
    """Per-phase CUDA-event timing (mhs_set_timing) works with captured
    per-round graphs and with direct launches, and does not change results."""
    inst = I.config_powerlaw(3, n=3000, m=6000)
    with mhs.Instance.load(inst, contraction=mode, use_graphs=graphs) as h:
        h.set_timing(True)
        h.kernelize()
        t = h.last_timing()
        _same(h.result(), O.reduce(inst), f"graphs={graphs}")
    assert t["dp_ms"] > 0 and t["md_ms"] > 0 and t["other_ms"] >= 0
    assert t["total_ms"] >= t["dp_ms"] + t["md_ms"] - 1e-3


def _oracle_alive(seed):
    """Worker: the oracle's result of batch instance `seed` as alive masks
    over its input ids, with k and the round count."""
    from oracle import oracle as O2
    from paper_2109_06042_gb300 import instances as I2
    inst = I2.config_batch_one(seed)
    r = O2.reduce(inst)
    av = np.zeros(inst.n, np.uint8)
    ae = np.zeros(inst.m, np.uint8)
    av[r["vertices"]] = 1
    ae[r["edges"]] = 1
    return av, ae, r["rounds"]


def test_full_batch_4096_every_instance(mhs):
    """The whole 4,096-instance batch the benchmark times (seeds 4000..4095),
    loaded the same way (device CSR arrays, one batch), reduced in one
    fixpoint launch; every instance's surviving vertex and hyperedge sets and
    round count equal the oracle's.  The oracle runs in a pool of spawned
    processes."""
    import multiprocessing as mp
    import os
    import torch
    count, seed0 = 4096, 4000
    insts = I.config_batch(count, seed0)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        ref_async = pool.map_async(_oracle_alive, [seed0 + b for b in range(count)], chunksize=16)
        dev = torch.device("cuda", 0)
        n = np.array([i.n for i in insts], np.int32)
        m = np.array([i.m for i in insts], np.int32)
        k = np.array([i.k for i in insts], np.int64)
        nnz = np.array([i.nnz for i in insts], np.int64)
        base = np.concatenate([[0], np.cumsum(nnz)])
        ptr = np.zeros(int(m.sum()) + 1, np.int64)
        e0 = 0
        for b, i in enumerate(insts):
            ptr[e0:e0 + i.m + 1] = i.edge_ptr.astype(np.int64) + base[b]
            e0 += i.m
        vtx = np.concatenate([i.edge_vtx for i in insts] + [np.zeros(1, np.int32)])
        dem = np.concatenate([i.demand for i in insts] + [np.zeros(1, np.int32)])
        av = torch.zeros(int(n.sum()) + 1, dtype=torch.uint8, device=dev)
        ae = torch.zeros(int(m.sum()) + 1, dtype=torch.uint8, device=dev)
        with mhs.Instance.load_batch_device(n, m, k, torch.from_numpy(ptr).to(dev),
                                            torch.from_numpy(vtx).to(dev),
                                            torch.from_numpy(dem).to(dev),
                                            contraction="fp8") as h:
            h.kernelize()
            h.result_batch_device(av, ae)
            torch.cuda.synchronize()
            rounds = [h.trace(b)[1] for b in range(count)]
        av = av.cpu().numpy()
        ae = ae.cpu().numpy()
        refs = ref_async.get(timeout=1800)
    vb = np.concatenate([[0], np.cumsum(n)])
    eb = np.concatenate([[0], np.cumsum(m)])
    for b, (rav, rae, rr) in enumerate(refs):
        assert np.array_equal(av[vb[b]:vb[b + 1]], rav), f"instance {b}: vertices"
        assert np.array_equal(ae[eb[b]:eb[b + 1]], rae), f"instance {b}: hyperedges"
        assert rounds[b] == rr, f"instance {b}: rounds {rounds[b]} != {rr}"

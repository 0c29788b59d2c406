"""Sharded passes (mhs_pass_*): one pass of Algorithm 3 split by tile rows.

Every share of a pass contracts the tile rows of its own 128-row blocks;
the pass's output is the OR of the shares' deletion flags (DP, SE) or the
sum of their dominator counts (MD).  Two checks on one GPU:
* one handle runs every share in a row (the in-place OR / sum is the
  merge): G = 1, 2, 3, 8 must all give the oracle's result;
* G replicas of the instance, each contracting only its own share, with
  the exchange done between them (element-wise maximum of the flags, sum
  of the counts, as an all-reduce would): every replica ends with the
  oracle's result, round for round in step.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_06042_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2109_06042_gb300 import build
    build.build()
    from paper_2109_06042_gb300 import mhs
    return torch, mhs


def _same(got, ref, ctx):
    for key in ("vertices", "edges", "demands"):
        assert got[key].tolist() == ref[key].tolist(), f"{key} differ {ctx}"
    assert got["k"] == ref["k"] and got["rounds"] == ref["rounds"], ctx


def _cases():
    return [I.config_uniform(5), I.uniform_random(700, 1500, 1, 8, 4, 70, 93_000),
            I.config_powerlaw(4, n=3000, m=6000), I.config_interval(4, n=3000, m=6000)]


@pytest.mark.parametrize("mode", ["fp8", "popcount"])
@pytest.mark.parametrize("g", [1, 2, 3, 8])
def test_all_shares_in_a_row(env, mode, g):
    torch, mhs = env
    for inst in _cases():
        ref = O.reduce(inst)
        with mhs.Instance.load(inst, contraction=mode, use_graphs=False) as h:
            while True:
                for phase in (0, 1):
                    h.pass_begin(phase)
                    for sh in range(g):
                        h.pass_contract(phase, sh, g)
                    st = h.pass_end(phase)
                if not st["active"]:
                    break
            _same(h.result(), ref, f"{inst.name} {mode} G={g}")


def _replicas_round(torch, handles, dev):
    g = len(handles)
    st = None
    for phase in (0, 1):
        for h in handles:
            h.pass_begin(phase)
        parts = []
        for sh, h in enumerate(handles):
            h.pass_contract(phase, sh, g)
            n = h.pass_elems(phase)
            buf = torch.zeros(max(n, 1), dtype=torch.uint8 if phase == 0 else torch.int32,
                              device=dev)
            torch.cuda.synchronize()  # the library copies on its own stream
            h.pass_partial(phase, buf)
            parts.append(buf)
        merged = torch.stack(parts)
        merged = merged.max(0).values if phase == 0 else merged.sum(0, dtype=torch.int32)
        merged = merged.contiguous()
        torch.cuda.synchronize()
        for h in handles:
            h.pass_merge(phase, merged)
        stats = [h.pass_end(phase) for h in handles]
        assert all(s == stats[0] for s in stats), stats  # the replicas stay in step
        st = stats[0]
    return st


@pytest.mark.parametrize("mode", ["fp8", "popcount"])
@pytest.mark.parametrize("g", [2, 3])
def test_replicas_exchange_partials(env, mode, g):
    torch, mhs = env
    dev = torch.device("cuda", 0)
    for inst in _cases():
        ref = O.reduce(inst)
        handles = [mhs.Instance.load(inst, contraction=mode, use_graphs=False) for _ in range(g)]
        try:
            while _replicas_round(torch, handles, dev)["active"]:
                pass
            for r, h in enumerate(handles):
                _same(h.result(), ref, f"{inst.name} {mode} G={g} replica {r}")
        finally:
            for h in handles:
                h.free()


@pytest.mark.parametrize("rule,fe", [("se", False), ("dp", True), ("se", True)])
def test_replicas_with_variants(env, rule, fe):
    torch, mhs = env
    dev = torch.device("cuda", 0)
    inst = I.config_powerlaw(6, n=2000, m=4000)
    ref = O.reduce_variant(inst, rule, fe)
    handles = [mhs.Instance.load(inst, contraction="fp8", use_graphs=False, rule=rule,
                                 full_edges=fe) for _ in range(3)]
    try:
        while _replicas_round(torch, handles, dev)["active"]:
            pass
        for h in handles:
            got = h.result()
            _same(got, ref, f"{rule} fe={fe}")
    finally:
        for h in handles:
            h.free()


def test_glue_single_replica(env):
    """shard.kernelize_sharded with one replica (no exchange) and with the
    exchange functions applied to a single replica's buffers."""
    torch, mhs = env
    from paper_2109_06042_gb300 import shard
    dev = torch.device("cuda", 0)
    inst = I.config_powerlaw(8, n=2500, m=5000)
    ref = O.reduce(inst)
    ident = lambda t: t
    with mhs.Instance.load(inst, contraction="fp8", use_graphs=False) as h:
        st = shard.kernelize_sharded(h, 0, 1, ident, ident, shard.torch_buffers(torch, dev),
                                     sync=shard.torch_sync(torch, dev))
        assert st["active"] == 0
        _same(h.result(), ref, "glue G=1")


def test_pass_order_is_enforced(env):
    torch, mhs = env
    inst = I.config_uniform(6)
    with mhs.Instance.load(inst, contraction="fp8", use_graphs=False) as h:
        for bad in (lambda: h.pass_contract(0, 0, 1), lambda: h.pass_end(0),
                    lambda: h.pass_begin(1)):
            with pytest.raises(mhs.MhsError) as ei:
                bad()
            assert ei.value.status == mhs.MHS_EINVAL
        h.pass_begin(0)
        with pytest.raises(mhs.MhsError):
            h.kernelize()  # a sharded round is open
        with pytest.raises(mhs.MhsError):
            h.pass_contract(0, 2, 2)  # shard out of range
        h.pass_contract(0, 0, 1)
        h.pass_end(0)
        h.pass_begin(1)
        h.pass_contract(1, 0, 1)
        h.pass_end(1)
        h.kernelize()  # the rest of the rounds, as usual
        _same(h.result(), O.reduce(inst), "after one sharded round")

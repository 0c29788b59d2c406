"""The two properties of Algorithm 3 that let a round leave out a pass's
operand (the passes without a candidate), checked on the oracle's per-round
trace over random instances: after the first round,

* a DP pass deletes nothing when the previous round's MD pass deleted no
  vertex (no hyperedge lost a vertex, so every pair's test gives the
  previous DP pass's answer, which deleted neither);
* an MD pass deletes nothing when the same round's DP pass deleted no
  hyperedge (no vertex lost a hyperedge: its maximum demand is unchanged and
  its dominator count can only have dropped).

These hold for the DP + MD rounds (FE, which changes demands, marks every
item a candidate again and is not part of this trace).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_06042_gb300 import instances as I


def _instances():
    out = [I.tiny_random(s, nmax=16, mmax=14) for s in range(120)]
    out += [I.config_uniform(s, n=60, m=120) for s in range(40)]
    out += [I.uniform_random(80, 160, 2, 6, 3, 8, seed=500 + s) for s in range(40)]
    return out


@pytest.mark.parametrize("chunk", range(4))
def test_passes_without_candidates_delete_nothing(chunk):
    insts = _instances()[chunk::4]
    checked = 0
    for idx, inst in enumerate(insts):
        _, _, rounds, _, trace = O.reduce_state(inst, trace_cap=64)
        dp = trace[:, 0].tolist()
        md = trace[:, 1].tolist()
        for r in range(1, len(dp)):
            if md[r - 1] == 0:
                assert dp[r] == 0, (chunk, idx, r, dp, md)
                checked += 1
            if dp[r] == 0:
                assert md[r] == 0, (chunk, idx, r, dp, md)
                checked += 1
    assert checked > 0


def test_the_trace_is_the_round_by_round_passes():
    """The trace's deletion counts are those of the single passes (so the
    properties above are checked on what the rounds do)."""
    inst = I.config_uniform(3, n=60, m=120)
    _, _, rounds, _, trace = O.reduce_state(inst, trace_cap=64)
    av = np.ones(inst.n, bool)
    ae = np.ones(inst.m, bool)
    for r in range(rounds):
        de = O.dp_pass(inst, av, ae)
        ae = ae & ~de
        dv, _, _ = O.md_pass(inst, av, ae)
        av = av & ~dv
        assert (int(de.sum()), int(dv.sum())) == (int(trace[r, 0]), int(trace[r, 1])), r

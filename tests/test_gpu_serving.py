"""The continuous-batching server (mhs_server_*).

Every served result must equal the oracle's and the result of the same
instance reduced alone (bit-exact), whatever else is in flight; admission
respects the HBM budget; queue limits, early polls, oversize requests and
shutdown with work pending behave as the C ABI documents.
"""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_06042_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mhs():
    from paper_2109_06042_gb300 import build
    build.build()
    from paper_2109_06042_gb300 import mhs as M
    return M


def _mix():
    insts = [I.config_batch_one(9000 + i) for i in range(24)]
    insts += [I.config_uniform(s) for s in range(6)]
    insts += [I.config_powerlaw(s, n=2500, m=5000) for s in range(2)]
    insts += [I.from_edges(0, [], []), I.from_edges(6, [], []), I.tiny_random(3),
              I.from_edges(5, [[0, 1], [1, 2, 3], [1, 2, 4]], [2, 2, 2], k=3)]
    return insts


def _poll_all(srv, tickets, seconds=120.0):
    """Poll every ticket against one overall deadline (fails instead of stalling)."""
    deadline = time.monotonic() + seconds
    out = []
    for t in tickets:
        left = max(0.0, deadline - time.monotonic())
        r = srv.poll(t, timeout_us=int(left * 1e6))
        assert r is not None, f"ticket {t} not finished within {seconds} s"
        out.append(r)
    return out


def _same(a, b, ctx):
    for key in ("vertices", "edges", "demands"):
        assert a[key].tolist() == b[key].tolist(), (key, ctx)
    assert a["k"] == b["k"] and a["rounds"] == b["rounds"], ctx


@pytest.mark.parametrize("mode,small_items", [("fp8", 0), ("popcount", 0), ("fp8", -1),
                                              ("fp8", 1)])
def test_served_equals_alone_and_oracle(mhs, mode, small_items):
    """Both lanes (default split), a single lane (-1), and everything in the
    large-request lane (1)."""
    insts = _mix()
    with mhs.Server(max_slots=16, contraction=mode, small_items=small_items) as srv:
        tickets = [srv.submit(i) for i in insts]
        results = _poll_all(srv, tickets)
        st = srv.stats()
    assert st["completed"] == len(insts) and st["pending"] == 0 and st["active"] == 0
    for idx, (inst, res) in enumerate(zip(insts, results)):
        assert res is not None
        _same(res, O.reduce(inst), f"oracle {idx}")
        _same(res, mhs.kernelize(inst, contraction=mode), f"alone {idx}")


def test_admission_by_footprint(mhs):
    insts = [I.config_batch_one(9100 + i) for i in range(12)]
    with mhs.Server(max_slots=64) as probe:
        pass
    # a budget that holds about two of these instances at a time
    big = max(i.m * i.n for i in insts)
    budget = 2 * (3 * big + 16 * (max(i.m for i in insts) + max(i.n for i in insts)) + (1 << 20))
    with mhs.Server(hbm_budget_bytes=budget, max_slots=64) as srv:
        tickets = [srv.submit(i) for i in insts]
        results = _poll_all(srv, tickets)
        st = srv.stats()
    assert st["peak_bytes"] <= budget
    for inst, res in zip(insts, results):
        _same(res, O.reduce(inst), inst.name)


def test_queue_full_and_early_poll(mhs):
    insts = [I.config_uniform(s) for s in range(4)]
    with mhs.Server(max_slots=4, queue_capacity=3) as srv:
        srv.pause(True)
        tickets = [srv.submit(i) for i in insts[:3]]
        with pytest.raises(mhs.MhsError) as ei:
            srv.submit(insts[3])
        assert ei.value.status == mhs.MHS_EBUSY
        assert srv.poll(tickets[0], timeout_us=0) is None          # not started
        assert srv.poll(tickets[0], timeout_us=20_000) is None      # paused: still waiting
        assert srv.stats()["pending"] == 3
        srv.pause(False)
        for r, inst in zip(_poll_all(srv, tickets), insts):
            _same(r, O.reduce(inst), inst.name)
        with pytest.raises(mhs.MhsError):
            srv.poll(tickets[0])                                     # already consumed


def test_oversize_request_rejected(mhs):
    with mhs.Server(hbm_budget_bytes=1 << 20) as srv:
        with pytest.raises(mhs.MhsError) as ei:
            srv.submit(I.config_powerlaw(0, n=3000, m=6000))
        assert ei.value.status == mhs.MHS_ENOMEM
        res = _poll_all(srv, [srv.submit(I.config_uniform(0, n=40, m=60))])[0]
        _same(res, O.reduce(I.config_uniform(0, n=40, m=60)), "small fits")


def test_destroy_with_pending_work(mhs):
    srv = mhs.Server(max_slots=2)
    srv.pause(True)
    for s in range(5):
        srv.submit(I.config_uniform(s))
    srv.close()  # must not hang


def test_loop_restarts_and_admits_while_running(mhs):
    """The device-resident loop ends when no slot holds work and is started
    again by the next submission; requests submitted while rounds run are
    admitted at a round boundary of the running loop.  Every result equals
    the oracle's."""
    waves = [[I.config_batch_one(9100 + 10 * w + i) for i in range(6)] for w in range(3)]
    with mhs.Server(max_slots=8) as srv:
        done = []
        for w, wave in enumerate(waves):  # each wave finishes: the loop goes idle
            tickets = [srv.submit(i) for i in wave]
            done.append((wave, _poll_all(srv, tickets)))
            time.sleep(0.05)
        rounds_idle = srv.stats()["rounds"]
        # staggered submissions into a loop that is running
        stag = [I.config_batch_one(9200 + i) for i in range(12)] + \
               [I.config_powerlaw(7, n=2500, m=5000)]
        tickets = []
        for inst in stag:
            tickets.append(srv.submit(inst))
            time.sleep(0.002)
        done.append((stag, _poll_all(srv, tickets)))
        st = srv.stats()
    assert rounds_idle > 0 and st["rounds"] > rounds_idle
    assert st["completed"] == sum(len(w) for w, _ in done) and st["active"] == 0
    for wave, results in done:
        for idx, (inst, res) in enumerate(zip(wave, results)):
            _same(res, O.reduce(inst), f"oracle {idx}")

"""The exchange glue of sharded passes (paper_2109_06042_gb300/shard.py) as
two gloo ranks on the CPU (127.0.0.1).  No GPU: each rank drives a stand-in
handle whose partial buffers depend on its rank, and the test checks that
every rank merges the element-wise maximum of the flags and the sum of the
counts, in pass order, and that both stop after the same round."""
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class FakeHandle:
    """Records the pass calls; round r's partials are rank-dependent."""

    def __init__(self, rank, m=7, n=5, rounds=3):
        self.rank, self.m, self.n, self.rounds = rank, m, n, rounds
        self.calls, self.merged, self.round = [], [], 0

    def pass_begin(self, phase):
        self.calls.append(("begin", phase))

    def pass_contract(self, phase, shard, nshards):
        self.calls.append(("contract", phase, shard, nshards))

    def pass_elems(self, phase):
        return self.m if phase == 0 else self.n

    def pass_partial(self, phase, buf):
        import torch
        k = torch.arange(buf.numel())
        if phase == 0:  # rank r flags positions with (k + r + round) % 3 == 0
            buf.copy_(((k + self.rank + self.round) % 3 == 0).to(torch.uint8))
        else:           # rank r counts k * (r + 1) + round
            buf.copy_((k * (self.rank + 1) + self.round).to(torch.int32))
        return buf.numel()

    def pass_merge(self, phase, buf):
        self.merged.append((phase, buf.clone()))

    def pass_end(self, phase):
        self.calls.append(("end", phase))
        if phase == 1:
            self.round += 1
        return {"active": int(self.round < self.rounds), "changed": 1, "rounds": self.round}


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2109_06042_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    h = FakeHandle(rank)
    rmax, rsum = shard.dist_exchange(dist)
    st = shard.kernelize_sharded(h, rank, world, rmax, rsum,
                                 shard.torch_buffers(torch, torch.device("cpu")))
    out.put((rank, st, h.calls, [(p, b.tolist()) for p, b in h.merged]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_exchange_max_and_sum():
    import torch
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, st0, calls0, merged0), (r1, st1, calls1, merged1) = res
    assert st0["active"] == st1["active"] == 0 and st0["rounds"] == st1["rounds"] == 3
    assert merged0 == merged1 and len(merged0) == 6  # 3 rounds x 2 passes
    k7, k5 = torch.arange(7), torch.arange(5)
    for i, (phase, buf) in enumerate(merged0):
        rnd = i // 2
        if phase == 0:
            want = (((k7 + 0 + rnd) % 3 == 0) | ((k7 + 1 + rnd) % 3 == 0)).to(torch.uint8)
        else:
            want = (k5 * 1 + rnd) + (k5 * 2 + rnd)
        assert buf == want.tolist(), (i, phase)
    for calls, shard_id in ((calls0, 0), (calls1, 1)):
        assert calls[:3] == [("begin", 0), ("contract", 0, shard_id, 2), ("end", 0)]
        assert calls[3:6] == [("begin", 1), ("contract", 1, shard_id, 2), ("end", 1)]

"""Sharded kernelization of one instance over several replicas.

Algorithm 3 (Section 4.1) tests every pair of a pass independently, so a
pass can be split by tile rows over replicas that each hold the whole
instance.  The only exchange per pass is its output: the DP (or SE) pass's
deletion flags, combined by element-wise maximum (a logical OR), and the MD
pass's dominator counts, combined by a sum.  Everything else -- encoding,
the decisions, the compaction -- is deterministic and runs identically on
every replica, so the replicas stay in step.

``kernelize_sharded`` runs the round loop for one replica; ``exchange`` is
the all-reduce it uses, given as two callables so that any transport fits:
``torch.distributed`` (NCCL on GPUs, gloo on CPU; see ``dist_exchange``) or,
for replicas that share one process, an in-process reduction.  Nothing here
reads another replica's memory: each replica copies its partial buffer out,
the reduction combines the copies, and the result is copied back.
"""
from __future__ import annotations


def dist_exchange(dist, group=None):
    """The exchange through torch.distributed: all_reduce with MAX for the
    flags and SUM for the counts (in place, on the buffer's device)."""
    def reduce_max(t):
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        return t

    def reduce_sum(t):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return t
    return reduce_max, reduce_sum


def sharded_round(handle, shard, nshards, reduce_max, reduce_sum, make_buffer, sync=None):
    """One round of Algorithm 3 on one replica; returns the round stats.

    handle      an object with the pass_* methods of mhs.Instance
    make_buffer make_buffer(phase, elems) -> a tensor the handle can fill:
                uint8 for phase 0, int32 for phase 1
    sync        called before the library reads or writes a buffer that other
                streams produced (the buffer's allocation, the reduction):
                the library works on its instance's own stream
    """
    stats = None
    for phase in (0, 1):
        handle.pass_begin(phase)
        handle.pass_contract(phase, shard, nshards)
        if nshards > 1:
            elems = handle.pass_elems(phase)
            if elems > 0:
                buf = make_buffer(phase, elems)
                if sync:
                    sync()
                handle.pass_partial(phase, buf)  # returns with the copy done
                buf = (reduce_max if phase == 0 else reduce_sum)(buf)
                if sync:
                    sync()
                handle.pass_merge(phase, buf)
        stats = handle.pass_end(phase)
    return stats


def kernelize_sharded(handle, shard, nshards, reduce_max, reduce_sum, make_buffer,
                      max_rounds=0, sync=None):
    """Rounds until the instance reaches its fixpoint (or max_rounds); the
    replicas must all run this with the same instance and options.  Returns
    the last round's stats (n_alive, m_alive, rounds, changed, active, ...)."""
    done = 0
    while True:
        stats = sharded_round(handle, shard, nshards, reduce_max, reduce_sum, make_buffer,
                              sync)
        done += 1
        if not stats["active"] or (max_rounds and done >= max_rounds):
            return stats


def torch_buffers(torch, device):
    """make_buffer for CUDA (or CPU) tensors on `device`."""
    def make(phase, elems):
        return torch.zeros(elems, dtype=torch.uint8 if phase == 0 else torch.int32,
                           device=device)
    return make


def torch_sync(torch, device):
    """sync for tensors on `device`: waits for the work queued on it."""
    if device.type == "cuda":
        return lambda: torch.cuda.synchronize(device)
    return None

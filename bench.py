#!/usr/bin/env python
"""Throughput of the exhaustive DP + MD kernelization (Algorithm 3) on GB300.

A step is the complete kernelization of one instance (repeated --reps
times, so that the timed region is long enough to sample the clocks), or
of one batch of instances, with the inputs (CSR arrays) already resident
in HBM:

* load from device arrays;
* every round of DP (Algorithm 1) and MD (Algorithm 2), with their
  contractions and compaction;
* the result masks written to device memory.

``value`` is reduced instances per second over all GPUs, on the power-law
20,000 x 40,000 instance (the headline).  The line also carries:

* pair tests per second;
* the roofline of the dominant kernel (the tcgen05 contraction): the
  tensor work it issues over its CUDA-event time, against the FP8 peak;
  beside it the dense formulation's ratio and the sparse intrinsic work;
* the CPU oracle timed on the host (bounded sample);
* an end-to-end figure through host buffers;
* the SM clocks seen;
* ``configs``: the other workloads on the same GPU -- uniform 200 x 400,
  interval 50,000 x 100,000, the batch of 4,096 uneven instances (with its
  autotuned and fixed tile shapes and the one-instance-per-launch loop),
  and a short serving sweep with measured latencies of the served and the
  plain one-at-a-time form under the same Poisson arrivals.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--workload all|powerlaw|uniform|interval|batch|stream] [--contraction fp8|popcount]
N > 1 runs under torchrun; each rank reduces its own instances, with no
data-path collective (weak scaling); the other workloads are measured at
N = 1 only.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reduced instances/s (exhaustive DP+MD kernelization)"
UNIT = "instances/s"
DATA = "synthetic (seeded generators with the shapes of the paper's workloads)"
DEFAULT_TILES = dict(tile_n=256, group_rows=16, half_stages=True)
# kernelizations per timed step of a single-instance workload
REPS = {"powerlaw": 16, "uniform": 64, "interval": 2, "batch": 1}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["all", "powerlaw", "uniform", "interval", "batch",
                                          "stream"], default="all",
                   help="all: the power-law headline plus the other workloads as sub-records")
    p.add_argument("--contraction", choices=["fp8", "popcount"], default="fp8")
    p.add_argument("--sparsity", choices=["skip", "dense"], default="skip",
                   help="tcgen05 block-sparse skipping (exact) or the dense formulation")
    p.add_argument("--rule", choices=["dp", "se"], default="dp",
                   help="hyperedge rule of each round: DP (Algorithm 1) or SE (MD+SE variant)")
    p.add_argument("--full-edges", action="store_true",
                   help="alternate with rule FE at every fixpoint (KernelGPU-FE variant)")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--reps", type=int, default=0,
                   help="kernelizations per timed step (0: per workload, see REPS)")
    p.add_argument("--batch-count", type=int, default=4096)
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="bound on the CPU oracle sample")
    p.add_argument("--sub-steps", type=int, default=10, help="timed steps of each sub-record")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-loop", action="store_true", help="batch: skip the per-instance loop")
    p.add_argument("--requests", type=int, default=1000, help="stream: requests per rate")
    p.add_argument("--pool", type=int, default=300, help="stream: distinct request instances")
    p.add_argument("--rates", type=str, default="0.25,0.5,1,1.5,2",
                   help="stream: arrival rates as multiples of the saturating rate")
    p.add_argument("--sub-requests", type=int, default=300,
                   help="all: requests per rate of the short serving sweep")
    p.add_argument("--sub-rates", type=str, default="0.5,1,2",
                   help="all: rates of the short serving sweep")
    return p.parse_args()


def headline_workload(args):
    return "powerlaw" if args.workload == "all" else args.workload


def make_instances(args, rank, workload=None):
    from paper_2109_06042_gb300 import instances as I
    workload = workload or headline_workload(args)
    if workload == "batch":
        seed0 = shard_seed0(args, rank, workload)
        insts = I.config_batch(args.batch_count, seed0)
        nn = sum(i.n for i in insts)
        mm = sum(i.m for i in insts)
        zz = sum(i.nnz for i in insts)
        desc = (f"batch of {len(insts)} uneven instances (n~U[50,2000], m~U[n,2n], "
                f"|e|~U[2,16]), sum n={nn} sum m={mm} nnz={zz} seeds {seed0}..{seed0 + len(insts) - 1}")
        return insts, desc
    seed = shard_seed0(args, rank, workload)
    f = {"powerlaw": I.config_powerlaw, "uniform": I.config_uniform,
         "interval": I.config_interval}[workload]
    inst = f(seed)
    desc = f"{workload} n={inst.n} m={inst.m} nnz={inst.nnz} seed={seed}"
    return [inst], desc


def shard_seed0(args, rank, workload=None):
    """First seed of this rank's instances: ranks reduce disjoint instances."""
    if (workload or headline_workload(args)) == "batch":
        return 4000 + rank * args.batch_count
    return args.seed + rank


def max_over_ranks(x, dist, device):
    """Max of a float over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_step, steps, ms_max):
    """Units (instances) all ranks processed per second of the slowest rank."""
    return world * units_per_step * steps / (ms_max / 1e3)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms from before
    the warm-up (so that the sampler is running when the timed region
    starts); only samples whose own timestamp falls inside the timed window
    are kept, or, for a window shorter than the interval, the ones nearest
    to it."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []  # (host receive time, line)
        self.proc = None
        self.thread = None
        self.window = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, t0, t1):
        """The timed window, in host time.time() seconds."""
        self.window = (t0, t1)

    @staticmethod
    def _stamp(text, fallback):
        try:
            return datetime.datetime.strptime(text, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return fallback

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        rows = []
        for recv, ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append((self._stamp(parts[0], recv), float(parts[2]), float(parts[3]),
                             float(parts[4]), parts[6:10]))
            except ValueError:
                continue
        inside = rows
        if self.window is not None and rows:
            t0, t1 = self.window
            inside = [r for r in rows if t0 <= r[0] <= t1]
            if not inside:  # a window shorter than the interval: the nearest samples
                before = [r for r in rows if r[0] < t0]
                after = [r for r in rows if r[0] > t1]
                inside = before[-1:] + after[:1]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = {nm for r in inside for nm, val in zip(names, r[4])
                   if val.lower().startswith("active")}
        sm = [r[1] for r in inside]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max((r[2] for r in rows), default=0.0) or None,
                "reasons": sorted(reasons), "samples": len(sm),
                "samples_in_window": sum(1 for r in rows if self.window
                                         and self.window[0] <= r[0] <= self.window[1]),
                "power_w_max": max((r[3] for r in inside), default=0.0) or None}


def algorithmic_work(rows_list):
    """2 x MACs of the symmetric halves of I^E and I^V over alive, unpadded
    sizes (DP: m_r^2 n_r / 2 MACs, MD: n_r^2 m'_r / 2), the unordered pair
    tests, and the bit-packed operand bytes one pass of each product reads
    ((m_r n_r + n_r m'_r) / 8), summed over the rounds of every instance."""
    flops = 0.0
    pairs = 0.0
    bits_bytes = 0.0
    for rows in rows_list:
        for m, n, mdp in rows.tolist():
            flops += float(m) * m * n + float(n) * n * mdp
            pairs += m * (m - 1) / 2 + n * (n - 1) / 2
            bits_bytes += (float(m) * n + float(n) * mdp) / 8.0
    return flops, pairs, bits_bytes


def sparse_intrinsic_work(inst, alive_per_round):
    """Nonzero products of the two products per round, summed over rounds:
    sum over alive vertices of deg^2 (I^E = A A^T, DP) plus sum over the
    hyperedges DP kept of their alive size^2 (I^V = A^T A, MD).  The
    dense formulation's MACs over this is its overhead factor.
    alive_per_round: (vertex mask, edge mask) entering each round, then the
    final state, over input ids."""
    ptr = inst.edge_ptr.astype(np.int64)
    vtx = inst.edge_vtx
    row = np.repeat(np.arange(inst.m), np.diff(ptr))
    total = 0.0
    for (av, ae), (_, ae_next) in zip(alive_per_round[:-1], alive_per_round[1:]):
        live = av[vtx] & ae[row]
        deg = np.bincount(vtx[live], minlength=inst.n).astype(np.float64)
        total += float((deg * deg).sum())
        kept = av[vtx] & ae_next[row]  # hyperedges DP kept, over the vertices MD sees
        size = np.bincount(row[kept], minlength=inst.m).astype(np.float64)
        total += float((size * size).sum())
    return total


class DeviceInputs:
    """CSR of the workload uploaded once; the timed steps start from here."""

    def __init__(self, torch, dev, insts):
        self.insts = insts
        self.count = len(insts)
        self.n = np.array([i.n for i in insts], np.int32)
        self.m = np.array([i.m for i in insts], np.int32)
        self.k = np.array([i.k for i in insts], np.int64)
        nnz = np.array([i.nnz for i in insts], np.int64)
        base = np.concatenate([[0], np.cumsum(nnz)])
        ptr = np.zeros(int(self.m.sum()) + 1, np.int64)
        e0 = 0
        for b, i in enumerate(insts):
            ptr[e0:e0 + i.m + 1] = i.edge_ptr.astype(np.int64) + base[b]
            e0 += i.m
        vtx = np.concatenate([i.edge_vtx for i in insts] + [np.zeros(1, np.int32)])
        dem = np.concatenate([i.demand for i in insts] + [np.zeros(1, np.int32)])
        self.host = (ptr, vtx, dem)
        self.ptr64 = torch.from_numpy(ptr).to(dev)
        self.vtx = torch.from_numpy(vtx).to(dev)
        self.dem = torch.from_numpy(dem).to(dev)
        if self.count == 1:
            self.ptr32 = torch.from_numpy(insts[0].edge_ptr.astype(np.int32)).to(dev)
        self.av = torch.empty(int(self.n.sum()) + 1, dtype=torch.uint8, device=dev)
        self.ae = torch.empty(int(self.m.sum()) + 1, dtype=torch.uint8, device=dev)


class Runner:
    """One workload on the library's stream: load from device arrays,
    kernelize, write the result masks; `reps` kernelizations per step."""

    def __init__(self, torch, mhs, stream, insts, args, tiles=None, reps=1):
        self.torch, self.mhs, self.stream = torch, mhs, stream
        dev = torch.device("cuda", torch.cuda.current_device())
        self.D = DeviceInputs(torch, dev, insts)
        self.insts = insts
        self.batch = len(insts) > 1
        self.args = args
        self.tiles = tiles
        self.reps = reps

    def load(self):
        D, a = self.D, self.args
        if self.batch:
            return self.mhs.Instance.load_batch_device(D.n, D.m, D.k, D.ptr64, D.vtx, D.dem,
                                                       contraction=a.contraction,
                                                       stream=self.stream, tiles=self.tiles)
        i = self.insts[0]
        return self.mhs.Instance.load_device(i.n, i.m, D.ptr32, D.vtx, D.dem, i.k,
                                             contraction=a.contraction, stream=self.stream,
                                             tiles=self.tiles)

    def one(self, timing=False):
        """One kernelization; with timing, the contraction's event times and
        the tensor work counter."""
        h = self.load()
        if timing:
            h.set_timing(True)  # per-round graphs with event nodes around the contractions
        h.kernelize()           # default: the whole fixpoint as one graph launch
        if self.batch:
            h.result_batch_device(self.D.av, self.D.ae)
        else:
            h.result_device(self.D.av, self.D.ae)
        t = None
        if timing:
            t = h.last_timing()
            if self.args.contraction == "fp8":
                t["kblocks"], t["tiles"] = h.work_stats()
        self.cfg = h.tile_config() if self.args.contraction == "fp8" else None
        h.free()
        return t

    def step(self):
        for _ in range(self.reps):
            self.one()

    def traces(self):
        h = self.load()
        st = h.kernelize()
        tr = [h.trace(b)[0] for b in range(self.D.count)]
        h.free()
        return tr, int(st["rounds"])

    def timed(self, steps, warmup):
        """(ms of `steps` steps on the library's stream, CUDA events; then
        the contraction's ms and work counter summed over as many timed
        kernelizations)."""
        torch = self.torch
        for _ in range(warmup):
            self.step()
            self.one(timing=True)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(self.stream)
        for _ in range(steps):
            self.step()
        ev1.record(self.stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        contract_ms, kblocks = 0.0, 0
        for _ in range(steps):
            t = self.one(timing=True)
            contract_ms += t["dp_ms"] + t["md_ms"]
            kblocks += t.get("kblocks", 0)
        torch.cuda.synchronize()
        return ms, contract_ms, kblocks


def contraction_roofline(args, peaks, kind, flops_per_k, contract_ms, kblocks, steps):
    """issued tensor TFLOP/s and fractions (per timed kernelization)."""
    s_per_k = contract_ms / steps / 1e3
    dense_equiv = flops_per_k / s_per_k / 1e12 if s_per_k > 0 else 0.0
    if args.contraction == "fp8":
        peak = 2.0 * peaks["bf16_tflops"]
        issued = kblocks * 2.0 * 128 * 128 * 32 / (contract_ms / 1e3) / 1e12 if contract_ms else 0
        return {"issued_tflops": round(issued, 2), "frac": round(issued / peak, 4),
                "dense_equiv_frac": round(dense_equiv / peak, 4),
                "contract_ms_per_kernelization": round(contract_ms / steps, 4)}
    return {"contract_ms_per_kernelization": round(contract_ms / steps, 4)}


def run_ours(args, rank, world, dist):
    import torch
    from paper_2109_06042_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if dist is not None:
        dist.barrier()
    from paper_2109_06042_gb300 import mhs
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)  # the library runs all its work on this stream
    workload = headline_workload(args)
    insts, desc = make_instances(args, rank)
    reps = args.reps or REPS.get(workload, 1)
    R = Runner(torch, mhs, stream, insts, args, reps=reps)
    D = R.D
    batch = R.batch

    mhs.set_default_sparsity(args.sparsity)
    mhs.set_default_variant(args.rule, args.full_edges)

    # untimed: the library's per-round trace of every instance -> algorithmic work
    traces, rounds = R.traces()
    flops, pairs, bits_bytes = algorithmic_work(traces)
    # untimed: round by round through the public API, the alive sets entering
    # each round (single instance) -> the sparse intrinsic work
    intrinsic = None
    if not batch and not args.full_edges:
        inst0 = insts[0]
        states = [(np.ones(inst0.n, bool), np.ones(inst0.m, bool))]
        with mhs.Instance.load(inst0, contraction=args.contraction, use_graphs=False,
                               stream=stream) as hr:
            for _ in range(rounds):
                hr.reduce_round()
                r = hr.result()
                av = np.zeros(inst0.n, bool)
                ae = np.zeros(inst0.m, bool)
                av[r["vertices"]] = True
                ae[r["edges"]] = True
                states.append((av, ae))
        intrinsic = sparse_intrinsic_work(inst0, states)

    gpu_index = rank
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis and vis.split(",")[0].strip().isdigit():
        gpu_index = int(vis.split(",")[torch.cuda.current_device()].strip())
    clocks = ClockSampler(gpu_index)
    clocks.start()  # running before the timed region starts
    for _ in range(args.warmup):
        R.step()
        R.one(timing=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_window0 = time.time()
    ms, contract_ms, kblocks = R.timed(args.steps, 0)
    clocks.mark(t_window0, time.time())
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist, dev)
    ms_per_step = ms / args.steps
    units_per_step = D.count * reps
    value = job_throughput(world, units_per_step, args.steps, ms)

    # end to end through host buffers: load from host arrays, result masks back to host
    e2e = None
    if not args.no_e2e:
        ptr, vtx, dem = D.host

        def e2e_step():
            if batch:
                h = mhs.Instance.load_batch_arrays(D.count, D.n, D.m, ptr, vtx, dem, D.k,
                                                   contraction=args.contraction, stream=stream)
                h.kernelize()
                h.result_batch_device(D.av, D.ae)
            else:
                h = mhs.Instance.load(insts[0], contraction=args.contraction, stream=stream)
                h.kernelize()
                h.result_device(D.av, D.ae)
            out_v = D.av.cpu()
            out_e = D.ae.cpu()
            h.free()
            return out_v, out_e

        for _ in range(max(1, args.warmup // 2)):
            e2e_step()
        torch.cuda.synchronize()
        n_e2e = args.steps * (reps if not batch else 1)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        h2d = 8 * ptr.size + 4 * (vtx.size + dem.size) if batch else \
            4 * (insts[0].m + 1 + insts[0].nnz + insts[0].m)
        e2e = {"value": round(world * D.count * n_e2e / e2e_s, 4), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(D.av.numel() + D.ae.numel()),
               "form": "mhs_load (host CSR) + mhs_kernelize + result masks to host, per instance"
                       if not batch else "mhs_load_batch (host CSR) + mhs_kernelize + masks to host"}

    peaks, kind = load_peaks()
    launches = 2 * rounds
    per_launch = contract_ms / args.steps / launches
    contract_s_per_step = contract_ms / args.steps / 1e3  # per timed kernelization
    dense_equiv = flops / contract_s_per_step / 1e12
    prof = kernel_profile(args)
    if args.contraction == "fp8":
        # FP8 dense = 2 x BF16 (4.5 / 2.25 PF nominal); the burst figure, since the
        # contraction is timed in short steps at full clock
        peak = 2.0 * peaks["bf16_tflops"]
        # tensor work actually issued: units of 128 x 128 x 32 MACs, counted by
        # the kernel (block-sparse skipping leaves out K blocks and tiles whose
        # products are all zero, so this is below the dense formulation's count)
        issued = kblocks * 2.0 * 128 * 128 * 32 / (contract_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": round(issued, 2), "peak": round(peak, 1),
                "unit": "TFLOP/s", "frac": round(issued / peak, 4),
                "traffic": prof.get("traffic_bytes_per_launch"),
                "kernel": "k_tc_contract", "peak_source": f"{kind}: 2 x bf16_tflops (burst)",
                "launches_per_kernelization": launches, "avg_launch_ms": round(per_launch, 4),
                "achieved_basis": "tensor MACs issued x 2 (kernel counter)",
                "issued_flops_per_kernelization": kblocks * 2.0 * 128 * 128 * 32 / args.steps,
                "dense_equiv_tflops": round(dense_equiv, 2),
                "dense_equiv_frac": round(dense_equiv / peak, 4),
                "dense_formulation_flops_per_kernelization": flops,
                "sparse_intrinsic_macs_per_kernelization": intrinsic,
                "ncu_tensor_active_pct": prof.get("tensor_active_pct"),
                "ncu_profile": prof.get("file"),
                "tile_shape": R.cfg,
                "sparsity": args.sparsity}
    else:
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 16 * 32 * 2 * sm_mhz * 1e6 / 1e12  # 16 POPC/clk/SM x 32 bit-MACs
        # bit-packed operand bytes one pass reads, against the measured copy rate
        hbm = bits_bytes / contract_s_per_step / 1e9
        roof = {"bound": "alu", "achieved": round(dense_equiv, 2), "peak": round(peak, 1),
                "unit": "TOP/s", "frac": round(dense_equiv / peak, 4), "traffic": None,
                "kernel": "k_pop_contract", "peak_source": "derived: 16 POPC/clk/SM nominal",
                "launches_per_kernelization": launches, "avg_launch_ms": round(per_launch, 4),
                "achieved_basis": "bit-MACs of the dense formulation x 2 (every 64 x 64 "
                                  "tile of the upper triangle is contracted)",
                "sparse_intrinsic_macs_per_kernelization": intrinsic,
                "hbm": {"achieved": round(hbm, 2), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": round(hbm / peaks["hbm_gbs"], 4),
                        "basis": "bit-packed operand bytes per pass, (m n + n m') / 8"}}

    cpu = seq = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(insts, desc, args.cpu_seconds, args)
        seq = cpu_sequential(insts, desc, args.cpu_seconds) if variant_name(args) == "DP+MD" \
            else None

    # Kernels of one kernelization.  Load: k_validate, k_init, k_vertex_degrees,
    # k_vertex_layout, k_layout_keys, k_layout_scan, k_layout_place,
    # k_layout_rank, k_layout_commit, k_edge_rows (a batch adds
    # k_gather_bounds and k_localize_ptr), then the
    # result-mask kernel.  Per round: k_plan, the A set scatter, [k_tile_list],
    # the DP contraction, k_compact_edges, k_plan, the fused A clear / A^T set
    # scatter, [k_tile_list], the MD contraction, the A^T clear scatter,
    # k_compact_vertices and the loop-condition kernel ([] tcgen05 only), plus
    # the three FE kernels with --full-edges.
    load_kernels = 11 + (2 if batch else 0)
    per_round = (12 if args.contraction == "fp8" else 10) + (3 if args.full_edges else 0)
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "e4m3" if args.contraction == "fp8" else "u32-popcount",
        "data": DATA,
        "config": {"workload": desc, "contraction": args.contraction, "rounds": rounds,
                   "sparsity": args.sparsity, "rules": variant_name(args),
                   "instances_per_step": units_per_step,
                   "kernelizations_per_step": reps,
                   "l2": "inputs larger than L2: dense operands "
                         f"{sum(i.m * i.n for i in insts) / 1e9:.2f} GB per product",
                   "parallelism": f"{world} GPU(s), independent instances per GPU"},
        "pair_tests_per_s": round(world * pairs * reps * args.steps / (ms / 1e3), 1),
        "roofline": roof,
        "cpu_baseline": cpu,
        "cpu_sequential": seq,
        "e2e": e2e,
        "gpu_launches": args.steps * reps * (load_kernels + per_round * rounds),
        "clocks": clk,
    }
    if batch and not args.no_loop:
        line["per_instance_loop"] = per_instance_loop(torch, mhs, stream, insts, args, D)
    if args.workload == "all" and world == 1:
        line["configs"] = sub_records(torch, mhs, stream, args, peaks, kind)
    return line


def per_instance_loop(torch, mhs, stream, insts, args, D):
    """The plain one-instance-per-call form of a batch on the same GPU."""
    dev = torch.device("cuda", torch.cuda.current_device())
    singles = []
    for i in insts:
        singles.append((i, torch.from_numpy(i.edge_ptr.astype(np.int32)).to(dev),
                        torch.from_numpy(i.edge_vtx if i.nnz else np.zeros(1, np.int32)).to(dev),
                        torch.from_numpy(i.demand if i.m else np.zeros(1, np.int32)).to(dev)))
    for i, p_, v_, d_ in singles[:8]:
        hh = mhs.Instance.load_device(i.n, i.m, p_, v_, d_, i.k, contraction=args.contraction,
                                      stream=stream)
        hh.kernelize()
        hh.free()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, p_, v_, d_ in singles:
        hh = mhs.Instance.load_device(i.n, i.m, p_, v_, d_, i.k, contraction=args.contraction,
                                      stream=stream)
        hh.kernelize()
        hh.result_device(D.av, D.ae)
        hh.free()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"value": round(len(insts) / dt, 2), "unit": UNIT,
            "form": "mhs_load_device + mhs_kernelize + mhs_result_device per instance"}


def sub_records(torch, mhs, stream, args, peaks, kind):
    """The other workloads on the same GPU (N = 1): instances/s with inputs in
    HBM (CUDA events), the contraction's issued tensor fraction, the tile
    shape; the batch with autotuned and fixed shapes and its one-instance
    loop; a short serving sweep."""
    out = {}
    steps, warmup = args.sub_steps, 3
    for wl in ("uniform", "interval", "batch"):
        insts, desc = make_instances(args, 0, wl)
        reps = REPS[wl]
        R = Runner(torch, mhs, stream, insts, args, reps=reps)
        traces, rounds = R.traces()
        flops, pairs, _ = algorithmic_work(traces)
        ms, cms, kb = R.timed(steps, warmup)
        rec = {"workload": desc, "rounds": rounds,
               "value": round(len(insts) * reps * steps / (ms / 1e3), 3), "unit": UNIT,
               "ms_per_kernelization": round(ms / steps / reps, 4),
               "pair_tests_per_s": round(pairs * reps * steps / (ms / 1e3), 1),
               "tile_shape": R.cfg}
        rec.update(contraction_roofline(args, peaks, kind, flops, cms, kb, steps))
        if wl == "batch":
            F = Runner(torch, mhs, stream, insts, args, tiles=DEFAULT_TILES, reps=1)
            ms_f, _, _ = F.timed(steps, warmup)
            rec["fixed_shape"] = {"tile_shape": DEFAULT_TILES,
                                  "value": round(len(insts) * steps / (ms_f / 1e3), 3)}
            if not args.no_loop:
                rec["per_instance_loop"] = per_instance_loop(torch, mhs, stream, insts, args, R.D)
            del F
        out[wl] = rec
        del R
        torch.cuda.empty_cache()
    out["stream"] = serve_sweep(mhs, torch, args, args.sub_requests, min(args.pool, 150),
                                args.sub_rates, rank=0)
    if args.contraction == "fp8":
        out["precision"] = precision_record(torch, mhs, stream, args, peaks)
    return out


def precision_record(torch, mhs, stream, args, peaks):
    """The headline instance through the bit-packed AND + popcount form and
    through the FP8 tensor-core form on the same GPU: time per kernelization
    of each, the popcount contraction's ALU and HBM fractions, and whether
    the two forms give the same result masks byte for byte."""
    import copy
    insts, desc = make_instances(args, 0, "powerlaw")
    pa = copy.copy(args)
    pa.contraction = "popcount"
    P = Runner(torch, mhs, stream, insts, pa, reps=1)
    traces, rounds = P.traces()
    flops, _, bits_bytes = algorithmic_work(traces)
    steps = 3
    ms, cms, _ = P.timed(steps, 1)
    P.one()
    av_p, ae_p = P.D.av.clone(), P.D.ae.clone()
    F = Runner(torch, mhs, stream, insts, args, reps=1)
    ms_f, _, _ = F.timed(steps, 1)
    F.one()
    nv, ne = int(F.D.n.sum()), int(F.D.m.sum())  # (the masks' last byte is padding)
    same = bool(torch.equal(av_p[:nv], F.D.av[:nv]) and torch.equal(ae_p[:ne], F.D.ae[:ne]))
    s_contract = cms / steps / 1e3
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    popc_peak = 152 * 16 * 32 * 2 * sm_mhz * 1e6 / 1e12  # 16 POPC/clk/SM x 32 bit-MACs
    alu = flops / s_contract / 1e12 if s_contract > 0 else 0.0
    hbm = bits_bytes / s_contract / 1e9 if s_contract > 0 else 0.0
    rec = {"workload": desc, "rounds": rounds,
           "popcount": {"kernel": "k_pop_contract",
                        "ms_per_kernelization": round(ms / steps, 3),
                        "value": round(steps / (ms / 1e3), 3), "unit": UNIT,
                        "alu": {"achieved": round(alu, 2), "peak": round(popc_peak, 1),
                                "unit": "TOP/s", "frac": round(alu / popc_peak, 4),
                                "basis": "bit-MACs of the dense formulation x 2"},
                        "hbm": {"achieved": round(hbm, 2), "peak": peaks["hbm_gbs"],
                                "unit": "GB/s", "frac": round(hbm / peaks["hbm_gbs"], 4),
                                "basis": "bit-packed operand bytes per pass"}},
           "fp8": {"kernel": "k_tc_contract", "ms_per_kernelization": round(ms_f / steps, 3),
                   "value": round(steps / (ms_f / 1e3), 3), "unit": UNIT},
           "identical_output": same,
           "speedup_fp8_over_popcount": round(ms / ms_f, 2) if ms_f > 0 else None}
    del P, F
    torch.cuda.empty_cache()
    return rec


def serve_sweep(mhs, torch, args, requests, pool_size, rates, rank=0):
    """Poisson arrivals of stream-shaped requests, at several rates, through
    the continuous-batching server and through the plain one-at-a-time form
    (mhs_load + mhs_kernelize + mhs_result per request, in arrival order),
    both measured under the same arrival times on the same GPU."""
    from paper_2109_06042_gb300 import instances as I
    rng = np.random.Generator(np.random.PCG64(777 + rank))
    pool = [I.config_stream_one(50_000 + rank * 100_000 + i) for i in range(pool_size)]
    order = rng.integers(0, len(pool), size=requests)
    reqs = [pool[i] for i in order]
    contraction = args.contraction
    for i in reqs[:3]:
        mhs.kernelize(i, contraction=contraction)
    torch.cuda.synchronize()
    # the plain form back to back: its saturating rate
    t0 = time.perf_counter()
    for i in reqs:
        mhs.kernelize(i, contraction=contraction)
    plain_rate = len(reqs) / (time.perf_counter() - t0)

    def pace(arrivals, t0, a):
        now = time.perf_counter() - t0
        if a > now:
            time.sleep(a - now)

    def serve(arrivals):
        """Server: (latencies s, makespan s)."""
        with mhs.Server(contraction=contraction) as srv:
            t0 = time.perf_counter()
            tickets = []
            for a, inst in zip(arrivals, reqs):
                pace(arrivals, t0, a)
                tickets.append(srv.submit(inst))
            lat = []
            for t in tickets:
                r = srv.poll(t, timeout_us=600_000_000)
                lat.append(r["times_ns"][2] / 1e9)
            makespan = time.perf_counter() - t0
        return np.array(lat), makespan

    def plain(arrivals):
        """One request at a time, in arrival order, each started at its
        arrival or when the previous one finished: (latencies s, makespan s)."""
        t0 = time.perf_counter()
        lat = []
        for a, inst in zip(arrivals, reqs):
            pace(arrivals, t0, a)
            mhs.kernelize(inst, contraction=contraction)
            lat.append(time.perf_counter() - t0 - a)
        return np.array(lat), time.perf_counter() - t0

    serve(np.zeros(min(len(reqs), 64)))  # warm-up
    lat0, mk0 = serve(np.zeros(len(reqs)))  # everything at once: the saturating rate
    sat = len(reqs) / mk0
    pct = lambda x, q: round(1e3 * float(np.percentile(x, q)), 3)
    sweep = []
    for mult in [float(x) for x in rates.split(",")]:
        rate = mult * sat
        arr = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
        lat, mk = serve(arr)
        plat, pmk = plain(arr)
        sweep.append({
            "rate_per_s": round(rate, 2), "x_saturating": mult,
            "served": {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                       "instances_per_s": round(len(reqs) / mk, 2)},
            "plain": {"p50_ms": pct(plat, 50), "p99_ms": pct(plat, 99),
                      "instances_per_s": round(len(reqs) / pmk, 2)},
        })
    return {"workload": f"{requests} requests per rate from {len(pool)} seeded instances "
                        "(n log-uniform [100,20000], m~U[n,3n], |e|~U[2,16], f<=3), "
                        "Poisson arrivals",
            "closed_loop_rate_per_s": round(sat, 2),
            "closed_loop_p50_ms": pct(lat0, 50), "closed_loop_p99_ms": pct(lat0, 99),
            "plain_rate_per_s": round(plain_rate, 2),
            "speedup_vs_plain": round(sat / plain_rate, 3),
            "server": "max_slots 256, budget 3/4 of free HBM",
            "plain_form": "mhs_load + mhs_kernelize + mhs_result per request, measured "
                          "under the same arrival times",
            "sweep": sweep}


def run_stream(args, rank, world):
    """Serving: the sweep of serve_sweep at --requests per rate."""
    import torch
    from paper_2109_06042_gb300 import build as B
    B.build()
    from paper_2109_06042_gb300 import mhs
    mhs.set_default_variant(args.rule, args.full_edges)
    sv = serve_sweep(mhs, torch, args, args.requests, args.pool, args.rates, rank)
    best = max(sv["sweep"], key=lambda r: r["served"]["instances_per_s"])
    return {
        "metric": "served instances/s (continuous batching) with p50/p99 latency",
        "value": best["served"]["instances_per_s"], "unit": UNIT, "n_gpus": world,
        "steps": len(sv["sweep"]), "warmup": 1, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "e4m3" if args.contraction == "fp8" else "u32-popcount", "data": DATA,
        "config": {"workload": sv["workload"], "contraction": args.contraction,
                   "server": sv["server"]},
        "serving": sv,
    }


PROFILE = os.path.join(ROOT, "profiles", "k_tc_contract_powerlaw_n20000_m40000.md")
PROFILE_SOURCES = ("contract_tc.cu", "kernels.cu", "mhs_internal.h")


def kernel_sources_sha256():
    """Digest of the sources that decide the contraction's counters."""
    import hashlib
    h = hashlib.sha256()
    for f in PROFILE_SOURCES:
        with open(os.path.join(ROOT, "paper_2109_06042_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def kernel_profile(args):
    """Counters of k_tc_contract from the committed ncu summary of this
    workload: DRAM bytes per launch (dram__bytes_read.sum +
    dram__bytes_write.sum, averaged over one kernelization's launches) and
    the tensor pipe's active share; empty when the workload or options
    differ or the kernel sources changed since the capture."""
    default = (headline_workload(args) == "powerlaw" and args.seed == 0 and
               args.sparsity == "skip" and
               args.rule == "dp" and not args.full_edges and args.contraction == "fp8")
    if not default or not os.path.exists(PROFILE):
        return {}
    fields = {}
    with open(PROFILE) as fh:
        for line in fh:
            if ":" in line and line.startswith(("traffic_bytes_per_launch", "source_sha256",
                                                "tensor_active_pct")):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
    if fields.get("source_sha256") != kernel_sources_sha256():
        return {}
    out = {"file": os.path.relpath(PROFILE, ROOT)}
    for k, conv in (("traffic_bytes_per_launch", lambda v: int(float(v))),
                    ("tensor_active_pct", float)):
        try:
            out[k] = conv(fields[k])
        except (KeyError, ValueError):
            pass
    return out


def variant_name(args):
    return ("SE+MD" if args.rule == "se" else "DP+MD") + ("+FE" if args.full_edges else "")


def cpu_baseline(insts, desc, seconds, args):
    """The oracle, as it stands, on a bounded sample of the workload."""
    from oracle import oracle as O
    O.build()
    done = 0
    t0 = time.perf_counter()
    for i in insts:
        O.reduce_variant(i, args.rule, args.full_edges)
        done += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    sample = (f"{done} of {len(insts)} instance(s) of the workload ({desc}), "
              f"single-threaded C oracle with exact pair pruning, {dt:.2f} s")
    return {"value": round(done / dt, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": sample}


def cpu_sequential(insts, desc, seconds):
    """The paper's sequential design (Section 4.2, Algorithms 4-6) with
    OpenMP on every host core, on a bounded sample of the workload."""
    from oracle import kernelcpu as KC
    KC.build()
    cores = os.cpu_count() or 1
    sized = [i for i in insts if KC.matrix_bytes(i.n, i.m) <= KC.DEFAULT_MAX_BYTES]
    if not sized:
        return {"value": None, "unit": UNIT, "cores": cores,
                "kind": "paper sequential algorithm (Algorithms 4-6)",
                "sample": f"not run: dense count matrices of {desc} exceed "
                          f"{KC.DEFAULT_MAX_BYTES >> 30} GiB"}
    done = 0
    t0 = time.perf_counter()
    for i in sized:
        KC.reduce(i, threads=cores)
        done += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": round(done / dt, 6), "unit": UNIT, "cores": cores,
            "kind": "paper sequential algorithm (Algorithms 4-6)",
            "sample": f"{done} of {len(insts)} instance(s) of the workload ({desc}), "
                      f"dense I^E/I^V count matrices, OpenMP over {cores} threads, {dt:.2f} s"}


def run_reference(args, rank, world):
    """The CPU oracle on the same workload; each step a bounded sample."""
    if rank != 0:
        return None
    from oracle import oracle as O
    O.build()
    insts, desc = make_instances(args, 0)
    per_step = max(1.0, args.cpu_seconds / max(args.steps, 1))

    def one_step():
        done, t0 = 0, time.perf_counter()
        for i in insts:
            O.reduce_variant(i, args.rule, args.full_edges)
            done += 1
            if time.perf_counter() - t0 > per_step:
                break
        return done, time.perf_counter() - t0

    for _ in range(args.warmup):
        one_step()
    total_done, total_t = 0, 0.0
    for _ in range(args.steps):
        d, t = one_step()
        total_done += d
        total_t += t
    value = total_done / total_t
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * total_t / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": DATA,
        "config": {"workload": desc, "contraction": "explicit pairwise set tests (oracle)",
                   "rules": variant_name(args), "parallelism": "host CPU, single thread"},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{total_done} kernelizations over {args.steps} steps, each "
                                   f"step at most ~{per_step:.1f} s of the workload ({desc})"},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    if args.workload == "stream":
        line = run_stream(args, rank, world)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as Dd
        Dd.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = Dd
    line = run_ours(args, rank, world, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

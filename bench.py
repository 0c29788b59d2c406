#!/usr/bin/env python
"""Throughput of the exhaustive DP + MD kernelization (Algorithm 3) on GB300.

A step is one complete kernelization of one instance: load from device
arrays (the CSR already resident in HBM), every round of DP (Algorithm 1)
and MD (Algorithm 2) with their contractions, compaction, and the result
masks written to device memory.  ``value`` is reduced instances per second
over all GPUs; the line also carries pair tests per second, the roofline of
the dominant kernel (the tcgen05 contraction), the CPU oracle timed on the
host, an end-to-end figure through host buffers and the SM clocks seen.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       (N > 1 runs under torchrun; each rank reduces its own instances.)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reduced instances/s (exhaustive DP+MD kernelization)"
UNIT = "instances/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["powerlaw", "uniform", "interval"], default="powerlaw")
    p.add_argument("--contraction", choices=["fp8", "popcount"], default="fp8")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


def make_instance(workload, seed):
    from paper_2109_06042_gb300 import instances as I
    return {"powerlaw": I.config_powerlaw, "uniform": I.config_uniform,
            "interval": I.config_interval}[workload](seed)


def workload_desc(inst, workload, seed):
    return f"{workload} n={inst.n} m={inst.m} nnz={inst.nnz} seed={seed}"


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def round_trace(mhs, inst, contraction):
    """Sizes per round (untimed): hyperedges and vertices entering the DP and
    MD passes, from the library's own per-round counters."""
    h = mhs.Instance.load(inst, contraction=contraction)
    m_r, n_r = inst.m, inst.n
    rows = []
    while True:
        st = h.reduce_round()
        m_after_dp = m_r - st["dp_deleted"]
        rows.append((m_r, n_r, m_after_dp))
        m_r, n_r = st["m_alive"], st["n_alive"]
        if not st["changed"]:
            break
    h.free()
    return rows


def algorithmic_work(rows):
    """2 x MACs of the symmetric halves of I^E and I^V over alive, unpadded
    sizes (DP: m_r^2 n_r / 2 MACs, MD: n_r^2 m'_r / 2), and the pair tests."""
    flops = sum(m * m * n + n * n * mdp for (m, n, mdp) in rows)
    pairs = sum(m * (m - 1) // 2 + n * (n - 1) // 2 for (m, n, _) in rows)
    return float(flops), float(pairs)


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
    seed = args.seed + rank
    inst = make_instance(args.workload, seed)
    ptr = torch.from_numpy(inst.edge_ptr).to(dev)
    vtx = torch.from_numpy(inst.edge_vtx if inst.nnz else inst.edge_vtx.reshape(0)).to(dev)
    dem = torch.from_numpy(inst.demand).to(dev)
    av = torch.empty(max(inst.n, 1), dtype=torch.uint8, device=dev)
    ae = torch.empty(max(inst.m, 1), dtype=torch.uint8, device=dev)
    rows = round_trace(mhs, inst, args.contraction)
    rounds = len(rows)
    flops, pairs = algorithmic_work(rows)

    def step(timing):
        h = mhs.Instance.load_device(inst.n, inst.m, ptr, vtx, dem, inst.k,
                                     contraction=args.contraction, stream=stream)
        if timing:
            h.set_timing(True)
        h.kernelize()
        h.result_device(av, ae)
        t = h.last_timing() if timing else None
        h.free()
        return t

    for _ in range(args.warmup):
        step(True)
    torch.cuda.synchronize()
    gpu_index = rank
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis and vis.split(",")[0].strip().isdigit():
        gpu_index = int(vis.split(",")[torch.cuda.current_device()].strip())
    clocks = ClockSampler(gpu_index)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    contract_ms = 0.0
    for _ in range(args.steps):
        t = step(True)
        contract_ms += t["dp_ms"] + t["md_ms"]
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    if dist is not None:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    ms_per_step = ms / args.steps
    value = world * args.steps / (ms / 1e3)

    # end to end: host CSR in, host result out, through the public API
    e2e = None
    if not args.no_e2e:
        import numpy as np
        for _ in range(max(1, args.warmup // 2)):
            mhs.kernelize(inst, contraction=args.contraction)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = None
        for _ in range(args.steps):
            res = mhs.kernelize(inst, contraction=args.contraction)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        h2d = 4 * (inst.m + 1 + inst.nnz + inst.m)
        d2h = 4 * (len(res["vertices"]) + 2 * len(res["edges"])) + 4 * inst.m
        e2e = {"value": world * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
        del np

    peaks, kind = load_peaks()
    if args.contraction == "fp8":
        # FP8 dense = 2 x BF16 (4.5 / 2.25 PF nominal); the burst figure, since the
        # contraction is timed in short steps (tens of ms) at full clock
        peak = 2.0 * peaks["bf16_tflops"]
        achieved = flops / (contract_ms / args.steps / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": round(achieved, 2), "peak": round(peak, 1),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": "k_tc_contract", "peak_source": f"{kind}: 2 x bf16_tflops (burst)",
                "launches_per_step": 2 * rounds}
    else:
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 16 * 32 * 2 * sm_mhz * 1e6 / 1e12  # 16 POPC/clk/SM x 32 bit-MACs
        achieved = flops / (contract_ms / args.steps / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak, 1),
                "unit": "TOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": "k_pop_contract", "peak_source": "derived: 16 POPC/clk/SM nominal",
                "launches_per_step": 2 * rounds}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        t0 = time.perf_counter()
        O.reduce(inst)
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one full {workload_desc(inst, args.workload, seed)} instance, "
                         f"single-threaded C oracle with exact pair pruning ({dt:.2f} s)"}

    launches = args.steps * (4 + 8 * rounds + 1)
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "e4m3" if args.contraction == "fp8" else "u32-popcount",
        "data": "synthetic (seeded generator, shapes of the paper's workloads)",
        "config": {"workload": workload_desc(inst, args.workload, seed),
                   "contraction": args.contraction, "rounds": rounds,
                   "l2": "inputs larger than L2: dense operands "
                         f"{inst.m * inst.n / 1e9:.2f} GB per product",
                   "parallelism": f"{world} independent instance(s), one per GPU"},
        "pair_tests_per_s": round(world * pairs * args.steps / (ms / 1e3), 1),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    return line


def run_reference(args, rank, world):
    """The CPU oracle on the same workload, one full kernelization per step."""
    if rank != 0:
        return None
    from oracle import oracle as O
    O.build()
    inst = make_instance(args.workload, args.seed)
    for _ in range(args.warmup):
        O.reduce(inst)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.reduce(inst)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    desc = workload_desc(inst, args.workload, args.seed)
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * dt / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded generator, shapes of the paper's workloads)",
        "config": {"workload": desc, "contraction": "explicit pairwise set tests",
                   "parallelism": "host CPU, single thread"},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"one full {desc} instance per step"},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as D
        D.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = D
    line = run_ours(args, rank, world, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

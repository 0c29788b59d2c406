"""Autotuner of the tcgen05 tile shape.

The tensor-core contraction has three free choices that change speed and
never a result: the tile width (128 x 256 tiles with two TMEM accumulators,
or 128 x 128 with four), the number of row blocks per L2 group of the tile
order, and whether a K block shared in one 64-column half only is loaded as
that half.  Which is fastest depends on the instance's size and structure.

This script times every shape on seeded workloads of each size class --
one kernelization per step (load from device arrays, every round, result
masks), CUDA events on the library's stream, the median of several steps
after warm-up -- and writes the fastest shape of each class to the table
the library reads when a load leaves the shape to the autotuner
(mhs_options.tile_n / group_rows / half_stages = 0).  Table lines:

    <kind> <log2 rows> <tile_n> <group_rows> <half_stages: 1 on, 2 off>

Usage (on the GPU): python -m paper_2109_06042_gb300.autotune [--out PATH]
[--reps N] [--classes name,...]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import sys

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TABLE = os.path.join(PKG, "tile_table.txt")

SHAPES = [dict(tile_n=tn, group_rows=g, half_stages=h)
          for tn in (256, 128) for g in (8, 16, 32) for h in (True, False)]
DEFAULT = dict(tile_n=256, group_rows=16, half_stages=True)


def classes():
    """(name, kind, instances) of every size class, from the seeded
    generators with the shapes of the workloads the library serves."""
    from paper_2109_06042_gb300 import instances as I
    out = [("uniform_200x400", "single", lambda: [I.config_uniform(0)])]
    for n in (1000, 4000, 16000):  # stream-shaped single requests
        out.append((f"stream_n{n}", "single",
                    lambda n=n: [I.uniform_random(n, 2 * n, 2, 16, 3, n // 10, 7_000 + n,
                                                  name=f"stream_n{n}")]))
    out.append(("powerlaw_20000x40000", "single", lambda: [I.config_powerlaw(0)]))
    out.append(("interval_50000x100000", "single", lambda: [I.config_interval(0)]))
    out.append(("batch_4096", "batch", lambda: I.config_batch(4096, 4000)))
    return out


def size_class(insts):
    rows = [max(i.n, i.m) for i in insts]
    typical = sum(rows) // len(rows)
    return int(math.floor(math.log2(max(typical, 1))))


def time_shape(torch, mhs, D, shape, reps, warmup, stream):
    def step():
        if D["count"] > 1:
            h = mhs.Instance.load_batch_device(D["n"], D["m"], D["k"], D["ptr64"], D["vtx"],
                                               D["dem"], contraction="fp8", stream=stream,
                                               tiles=shape)
            h.kernelize()
            h.result_batch_device(D["av"], D["ae"])
        else:
            i = D["inst"]
            h = mhs.Instance.load_device(i.n, i.m, D["ptr32"], D["vtx"], D["dem"], i.k,
                                         contraction="fp8", stream=stream, tiles=shape)
            h.kernelize()
            h.result_device(D["av"], D["ae"])
        h.free()

    for _ in range(warmup):
        step()
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def device_inputs(torch, insts):
    dev = torch.device("cuda", torch.cuda.current_device())
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
    D = {"count": len(insts), "n": n, "m": m, "k": k, "inst": insts[0],
         "ptr64": torch.from_numpy(ptr).to(dev), "vtx": torch.from_numpy(vtx).to(dev),
         "dem": torch.from_numpy(dem).to(dev),
         "av": torch.empty(int(n.sum()) + 1, dtype=torch.uint8, device=dev),
         "ae": torch.empty(int(m.sum()) + 1, dtype=torch.uint8, device=dev)}
    if len(insts) == 1:
        D["ptr32"] = torch.from_numpy(insts[0].edge_ptr.astype(np.int32)).to(dev)
    return D


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--out", default=TABLE)
    p.add_argument("--json", default=None, help="also write every timing here")
    p.add_argument("--reps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=2)
    p.add_argument("--margin", type=float, default=0.02,
                   help="a shape replaces the default only if faster by this fraction")
    p.add_argument("--classes", default="", help="comma-separated class names (default: all)")
    args = p.parse_args()
    import torch
    from paper_2109_06042_gb300 import build
    build.build()
    from paper_2109_06042_gb300 import mhs
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    wanted = set(filter(None, args.classes.split(",")))
    lines, report = [], []
    for name, kind, make in classes():
        if wanted and name not in wanted:
            continue
        insts = make()
        D = device_inputs(torch, insts)
        lg = size_class(insts)
        timed = []
        for shape in SHAPES:
            ms = time_shape(torch, mhs, D, shape, args.reps, args.warmup, stream)
            timed.append((ms, shape))
            report.append({"class": name, "kind": kind, "log2_rows": lg, "ms": round(ms, 4),
                           **shape})
            print(f"{name:24s} {shape} {ms:9.3f} ms", flush=True)
        timed.sort(key=lambda t: t[0])
        ms, best = timed[0]
        default = next(t for t, s in timed if s == DEFAULT)
        # keep the default unless another shape is faster by more than the
        # run-to-run spread of these timings
        if ms > default * (1.0 - args.margin):
            ms, best = default, DEFAULT
        lines.append((kind, lg, best, ms, default, name))
        del D
        torch.cuda.empty_cache()
    with open(args.out, "w") as fh:
        fh.write("# Tile shapes of the tcgen05 contraction, fastest per size class, written by\n"
                 "# paper_2109_06042_gb300/autotune.py from timings on the GPU.\n"
                 "# kind log2_rows tile_n group_rows half_stages(1 on, 2 off)"
                 "  # class: best ms vs default (256, 16, on) ms\n")
        for kind, lg, best, ms, default, name in lines:
            fh.write(f"{kind} {lg} {best['tile_n']} {best['group_rows']} "
                     f"{1 if best['half_stages'] else 2}  # {name}: {ms:.4f} ms vs "
                     f"{default:.4f} ms\n")
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(report, fh, indent=1)
    print(f"wrote {args.out}")


if __name__ == "__main__":
    main()

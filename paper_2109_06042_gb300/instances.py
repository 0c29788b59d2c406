"""Seeded synthetic Multiple Hitting Set instances.

This module only draws random hypergraphs; it holds none of the reduction
arithmetic, so both the CUDA path and the CPU oracle can take their inputs
from it.  An instance is the problem input of Problem 1.1 (Section 1): a
hypergraph H=(V,E) with V={0..n-1}, hyperedges as sorted vertex lists in CSR
form, a demand f(e) >= 1 per hyperedge and the budget k.

Workload shapes (the paper's own data sets are not available; these stand in
for them, with the shapes of the experiments in Section 6):

* ``uniform``      n=200, m=400, |e|~U{2..8}, distinct uniform vertices,
                   f~U{1..min(3,|e|)}, k=60.
* ``powerlaw``     n=20,000, m=40,000, P(|e|=s) ~ s^-2.5 on {2..64},
                   vertices drawn without replacement with Zipf(1.1)
                   popularity over a seeded permutation of ids,
                   f~U{1..min(4,|e|)}, k=n/10.
* ``interval``     n=50,000 vertices on a line, m=100,000 hyperedges, each an
                   interval with uniform start and geometric length (mean 12)
                   clipped to the line, 5% of members replaced by uniform
                   vertices then deduplicated, f~U{1..min(2,|e|)}, k=n/10.
                   Interval hypergraphs have low Dilworth number (Section 2.3).
* ``batch``        many independent instances, n~U{50..2000}, m~U{n..2n},
                   |e|~U{2..16}, f~U{1..min(3,|e|)}, k=floor(n/10).
* ``stream``       n log-uniform in [100, 20000], m~U{n..3n}, sizes and
                   demands as ``batch``.

Every generator takes an explicit integer seed and uses
``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import hashlib

import numpy as np


@dataclasses.dataclass
class Instance:
    """A Multiple Hitting Set instance (H=(V,E), f, k) in CSR form."""

    n: int
    m: int
    edge_ptr: np.ndarray  # int32[m+1]
    edge_vtx: np.ndarray  # int32[nnz], each row sorted ascending, no duplicates
    demand: np.ndarray  # int32[m], >= 1
    k: int
    name: str = ""
    seed: int = -1

    @property
    def nnz(self) -> int:
        return int(self.edge_ptr[-1])

    def edges(self):
        """Hyperedges as Python lists (for small instances only)."""
        p = self.edge_ptr
        return [self.edge_vtx[p[i]:p[i + 1]].tolist() for i in range(self.m)]

    def sha256(self) -> str:
        h = hashlib.sha256()
        h.update(np.array([self.n, self.m, self.k], dtype=np.int64).tobytes())
        h.update(np.ascontiguousarray(self.edge_ptr, dtype=np.int32).tobytes())
        h.update(np.ascontiguousarray(self.edge_vtx, dtype=np.int32).tobytes())
        h.update(np.ascontiguousarray(self.demand, dtype=np.int32).tobytes())
        return h.hexdigest()


def from_edges(n: int, edges, demand, k: int = 0, name: str = "") -> Instance:
    """Build an Instance from a list of vertex lists (deduplicated, sorted)."""
    rows = [sorted(set(int(v) for v in e)) for e in edges]
    ptr = np.zeros(len(rows) + 1, dtype=np.int32)
    for i, r in enumerate(rows):
        ptr[i + 1] = ptr[i] + len(r)
    vtx = np.array([v for r in rows for v in r], dtype=np.int32)
    dem = np.asarray(demand, dtype=np.int32).reshape(-1)
    if dem.size != len(rows):
        raise ValueError("one demand per hyperedge")
    return Instance(n=int(n), m=len(rows), edge_ptr=ptr, edge_vtx=vtx,
                    demand=dem, k=int(k), name=name)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _distinct_rows(rng, sizes: np.ndarray, draw) -> list:
    """Draw, for every row r, ``sizes[r]`` distinct values.

    ``draw(shape)`` returns i.i.d. samples; entries that repeat an earlier
    entry of the same row are redrawn until every row is duplicate-free.
    Rows are returned sorted.
    """
    m = sizes.size
    smax = int(sizes.max()) if m else 0
    cand = draw((m, smax))
    col = np.arange(smax)[None, :]
    valid = col < sizes[:, None]
    while True:
        # mark the second and later occurrences of a value within a row
        key = np.where(valid, cand, -1 - col)  # padding never collides
        order = np.argsort(key, axis=1, kind="stable")
        sk = np.take_along_axis(key, order, axis=1)
        dup_sorted = np.zeros_like(sk, dtype=bool)
        dup_sorted[:, 1:] = sk[:, 1:] == sk[:, :-1]
        dup = np.zeros_like(dup_sorted)
        np.put_along_axis(dup, order, dup_sorted, axis=1)
        dup &= valid
        nd = int(dup.sum())
        if nd == 0:
            break
        cand[dup] = draw((nd,))
    out = np.sort(np.where(valid, cand, np.iinfo(np.int64).max), axis=1)
    return out, valid


def _pack(n, sizes, rows_sorted, demand, k, name, seed) -> Instance:
    m = sizes.size
    ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(sizes, out=ptr[1:])
    smax = rows_sorted.shape[1] if m else 0
    mask = np.arange(smax)[None, :] < sizes[:, None]
    vtx = rows_sorted[mask].astype(np.int32)
    return Instance(n=int(n), m=int(m), edge_ptr=ptr.astype(np.int32),
                    edge_vtx=vtx, demand=demand.astype(np.int32), k=int(k),
                    name=name, seed=int(seed))


def _demands(rng, sizes, alpha):
    hi = np.minimum(alpha, sizes)
    return rng.integers(1, hi + 1)


def uniform_random(n: int, m: int, smin: int, smax: int, alpha: int, k: int,
                   seed: int, name: str = "uniform") -> Instance:
    """|e|~U{smin..smax} (clipped to n), distinct uniform vertices,
    f~U{1..min(alpha,|e|)}."""
    rng = _rng(seed)
    sizes = rng.integers(smin, smax + 1, size=m)
    sizes = np.minimum(sizes, n).astype(np.int64)
    if m == 0:
        return _pack(n, sizes, np.zeros((0, 0), np.int64), np.zeros(0, np.int32), k, name, seed)
    rows, _ = _distinct_rows(rng, sizes, lambda shape: rng.integers(0, n, size=shape))
    dem = _demands(rng, sizes, alpha)
    return _pack(n, sizes, rows, dem, k, name, seed)


def config_uniform(seed: int = 0, n: int = 200, m: int = 400) -> Instance:
    """Plain single-instance workload: n=200, m=400, |e|~U{2..8}, f<=3, k=60."""
    return uniform_random(n, m, 2, 8, 3, 60, seed, name=f"uniform_n{n}_m{m}")


def config_powerlaw(seed: int = 0, n: int = 20000, m: int = 40000) -> Instance:
    """Large random workload with power-law sizes and Zipf(1.1) vertex popularity."""
    rng = _rng(seed)
    svals = np.arange(2, 65)
    ps = svals.astype(np.float64) ** -2.5
    ps /= ps.sum()
    sizes = rng.choice(svals, size=m, p=ps).astype(np.int64)
    sizes = np.minimum(sizes, n)
    perm = rng.permutation(n)
    pop = (np.arange(n, dtype=np.float64) + 1.0) ** -1.1
    cdf = np.cumsum(pop)
    cdf /= cdf[-1]

    def draw(shape):
        u = rng.random(size=shape)
        r = np.searchsorted(cdf, u, side="right")
        return perm[np.minimum(r, n - 1)]

    rows, _ = _distinct_rows(rng, sizes, draw)
    dem = _demands(rng, sizes, 4)
    return _pack(n, sizes, rows, dem, n // 10, f"powerlaw_n{n}_m{m}", seed)


def config_interval(seed: int = 0, n: int = 50000, m: int = 100000) -> Instance:
    """Interval hyperedges on a line with 5% noise (low Dilworth number)."""
    rng = _rng(seed)
    start = rng.integers(0, n, size=m)
    length = rng.geometric(1.0 / 12.0, size=m)
    end = np.minimum(start + length - 1, n - 1)
    length = end - start + 1
    lmax = int(length.max())
    col = np.arange(lmax)[None, :]
    valid = col < length[:, None]
    members = start[:, None] + col
    noise = rng.random(size=members.shape) < 0.05
    repl = rng.integers(0, n, size=members.shape)
    members = np.where(noise, repl, members)
    members = np.where(valid, members, np.iinfo(np.int64).max)
    members.sort(axis=1)
    # deduplicate within each row (a replacement may hit an existing member)
    dup = np.zeros_like(valid)
    dup[:, 1:] = (members[:, 1:] == members[:, :-1]) & valid[:, 1:]
    members = np.where(dup, np.iinfo(np.int64).max, members)
    members.sort(axis=1)
    sizes = (valid.sum(axis=1) - dup.sum(axis=1)).astype(np.int64)
    dem = _demands(rng, sizes, 2)
    return _pack(n, sizes, members, dem, n // 10, f"interval_n{n}_m{m}", seed)


def config_batch_one(seed: int) -> Instance:
    """One instance of the batched uneven workload."""
    rng = _rng(seed)
    n = int(rng.integers(50, 2001))
    m = int(rng.integers(n, 2 * n + 1))
    return uniform_random(n, m, 2, 16, 3, n // 10, seed + 7919, name=f"batch_{seed}")


def config_batch(count: int = 4096, seed0: int = 4000):
    """``count`` independent uneven instances; instance i uses seed seed0+i."""
    return [config_batch_one(seed0 + i) for i in range(count)]


def config_stream_one(seed: int) -> Instance:
    """One request of the serving stream: n log-uniform in [100, 20000]."""
    rng = _rng(seed)
    n = int(round(float(np.exp(rng.uniform(np.log(100.0), np.log(20000.0))))))
    m = int(rng.integers(n, 3 * n + 1))
    return uniform_random(n, m, 2, 16, 3, n // 10, seed + 104729, name=f"stream_{seed}")


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = _rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def tiny_random(seed: int, nmax: int = 16, mmax: int = 12) -> Instance:
    """Tiny instances for brute force: n<=16, sizes in [1,6], f in [1,|e|],
    with deliberate duplicate hyperedges and identical vertex columns so that
    the lowest-index tie-breaks are exercised."""
    rng = _rng(seed)
    n = int(rng.integers(1, nmax + 1))
    m = int(rng.integers(0, mmax + 1))
    edges = []
    for _ in range(m):
        s = int(rng.integers(1, min(6, n) + 1))
        edges.append(sorted(rng.choice(n, size=s, replace=False).tolist()))
    if m >= 2 and rng.random() < 0.5:  # duplicate hyperedge
        edges[int(rng.integers(0, m))] = list(edges[int(rng.integers(0, m))])
    if n >= 2 and rng.random() < 0.5:  # make vertex b a twin of vertex a
        a, b = rng.choice(n, size=2, replace=False).tolist()
        for e in edges:
            has_a = a in e
            if has_a and b not in e:
                e.append(b)
            elif not has_a and b in e:
                e.remove(b)
        edges = [sorted(e) if e else sorted([a, b]) for e in edges]
    if rng.random() < 0.2:  # occasionally an infeasible demand
        dem = [int(rng.integers(1, len(e) + 2)) for e in edges]
    else:
        dem = [int(rng.integers(1, len(e) + 1)) for e in edges]
    return from_edges(n, edges, dem, k=n, name=f"tiny_{seed}")


CONFIGS = {
    "uniform": config_uniform,
    "powerlaw": config_powerlaw,
    "interval": config_interval,
}

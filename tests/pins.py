"""Independent checks that pin the CPU oracle to the paper.

Nothing here calls the oracle or the CUDA library.  Each helper restates a
fact the paper fixes in a different form from the oracle's explicit pairwise
set tests:

* ``matrix_kernelize``  Algorithms 1-3 (Section 4.1) written literally with
  the intersection matrices of Eq. (1) and Eq. (2), I^E = A A^T and
  I^V = A^T A, in int64 numpy.
* ``fone_kernelize``    for f = 1 the two rules are Weihe's W1/W2
  (Section 1): a DP pass keeps the inclusion-minimal hyperedges, a MD pass
  keeps the vertices whose hyperedge sets are inclusion-maximal, equal
  items resolved to the lowest index (the tie-breaks of Algorithms 1 and 2).
* ``min_mhs_size``      brute force over all vertex subsets of the ILP model
  of Eq. (7) (Section 5.1), for n <= 16.
* ``matrix_kernelize_fe``  the same with rule FE applied to all full
  hyperedges at once between fixpoints (KernelGPU-FE, Section 5.1),
  where the oracle applies FE one hyperedge at a time as the rule states.
* ``matching_number``   the matching number of the incidence graph, which
  bounds the rounds by nu + 1 (proof of the parallel kernelization theorem,
  Section 4.1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import maximum_bipartite_matching


def dense_incidence(inst) -> np.ndarray:
    """A (m x n) of Section 2.1: A[i, j] = 1 iff v_j in e_i."""
    A = np.zeros((inst.m, inst.n), dtype=np.int64)
    for i in range(inst.m):
        A[i, inst.edge_vtx[inst.edge_ptr[i]:inst.edge_ptr[i + 1]]] = 1
    return A


def matrix_rounds(A, f, alive_v, alive_e, max_rounds: int = 0, rule: str = "dp"):
    """Algorithm 3 with Algorithms 1 and 2 in their matrix form, from the
    state (alive_v, alive_e) with demands f; updates the masks in place.

    rule "dp": D_ij = [f_i - (I^E_ii - I^E_ij) >= f_j] (Algorithm 1);
    rule "se": D_ij = [I^E_ij = I^E_ii and f_i >= f_j] (rule SE: e_i is a
    subset of e_j exactly when their intersection is all of e_i).
    Returns (rounds, trace) with trace rows
    [edges deleted by DP, vertices deleted by MD, alive edges, alive vertices].
    """
    f = np.asarray(f, dtype=np.int64)
    trace = []
    rounds = 0
    while True:
        # Algorithm 1 on the current incidence matrix
        E = np.nonzero(alive_e)[0]
        V = np.nonzero(alive_v)[0]
        Ac = A[np.ix_(E, V)]
        IE = Ac @ Ac.T                                   # Eq. (1)
        s = np.diag(IE)
        fe = f[E]
        if rule == "se":
            D = (IE == s[:, None]) & (fe[:, None] >= fe[None, :])
        else:
            D = (fe[:, None] - (s[:, None] - IE)) >= fe[None, :]   # D_ij
        np.fill_diagonal(D, False)
        idx = np.arange(E.size)
        i_lt_j = idx[:, None] < idx[None, :]
        R_del = (D & (~D.T | i_lt_j)).any(axis=0)         # some i deletes j
        de = int(R_del.sum())
        alive_e[E[R_del]] = False
        # Algorithm 2 on the output of Algorithm 1
        E = np.nonzero(alive_e)[0]
        Ac = A[np.ix_(E, V)]
        IV = Ac.T @ Ac                                   # Eq. (2)
        d = np.diag(IV)
        vidx = np.arange(V.size)
        v_lt = vidx[:, None] < vidx[None, :]
        Dv = (IV == d[None, :]) & ((IV != d[:, None]) | v_lt)   # D_ij
        np.fill_diagonal(Dv, False)
        C = Dv.sum(axis=0)                               # C = 1^T D
        fe = f[E]
        # v_j deleted iff every hyperedge e_i containing it has C_j >= f(e_i)
        ok = (Ac == 0) | (C[None, :] >= fe[:, None])
        V_del = ok.all(axis=0)
        dv = int(V_del.sum())
        alive_v[V[V_del]] = False
        rounds += 1
        trace.append([de, dv, int(alive_e.sum()), int(alive_v.sum())])
        if de + dv == 0 or (max_rounds > 0 and rounds >= max_rounds):
            break
    return rounds, np.array(trace, dtype=np.int64)


def matrix_kernelize(inst, max_rounds: int = 0, rule: str = "dp"):
    """Algorithm 3 with Algorithms 1 and 2 in their matrix form.

    Returns (alive_v, alive_e, rounds, trace) with trace rows
    [edges deleted by DP, vertices deleted by MD, alive edges, alive vertices].
    """
    A = dense_incidence(inst)
    alive_e = np.ones(inst.m, dtype=bool)
    alive_v = np.ones(inst.n, dtype=bool)
    rounds, trace = matrix_rounds(A, inst.demand, alive_v, alive_e, max_rounds, rule)
    return alive_v, alive_e, rounds, trace


def full_edges_at_once(A, f, alive_v, alive_e):
    """Exhaustive FE (Section 3.1) as ONE simultaneous step: S = all alive
    vertices of all full hyperedges (|e| = f(e)); every other alive
    hyperedge loses |e & S| demand and goes at demand <= 0.  Updates f and
    the masks in place; returns the bool mask S."""
    Ac = A * alive_v[None, :]
    size = Ac.sum(axis=1)
    full = alive_e & (size == f)
    S = alive_v & (Ac[full].sum(axis=0) > 0)
    lost = Ac[:, S].sum(axis=1)
    rest = alive_e & ~full
    f[rest] -= lost[rest]
    alive_e[full] = False
    alive_e[rest & (f <= 0)] = False
    alive_v[S] = False
    return S


def matrix_kernelize_fe(inst, rule: str = "dp"):
    """KernelGPU-FE (Section 5.1): Algorithm 3 in matrix form to its fixpoint,
    then FE at once, until FE finds no full hyperedge.  Returns a dict like
    the oracle's reduce_variant."""
    A = dense_incidence(inst)
    f = np.asarray(inst.demand, dtype=np.int64).copy()
    alive_e = np.ones(inst.m, dtype=bool)
    alive_v = np.ones(inst.n, dtype=bool)
    forced = np.zeros(inst.n, dtype=bool)
    rounds = passes = 0
    while True:
        r, _ = matrix_rounds(A, f, alive_v, alive_e, 0, rule)
        rounds += r
        passes += 1
        S = full_edges_at_once(A, f, alive_v, alive_e)
        if not S.any():  # f >= 1, so a full hyperedge has a vertex
            break
        forced |= S
    E = np.nonzero(alive_e)[0]
    return {"vertices": np.nonzero(alive_v)[0].tolist(), "edges": E.tolist(),
            "demands": f[E].tolist(), "k": int(inst.k) - int(forced.sum()),
            "forced": np.nonzero(forced)[0].tolist(), "rounds": rounds, "fe_passes": passes}


def fone_kernelize(inst):
    """Exhaustive W1/W2 (f = 1) with lowest-index tie-breaks, by set algebra."""
    edges = {i: frozenset(e) for i, e in enumerate(inst.edges())}
    verts = set(range(inst.n))
    rounds = 0
    while True:
        # W2 pass: keep e_j unless some e_i is a proper subset, or an equal
        # hyperedge has a lower index.
        cur = {i: e & verts for i, e in edges.items()}
        drop_e = {j for j, ej in cur.items()
                  if any((ei < ej) or (ei == ej and i < j)
                         for i, ei in cur.items() if i != j)}
        for j in drop_e:
            del edges[j]
        # W1 pass: E(v) over the remaining hyperedges; keep v_j unless some
        # other vertex has a proper superset, or an equal set and lower index.
        # A vertex in no hyperedge is deleted (maximum demand over nothing is 0).
        Ev = {v: frozenset(i for i, e in edges.items() if v in e) for v in verts}
        drop_v = set()
        for j in verts:
            if not Ev[j]:
                drop_v.add(j)
                continue
            if any((Ev[j] < Ev[i]) or (Ev[j] == Ev[i] and i < j)
                   for i in verts if i != j):
                drop_v.add(j)
        verts -= drop_v
        rounds += 1
        if not drop_e and not drop_v:
            break
    return sorted(verts), sorted(edges), rounds


def min_mhs_size(n: int, edges, demand, allowed=None):
    """Minimum |S| with |e & S| >= f(e) for all e (Eq. (7)), S within
    ``allowed`` (default: all n vertices).  None if infeasible.  n <= 16."""
    assert n <= 20
    subsets = np.arange(1 << n, dtype=np.uint32)
    ok = np.ones(subsets.size, dtype=bool)
    if allowed is not None:
        amask = 0
        for v in allowed:
            amask |= 1 << int(v)
        ok &= (subsets & np.uint32(~amask & ((1 << n) - 1))) == 0
    for e, fe in zip(edges, demand):
        emask = 0
        for v in e:
            emask |= 1 << int(v)
        ok &= np.bitwise_count(subsets & np.uint32(emask)) >= fe
    if not ok.any():
        return None
    return int(np.bitwise_count(subsets[ok]).min())


def matching_number(inst) -> int:
    """Maximum matching in the incidence graph I(H) (Section 2.1)."""
    if inst.m == 0 or inst.n == 0 or inst.nnz == 0:
        return 0
    data = np.ones(inst.nnz, dtype=np.int8)
    g = sp.csr_matrix((data, inst.edge_vtx, inst.edge_ptr), shape=(inst.m, inst.n))
    match = maximum_bipartite_matching(g, perm_type="column")
    return int((match >= 0).sum())


def supersedes_sets(e_i: set, e_j: set, f_i: int, f_j: int) -> bool:
    """Definition of supersedence (Section 3.1)."""
    return f_i - len(e_i - e_j) >= f_j

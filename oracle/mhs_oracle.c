/*
 * mhs_oracle.c -- CPU oracle for the exhaustive DP + MD kernelization.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this file's library; the product path
 * never calls it.  It shares no code, header or table with the CUDA path.
 *
 * It is a plain, single-threaded restatement of the paper's round-based
 * reduction, written from the definitions rather than from the matrix
 * formulation the GPU uses:
 *
 *   Definition (supersedes), Section 3.1: e_i supersedes e_j iff
 *       f(e_i) - |e_i \ e_j| >= f(e_j).
 *   Definition (dominates), Section 3.1: v_i dominates v_j iff
 *       E(v_j) is a subset of E(v_i).
 *   Algorithm 1 (exhaustive DP): with D_ij = [e_i supersedes e_j], delete
 *       e_j iff some i != j has D_ij and (not D_ji or i < j); all deletions
 *       of one pass happen at once.
 *   Algorithm 2 (exhaustive MD): with D_ij = [v_i dominates v_j and
 *       (v_j does not dominate v_i or i < j)], C_j = sum_i D_ij, delete v_j
 *       iff C_j >= max_{e in E(v_j)} f(e) (the maximum over the empty set
 *       is 0, so a vertex in no hyperedge is deleted); all at once.
 *   Algorithm 3: repeat { Algorithm 1; then Algorithm 2 on its output }
 *       while the hypergraph changes.  The round count includes the final
 *       pass that changes nothing.
 *
 * Set differences and subset tests are explicit merges of sorted lists,
 * restricted to the items still alive.  Indices are the input indices:
 * deleting items never renumbers the others, so "i < j" is the input order.
 *
 * Optional exact pruning (prune != 0) only skips pairs whose test is known
 * to be false:
 *   DP: if e_i and e_j share no alive vertex, |e_i \ e_j| = |e_i| and
 *       e_i supersedes e_j only if f(e_i) - |e_i| >= f(e_j) >= 1.  So the
 *       candidates for e_j are the hyperedges meeting e_j plus the few with
 *       f(e_i) > |e_i|.
 *   MD: a dominator of v_j (E(v_j) non-empty) lies in every hyperedge of
 *       E(v_j), in particular in the first one.
 * prune == 0 scans all pairs; the tests check that both agree.
 *
 * Two further rules of Section 3.1, for the variants of the experiments:
 *   SE (superedge rule): e_j goes if some distinct e_i is a subset of e_j
 *       with f(e_i) >= f(e_j).  The "MD+SE" variant runs Algorithm 3 with
 *       this test in place of "e_i supersedes e_j" (same simultaneous
 *       deletions and lowest-index tie-break).  The pruning above stays
 *       exact: a non-empty e_i inside e_j meets e_j, and an empty e_i has
 *       f(e_i) > |e_i|.
 *   FE (full-edge rule): while some alive e_j has |e_j| = f(e_j), take the
 *       lowest such j, delete e_j and each alive v in e_j (v goes into the
 *       solution, k drops by one), lower f of every other alive hyperedge
 *       holding v by one and delete those whose demand reaches 0.
 *   KernelGPU-FE (Section 5.1): alternate Algorithm 3 to its fixpoint and
 *       exhaustive FE until FE changes nothing.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n, m;
    const int32_t *eptr, *evtx, *f;
    int32_t *vptr, *vedg; /* vertex -> hyperedges, ascending */
    int32_t rule;         /* 0: DP (supersedes), 1: SE (subset, f_i >= f_j) */
} hyper_t;

enum { RULE_DP = 0, RULE_SE = 1 };

static int build_incidence(hyper_t *h) {
    int32_t n = h->n, m = h->m;
    h->vptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t nnz = h->eptr[m];
    h->vedg = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!h->vptr || !h->vedg) return -1;
    for (int32_t e = 0; e < m; ++e)
        for (int32_t p = h->eptr[e]; p < h->eptr[e + 1]; ++p) h->vptr[h->evtx[p] + 1]++;
    for (int32_t v = 0; v < n; ++v) h->vptr[v + 1] += h->vptr[v];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!fill) return -1;
    memcpy(fill, h->vptr, sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t e = 0; e < m; ++e) /* ascending e => ascending lists */
        for (int32_t p = h->eptr[e]; p < h->eptr[e + 1]; ++p) h->vedg[fill[h->evtx[p]]++] = e;
    free(fill);
    return 0;
}

static void free_incidence(hyper_t *h) {
    free(h->vptr);
    free(h->vedg);
}

/* |e_i \ e_j| over alive vertices (sorted-list merge). */
static int32_t diff_size(const hyper_t *h, const uint8_t *alive_v, int32_t i, int32_t j) {
    int32_t a = h->eptr[i], ae = h->eptr[i + 1];
    int32_t b = h->eptr[j], be = h->eptr[j + 1];
    int32_t d = 0;
    while (a < ae) {
        int32_t x = h->evtx[a];
        if (!alive_v[x]) { ++a; continue; }
        while (b < be && h->evtx[b] < x) ++b;
        int in_j = (b < be && h->evtx[b] == x && alive_v[x]);
        if (!in_j) ++d;
        ++a;
    }
    return d;
}

/* e_i supersedes e_j (Definition in Section 3.1); under rule SE: e_i is a
   subset of e_j and f(e_i) >= f(e_j) (rule SE, Section 3.1). */
static int supersedes(const hyper_t *h, const uint8_t *alive_v, int32_t i, int32_t j) {
    if (h->rule == RULE_SE) {
#ifdef ORACLE_MUTANT_SE_IGNORE_DEMAND
        return diff_size(h, alive_v, i, j) == 0;
#elif defined(ORACLE_MUTANT_SE_DEMAND_REVERSED)
        return diff_size(h, alive_v, i, j) == 0 && h->f[i] <= h->f[j];
#else
        return diff_size(h, alive_v, i, j) == 0 && h->f[i] >= h->f[j];
#endif
    }
#ifdef ORACLE_MUTANT_DP_TRANSPOSED
    return h->f[i] - diff_size(h, alive_v, j, i) >= h->f[j];
#elif defined(ORACLE_MUTANT_DP_DROP_FI)
    return h->f[j] - diff_size(h, alive_v, i, j) >= h->f[j];
#else
    return h->f[i] - diff_size(h, alive_v, i, j) >= h->f[j];
#endif
}

/* v_i dominates v_j: E(v_j) subset of E(v_i), over alive hyperedges. */
static int dominates(const hyper_t *h, const uint8_t *alive_e, int32_t i, int32_t j) {
    int32_t a = h->vptr[j], ae = h->vptr[j + 1]; /* E(v_j) */
    int32_t b = h->vptr[i], be = h->vptr[i + 1]; /* E(v_i) */
    while (a < ae) {
        int32_t e = h->vedg[a++];
        if (!alive_e[e]) continue;
        while (b < be && h->vedg[b] < e) ++b;
        if (b >= be || h->vedg[b] != e) return 0;
    }
    return 1;
}

static int32_t alive_size(const hyper_t *h, const uint8_t *alive_v, int32_t e) {
    int32_t s = 0;
    for (int32_t p = h->eptr[e]; p < h->eptr[e + 1]; ++p) s += alive_v[h->evtx[p]] != 0;
    return s;
}

/* Does e_i cause the deletion of e_j in Algorithm 1? */
static int dp_arc(const hyper_t *h, const uint8_t *alive_v, int32_t i, int32_t j) {
    if (!supersedes(h, alive_v, i, j)) return 0;
#ifdef ORACLE_MUTANT_DP_TIEBREAK_HIGH
    return !supersedes(h, alive_v, j, i) || i > j;
#elif defined(ORACLE_MUTANT_DP_NO_TIEBREAK)
    return 1;
#else
    return !supersedes(h, alive_v, j, i) || i < j;
#endif
}

/*
 * One pass of Algorithm 1.  del_e[j] is set to 1 for every alive e_j that
 * the pass deletes (and left 0 otherwise); alive arrays are not modified.
 * Returns the number of deleted hyperedges.
 */
static int32_t dp_pass(const hyper_t *h, const uint8_t *alive_v, const uint8_t *alive_e,
                       int prune, uint8_t *del_e) {
    int32_t m = h->m, count = 0;
    memset(del_e, 0, (size_t)m);
    if (!prune) {
        for (int32_t j = 0; j < m; ++j) {
            if (!alive_e[j]) continue;
            for (int32_t i = 0; i < m; ++i) {
                if (i == j || !alive_e[i]) continue;
                if (dp_arc(h, alive_v, i, j)) { del_e[j] = 1; ++count; break; }
            }
        }
        return count;
    }
    /* loose hyperedges: f(e) > |e| over alive vertices */
    int32_t *loose = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int32_t nloose = 0;
    for (int32_t i = 0; i < m; ++i)
        if (alive_e[i] && h->f[i] > alive_size(h, alive_v, i)) loose[nloose++] = i;
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    for (int32_t i = 0; i < m; ++i) mark[i] = -1;
    for (int32_t j = 0; j < m; ++j) {
        if (!alive_e[j]) continue;
        int hit = 0;
        for (int32_t p = h->eptr[j]; p < h->eptr[j + 1] && !hit; ++p) {
            int32_t v = h->evtx[p];
            if (!alive_v[v]) continue;
            for (int32_t q = h->vptr[v]; q < h->vptr[v + 1]; ++q) {
                int32_t i = h->vedg[q];
                if (i == j || !alive_e[i] || mark[i] == j) continue;
                mark[i] = j;
                if (dp_arc(h, alive_v, i, j)) { hit = 1; break; }
            }
        }
        for (int32_t t = 0; t < nloose && !hit; ++t) {
            int32_t i = loose[t];
            if (i == j || mark[i] == j) continue;
            mark[i] = j;
            if (dp_arc(h, alive_v, i, j)) hit = 1;
        }
        if (hit) { del_e[j] = 1; ++count; }
    }
    free(mark);
    free(loose);
    return count;
}

/* D_ij of Algorithm 2: v_i dominates v_j, ties broken towards lower index. */
static int md_arc(const hyper_t *h, const uint8_t *alive_e, int32_t i, int32_t j) {
    if (!dominates(h, alive_e, i, j)) return 0;
#ifdef ORACLE_MUTANT_MD_STRICT_ONLY
    return !dominates(h, alive_e, j, i);
#elif defined(ORACLE_MUTANT_MD_TIEBREAK_HIGH)
    return !dominates(h, alive_e, j, i) || i > j;
#else
    return !dominates(h, alive_e, j, i) || i < j;
#endif
}

static int32_t max_demand(const hyper_t *h, const uint8_t *alive_e, int32_t j) {
    int32_t mx = 0;
    for (int32_t q = h->vptr[j]; q < h->vptr[j + 1]; ++q) {
        int32_t e = h->vedg[q];
#ifdef ORACLE_MUTANT_MD_MAXF_ALL_EDGES
        if (h->f[e] > mx) mx = h->f[e];
#else
        if (alive_e[e] && h->f[e] > mx) mx = h->f[e];
#endif
    }
    return mx;
}

/*
 * One pass of Algorithm 2 on the hypergraph (alive_v, alive_e).
 * Sets del_v[j] = 1 for every deleted vertex; returns their number.
 * If cnt is non-NULL it receives C_j (only for alive vertices that have at
 * least one alive hyperedge; 0 otherwise) and maxf receives the maximum
 * demand over E(v_j).
 */
static int32_t md_pass(const hyper_t *h, const uint8_t *alive_v, const uint8_t *alive_e,
                       int prune, uint8_t *del_v, int32_t *cnt_out, int32_t *maxf_out) {
    int32_t n = h->n, count = 0;
    memset(del_v, 0, (size_t)n);
    for (int32_t j = 0; j < n; ++j) {
        if (cnt_out) cnt_out[j] = 0;
        if (maxf_out) maxf_out[j] = 0;
        if (!alive_v[j]) continue;
        int32_t maxf = max_demand(h, alive_e, j);
        if (maxf_out) maxf_out[j] = maxf;
        int32_t c = 0;
        int32_t first = -1; /* first alive hyperedge containing v_j */
        for (int32_t q = h->vptr[j]; q < h->vptr[j + 1]; ++q)
            if (alive_e[h->vedg[q]]) { first = h->vedg[q]; break; }
        if (!prune || first < 0) {
            if (first < 0 && prune) {
                c = 0; /* E(v_j) empty: maxf = 0 <= C_j, deleted whatever C_j is */
            } else {
                for (int32_t i = 0; i < n; ++i)
                    if (i != j && alive_v[i] && md_arc(h, alive_e, i, j)) ++c;
            }
        } else {
            for (int32_t p = h->eptr[first]; p < h->eptr[first + 1]; ++p) {
                int32_t i = h->evtx[p];
                if (i != j && alive_v[i] && md_arc(h, alive_e, i, j)) ++c;
            }
        }
        if (cnt_out && first >= 0) cnt_out[j] = c;
#ifdef ORACLE_MUTANT_MD_STRICT_GT
        int del = (c > maxf) || first < 0;
#elif defined(ORACLE_MUTANT_MD_KEEP_ISOLATED)
        int del = first >= 0 && c >= maxf;
#else
        int del = c >= maxf;
#endif
        if (del) { del_v[j] = 1; ++count; }
    }
    return count;
}

/* ---------------------------------------------------------------------- */
/* exported entry points (ctypes)                                          */
/* ---------------------------------------------------------------------- */

/*
 * Run Algorithm 3 from the state (alive_v, alive_e), updating them in place.
 * max_rounds <= 0: until a round changes nothing; otherwise at most
 * max_rounds rounds.  *rounds_out = rounds executed (each a DP pass then an
 * MD pass); *changed_out = whether the last executed round deleted anything.
 * If trace != NULL it receives, per executed round r, four int32 values:
 * [edges deleted by DP, vertices deleted by MD, alive edges, alive vertices]
 * (at most trace_cap rounds are recorded).  Returns 0, or -1 on allocation
 * failure.
 */
static int algorithm3(hyper_t *hp, int32_t max_rounds, int32_t prune, uint8_t *alive_v,
                      uint8_t *alive_e, int32_t *rounds_out, int32_t *changed_out,
                      int32_t *trace, int32_t trace_cap) {
    hyper_t h = *hp;
    const int32_t n = h.n, m = h.m;
    uint8_t *del_e = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
    uint8_t *del_v = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!del_e || !del_v) { free(del_e); free(del_v); return -1; }
    int32_t rounds = 0, changed = 0;
    int32_t alive_m = 0, alive_n = 0;
    for (int32_t e = 0; e < m; ++e) alive_m += alive_e[e] != 0;
    for (int32_t v = 0; v < n; ++v) alive_n += alive_v[v] != 0;
    do {
        int32_t de = dp_pass(&h, alive_v, alive_e, prune, del_e);
#ifdef ORACLE_MUTANT_SEQUENTIAL_MD_BEFORE_DP
        int32_t dv = 0;
        (void)de;
        dv = md_pass(&h, alive_v, alive_e, prune, del_v, NULL, NULL);
        for (int32_t v = 0; v < n; ++v) if (del_v[v]) alive_v[v] = 0;
        de = dp_pass(&h, alive_v, alive_e, prune, del_e);
        for (int32_t e = 0; e < m; ++e) if (del_e[e]) alive_e[e] = 0;
#else
        for (int32_t e = 0; e < m; ++e) if (del_e[e]) alive_e[e] = 0;
        int32_t dv = md_pass(&h, alive_v, alive_e, prune, del_v, NULL, NULL);
        for (int32_t v = 0; v < n; ++v) if (del_v[v]) alive_v[v] = 0;
#endif
        alive_m -= de;
        alive_n -= dv;
        if (trace && rounds < trace_cap) {
            trace[4 * rounds + 0] = de;
            trace[4 * rounds + 1] = dv;
            trace[4 * rounds + 2] = alive_m;
            trace[4 * rounds + 3] = alive_n;
        }
        ++rounds;
        changed = (de + dv) > 0;
    } while (changed && (max_rounds <= 0 || rounds < max_rounds));
    *rounds_out = rounds;
    *changed_out = changed;
    free(del_e);
    free(del_v);
    return 0;
}

int mhs_oracle_reduce(int32_t n, int32_t m, const int32_t *edge_ptr, const int32_t *edge_vtx,
                      const int32_t *demand, int32_t max_rounds, int32_t prune,
                      uint8_t *alive_v, uint8_t *alive_e, int32_t *rounds_out,
                      int32_t *changed_out, int32_t *trace, int32_t trace_cap) {
    hyper_t h = {n, m, edge_ptr, edge_vtx, demand, NULL, NULL, RULE_DP};
    if (build_incidence(&h)) return -1;
    int rc = algorithm3(&h, max_rounds, prune, alive_v, alive_e, rounds_out, changed_out, trace,
                        trace_cap);
    free_incidence(&h);
    return rc;
}

/*
 * Exhaustive FE (rule FE, Section 3.1), one full hyperedge at a time in
 * increasing index order, on the state (alive_v, alive_e, f).  f is the
 * current demand per hyperedge (updated), forced[v] is set for every vertex
 * the rule puts into the solution, *k is lowered by their number.  Returns
 * the number of hyperedges and vertices deleted.
 */
static int32_t fe_exhaustive(const hyper_t *h, uint8_t *alive_v, uint8_t *alive_e, int32_t *f,
                             uint8_t *forced, int64_t *k) {
    int32_t deleted = 0;
    for (;;) {
        int32_t j = -1;
        for (int32_t e = 0; e < h->m && j < 0; ++e)
            if (alive_e[e] && alive_size(h, alive_v, e) == f[e]) j = e;
        if (j < 0) return deleted;
        alive_e[j] = 0;
        ++deleted;
        for (int32_t p = h->eptr[j]; p < h->eptr[j + 1]; ++p) {
            const int32_t v = h->evtx[p];
            if (!alive_v[v]) continue;
            alive_v[v] = 0;
            forced[v] = 1;
#ifndef ORACLE_MUTANT_FE_K_UNCHANGED
            *k -= 1;
#endif
            ++deleted;
            for (int32_t q = h->vptr[v]; q < h->vptr[v + 1]; ++q) {
                const int32_t i = h->vedg[q];
                if (!alive_e[i]) continue;
#ifndef ORACLE_MUTANT_FE_SKIP_DECREMENT
                f[i] -= 1;
#endif
#ifndef ORACLE_MUTANT_FE_KEEP_ZERO_DEMAND
                if (f[i] == 0) { alive_e[i] = 0; ++deleted; }
#endif
            }
        }
    }
}

/*
 * The reduction variants of the experiments (Section 5.1), from the input
 * state (everything alive):
 *   rule 0 / 1: Algorithm 3 with DP or SE as the hyperedge pass;
 *   full_edges != 0: alternate that to its fixpoint with exhaustive FE
 *   until FE changes nothing (KernelGPU-FE).
 * Outputs: alive masks, current demands f_out[m] (input demands unless FE
 * lowered them), forced_v[n] (vertices FE put into the solution), *k_out,
 * *rounds_out (Algorithm 3 rounds over all alternations, each run counting
 * its final round that changes nothing), *fe_passes_out (FE applications,
 * counting the last one that changes nothing; 0 without FE).  max_rounds
 * bounds Algorithm 3 when full_edges == 0 and is ignored otherwise.
 */
int mhs_oracle_reduce_ext(int32_t n, int32_t m, const int32_t *edge_ptr, const int32_t *edge_vtx,
                          const int32_t *demand, int64_t k, int32_t rule, int32_t full_edges,
                          int32_t max_rounds, int32_t prune, uint8_t *alive_v, uint8_t *alive_e,
                          int32_t *f_out, uint8_t *forced_v, int64_t *k_out,
                          int32_t *rounds_out, int32_t *fe_passes_out, int32_t *changed_out) {
    for (int32_t e = 0; e < m; ++e) f_out[e] = demand[e];
    for (int32_t v = 0; v < n; ++v) forced_v[v] = 0;
    hyper_t h = {n, m, edge_ptr, edge_vtx, f_out, NULL, NULL, rule};
    if (build_incidence(&h)) return -1;
    int32_t rounds = 0, passes = 0, changed = 0;
    int rc = 0;
    for (;;) {
        int32_t r = 0;
        rc = algorithm3(&h, full_edges ? 0 : max_rounds, prune, alive_v, alive_e, &r, &changed,
                        NULL, 0);
        rounds += r;
        if (rc || !full_edges) break;
        ++passes;
        if (fe_exhaustive(&h, alive_v, alive_e, f_out, forced_v, &k) == 0) break;
#ifdef ORACLE_MUTANT_FE_NO_ALTERNATION
        ++passes;
        break;
#endif
    }
    *k_out = k;
    *rounds_out = rounds;
    *fe_passes_out = passes;
    *changed_out = changed;
    free_incidence(&h);
    return rc;
}

/* One Algorithm 1 pass: del_e[j] = 1 for deleted hyperedges. Returns count or -1. */
int mhs_oracle_dp_pass(int32_t n, int32_t m, const int32_t *edge_ptr, const int32_t *edge_vtx,
                       const int32_t *demand, int32_t prune, const uint8_t *alive_v,
                       const uint8_t *alive_e, uint8_t *del_e) {
    hyper_t h = {n, m, edge_ptr, edge_vtx, demand, NULL, NULL, RULE_DP};
    if (build_incidence(&h)) return -1;
    int32_t c = dp_pass(&h, alive_v, alive_e, prune, del_e);
    free_incidence(&h);
    return c;
}

/* One Algorithm 2 pass: del_v[j] = 1 for deleted vertices; cnt/maxf as in md_pass. */
int mhs_oracle_md_pass(int32_t n, int32_t m, const int32_t *edge_ptr, const int32_t *edge_vtx,
                       const int32_t *demand, int32_t prune, const uint8_t *alive_v,
                       const uint8_t *alive_e, uint8_t *del_v, int32_t *cnt, int32_t *maxf) {
    hyper_t h = {n, m, edge_ptr, edge_vtx, demand, NULL, NULL, RULE_DP};
    if (build_incidence(&h)) return -1;
    int32_t c = md_pass(&h, alive_v, alive_e, prune, del_v, cnt, maxf);
    free_incidence(&h);
    return c;
}

/* Pairwise relations on a state, for invariant tests. */
int mhs_oracle_supersedes(int32_t n, int32_t m, const int32_t *edge_ptr, const int32_t *edge_vtx,
                          const int32_t *demand, const uint8_t *alive_v, int32_t i, int32_t j) {
    hyper_t h = {n, m, edge_ptr, edge_vtx, demand, NULL, NULL, RULE_DP};
    return supersedes(&h, alive_v, i, j);
}

int mhs_oracle_dominates(int32_t n, int32_t m, const int32_t *edge_ptr, const int32_t *edge_vtx,
                         const uint8_t *alive_e, int32_t i, int32_t j) {
    hyper_t h = {n, m, edge_ptr, edge_vtx, NULL, NULL, NULL, RULE_DP};
    if (build_incidence(&h)) return -1;
    int r = dominates(&h, alive_e, i, j);
    free_incidence(&h);
    return r;
}

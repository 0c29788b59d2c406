/*
 * mhs_kernelcpu.c -- the paper's sequential design for exhaustive DP + MD
 * (Section 4.2, Algorithms 4-6), as a CPU baseline and an independent third
 * implementation for the parity tests.
 *
 * TEST AND BASELINE INFRASTRUCTURE ONLY: the tests and the benchmark's CPU
 * baseline call it; the product path never does.  It shares no code with
 * the CUDA path or with the pairwise oracle.
 *
 * What it computes (written from the description in Section 4.2):
 *   - I^E = A A^T and I^V = A^T A are built once by enumerating, for every
 *     vertex, the pairs of its hyperedges and, for every hyperedge, the
 *     pairs of its vertices (Eq. (1), Eq. (2)).
 *   - A DP pass (Algorithm 4) tests every alive e_j against the candidate
 *     superseders in P^E with D_ij = [f_i - (I^E_ii - I^E_ij) >= f_j] and the
 *     lowest-index tie-break of Algorithm 1, collects the deleted
 *     hyperedges, then removes them at once: each removal decrements I^V
 *     over the vertex pairs of the hyperedge and puts its vertices into P^V.
 *     P^E is emptied.
 *   - An MD pass (Algorithm 5) counts, for every alive v_j in P^V, the
 *     dominators i with I_ij = I_jj and (I_ij != I_ii or i < j) until it
 *     reaches max f over E(v_j); removals decrement I^E over the hyperedge
 *     pairs of the vertex and put those hyperedges into P^E.  P^V is emptied.
 *   - Algorithm 6 starts with P^E and P^V holding everything and alternates
 *     the two passes until neither removes anything.
 * One reading differs from the printed Algorithm 5: a vertex in no alive
 * hyperedge is deleted (maximum demand over nothing is 0), as in
 * Algorithm 2, so that this implementation and the parallel one agree.
 *
 * The count matrices are dense (m^2 + n^2 entries of 16 or 32 bits), as in
 * the paper; instances whose matrices exceed max_bytes are refused.  With
 * threads > 1 the independent tests of a pass run in parallel (OpenMP); the
 * removals stay sequential.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t n, m;
    const int32_t *eptr, *evtx, *f;
    int32_t *vptr, *vedg;
    int wide;          /* 1: 32-bit counts, 0: 16-bit */
    void *IE, *IV;     /* m*m and n*n */
} kc_t;

static inline uint32_t ie_get(const kc_t *k, int64_t i, int64_t j) {
    return k->wide ? ((uint32_t *)k->IE)[i * k->m + j] : ((uint16_t *)k->IE)[i * k->m + j];
}
static inline uint32_t iv_get(const kc_t *k, int64_t i, int64_t j) {
    return k->wide ? ((uint32_t *)k->IV)[i * k->n + j] : ((uint16_t *)k->IV)[i * k->n + j];
}
static inline void ie_add(kc_t *k, int64_t i, int64_t j, int d) {
    if (k->wide) ((uint32_t *)k->IE)[i * k->m + j] += d;
    else ((uint16_t *)k->IE)[i * k->m + j] += d;
}
static inline void iv_add(kc_t *k, int64_t i, int64_t j, int d) {
    if (k->wide) ((uint32_t *)k->IV)[i * k->n + j] += d;
    else ((uint16_t *)k->IV)[i * k->n + j] += d;
}

static int build_csc(kc_t *k) {
    k->vptr = (int32_t *)calloc((size_t)k->n + 1, sizeof(int32_t));
    int32_t nnz = k->eptr[k->m];
    k->vedg = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * ((size_t)k->n + 1));
    if (!k->vptr || !k->vedg || !fill) { free(fill); return -1; }
    for (int32_t e = 0; e < k->m; ++e)
        for (int32_t p = k->eptr[e]; p < k->eptr[e + 1]; ++p) k->vptr[k->evtx[p] + 1]++;
    for (int32_t v = 0; v < k->n; ++v) k->vptr[v + 1] += k->vptr[v];
    memcpy(fill, k->vptr, sizeof(int32_t) * ((size_t)k->n + 1));
    for (int32_t e = 0; e < k->m; ++e)
        for (int32_t p = k->eptr[e]; p < k->eptr[e + 1]; ++p) k->vedg[fill[k->evtx[p]]++] = e;
    free(fill);
    return 0;
}

/* Candidate lists with membership flags (each index at most once). */
typedef struct {
    int32_t *items;
    uint8_t *in;
    int32_t len;
} cand_t;

static void cand_add(cand_t *c, int32_t x) {
    if (!c->in[x]) {
        c->in[x] = 1;
        c->items[c->len++] = x;
    }
}
static void cand_clear(cand_t *c) {
    for (int32_t t = 0; t < c->len; ++t) c->in[c->items[t]] = 0;
    c->len = 0;
}

/*
 * Returns 0 on success, -1 on allocation failure, -2 if the dense count
 * matrices would exceed max_bytes.  alive_v / alive_e receive the result,
 * *rounds_out the number of passes pairs (DP then MD) executed, counting the
 * final one that removes nothing.
 */
int mhs_kernelcpu(int32_t n, int32_t m, const int32_t *edge_ptr, const int32_t *edge_vtx,
                  const int32_t *demand, int64_t max_bytes, int32_t threads, uint8_t *alive_v,
                  uint8_t *alive_e, int32_t *rounds_out) {
    kc_t k;
    memset(&k, 0, sizeof(k));
    k.n = n;
    k.m = m;
    k.eptr = edge_ptr;
    k.evtx = edge_vtx;
    k.f = demand;
    if (build_csc(&k)) return -1;
    int32_t max_size = 0, max_deg = 0;
    for (int32_t e = 0; e < m; ++e)
        if (edge_ptr[e + 1] - edge_ptr[e] > max_size) max_size = edge_ptr[e + 1] - edge_ptr[e];
    for (int32_t v = 0; v < n; ++v)
        if (k.vptr[v + 1] - k.vptr[v] > max_deg) max_deg = k.vptr[v + 1] - k.vptr[v];
    k.wide = (max_size >= 65535 || max_deg >= 65535);
    const int64_t esz = k.wide ? 4 : 2;
    const int64_t need = esz * ((int64_t)m * m + (int64_t)n * n);
    if (need > max_bytes) {
        free(k.vptr);
        free(k.vedg);
        return -2;
    }
    k.IE = calloc((size_t)m * (size_t)m + 1, (size_t)esz);
    k.IV = calloc((size_t)n * (size_t)n + 1, (size_t)esz);
    uint8_t *RE = (uint8_t *)malloc((size_t)m + 1), *RV = (uint8_t *)malloc((size_t)n + 1);
    cand_t PE = {(int32_t *)malloc(sizeof(int32_t) * ((size_t)m + 1)), (uint8_t *)calloc((size_t)m + 1, 1), 0};
    cand_t PV = {(int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1)), (uint8_t *)calloc((size_t)n + 1, 1), 0};
    int32_t *Q = (int32_t *)malloc(sizeof(int32_t) * ((size_t)(m > n ? m : n) + 1));
    uint8_t *hit = (uint8_t *)calloc((size_t)(m > n ? m : n) + 1, 1);
    int64_t *diag = (int64_t *)malloc(sizeof(int64_t) * ((size_t)(m > n ? m : n) + 1));
    if (!k.IE || !k.IV || !RE || !RV || !PE.items || !PE.in || !PV.items || !PV.in || !Q || !hit ||
        !diag) {
        free(k.IE); free(k.IV); free(RE); free(RV); free(PE.items); free(PE.in);
        free(PV.items); free(PV.in); free(Q); free(hit); free(diag); free(k.vptr); free(k.vedg);
        return -1;
    }
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    /* I^E_ij = |e_i & e_j|: every vertex adds one to each pair of its hyperedges */
    for (int32_t v = 0; v < n; ++v)
        for (int32_t a = k.vptr[v]; a < k.vptr[v + 1]; ++a)
            for (int32_t b = k.vptr[v]; b < k.vptr[v + 1]; ++b) ie_add(&k, k.vedg[a], k.vedg[b], 1);
    /* I^V_ij = |E(v_i) & E(v_j)|: every hyperedge adds one to each pair of its vertices */
    for (int32_t e = 0; e < m; ++e)
        for (int32_t a = edge_ptr[e]; a < edge_ptr[e + 1]; ++a)
            for (int32_t b = edge_ptr[e]; b < edge_ptr[e + 1]; ++b)
                iv_add(&k, edge_vtx[a], edge_vtx[b], 1);
    memset(RE, 1, (size_t)m + 1);
    memset(RV, 1, (size_t)n + 1);
    for (int32_t e = 0; e < m; ++e) cand_add(&PE, e);
    for (int32_t v = 0; v < n; ++v) cand_add(&PV, v);

    int32_t rounds = 0, changed;
    do {
        changed = 0;
        /* ---- DP pass (Algorithm 4): which alive e_j does some candidate supersede? ---- */
        memset(hit, 0, (size_t)m + 1);
        for (int32_t e = 0; e < m; ++e) diag[e] = ie_get(&k, e, e); /* |e| of every hyperedge */
#pragma omp parallel for schedule(dynamic, 64)
        for (int32_t j = 0; j < m; ++j) {
            if (!RE[j]) continue;
            const int64_t sj = diag[j];
            for (int32_t t = 0; t < PE.len; ++t) {
                const int32_t i = PE.items[t];
                if (i == j || !RE[i]) continue;
                const int64_t x = ie_get(&k, j, i); /* I^E is symmetric: read along row j */
                const int64_t si = diag[i];
                const int dij = (int64_t)k.f[i] - (si - x) >= k.f[j];
                const int dji = (int64_t)k.f[j] - (sj - x) >= k.f[i];
                if (dij && (!dji || i < j)) {
                    hit[j] = 1;
                    break;
                }
            }
        }
        int32_t nq = 0;
        for (int32_t j = 0; j < m; ++j)
            if (hit[j]) Q[nq++] = j;
        for (int32_t t = 0; t < nq; ++t) { /* remove them all at once */
            const int32_t j = Q[t];
            RE[j] = 0;
            for (int32_t a = edge_ptr[j]; a < edge_ptr[j + 1]; ++a)
                for (int32_t b = edge_ptr[j]; b < edge_ptr[j + 1]; ++b)
                    iv_add(&k, edge_vtx[a], edge_vtx[b], -1);
            for (int32_t a = edge_ptr[j]; a < edge_ptr[j + 1]; ++a)
                if (RV[edge_vtx[a]]) cand_add(&PV, edge_vtx[a]);
        }
        cand_clear(&PE);
        changed |= nq > 0;

        /* ---- MD pass (Algorithm 5): count tie-broken dominators of the candidates ---- */
        memset(hit, 0, (size_t)n + 1);
        for (int32_t v = 0; v < n; ++v) diag[v] = iv_get(&k, v, v); /* d_v of every vertex */
#pragma omp parallel for schedule(dynamic, 16)
        for (int32_t t = 0; t < PV.len; ++t) {
            const int32_t j = PV.items[t];
            if (!RV[j]) continue;
            int32_t need_c = 0; /* max demand over alive hyperedges of v_j */
            for (int32_t q = k.vptr[j]; q < k.vptr[j + 1]; ++q)
                if (RE[k.vedg[q]] && k.f[k.vedg[q]] > need_c) need_c = k.f[k.vedg[q]];
            if (need_c == 0) { /* in no alive hyperedge */
                hit[j] = 1;
                continue;
            }
            const int64_t djj = diag[j];
            for (int32_t i = 0; i < n; ++i) {
                if (i == j || !RV[i]) continue;
                const int64_t x = iv_get(&k, j, i);
                if (x == djj && (x != diag[i] || i < j)) {
                    if (--need_c == 0) {
                        hit[j] = 1;
                        break;
                    }
                }
            }
        }
        nq = 0;
        for (int32_t t = 0; t < PV.len; ++t)
            if (hit[PV.items[t]]) Q[nq++] = PV.items[t];
        for (int32_t t = 0; t < nq; ++t) {
            const int32_t j = Q[t];
            RV[j] = 0;
            for (int32_t a = k.vptr[j]; a < k.vptr[j + 1]; ++a)
                for (int32_t b = k.vptr[j]; b < k.vptr[j + 1]; ++b)
                    ie_add(&k, k.vedg[a], k.vedg[b], -1);
            for (int32_t a = k.vptr[j]; a < k.vptr[j + 1]; ++a)
                if (RE[k.vedg[a]]) cand_add(&PE, k.vedg[a]);
        }
        cand_clear(&PV);
        changed |= nq > 0;
        ++rounds;
    } while (changed);

    for (int32_t v = 0; v < n; ++v) alive_v[v] = RV[v];
    for (int32_t e = 0; e < m; ++e) alive_e[e] = RE[e];
    *rounds_out = rounds;
    free(k.IE); free(k.IV); free(RE); free(RV); free(PE.items); free(PE.in);
    free(PV.items); free(PV.in); free(Q); free(hit); free(diag); free(k.vptr); free(k.vedg);
    return 0;
}

/*
 * mhs.h -- C ABI of the GB300 kernelization library for Multiple Hitting Set.
 *
 * The library applies the paper's two demand-aware rules exhaustively, in
 * rounds, on one GPU (arXiv 2109.06042, Section 4.1):
 *
 *   DP (demand pushing, Section 3.1): hyperedge e_i supersedes e_j if
 *       f(e_i) - |e_i \ e_j| >= f(e_j); a superseded hyperedge is deleted.
 *       Algorithm 1 computes this for all pairs from I^E = A A^T (Eq. (1)):
 *       D_ij = [f_i - (I^E_ii - I^E_ij) >= f_j], and deletes e_j iff some
 *       i has D_ij and (not D_ji or i < j).
 *   MD (multiple domination, Section 3.1): vertex v_j is deleted if it has
 *       at least max_{e in E(v_j)} f(e) dominators (v_i with E(v_j) within
 *       E(v_i)).  Algorithm 2 computes this from I^V = A^T A (Eq. (2)):
 *       D_ij = [I_ij = I_jj and (I_ij != I_ii or i < j)], C_j = sum_i D_ij,
 *       delete v_j iff C_j >= max f over E(v_j) (0 if E(v_j) is empty).
 *   Algorithm 3: repeat (Algorithm 1, then Algorithm 2 on its output) until
 *       a round deletes nothing.
 *
 * Two variants of the experiments (Section 5.1) are options:
 *   MHS_RULE_SE ("MD+SE"): the hyperedge pass tests the superedge rule SE
 *       of Section 3.1 instead of DP: e_j goes if some e_i lies within e_j
 *       with f(e_i) >= f(e_j), i.e. D_ij = [I^E_ij = I^E_ii and f_i >= f_j],
 *       with the same simultaneous deletions and tie-break.
 *   full_edges (KernelGPU-FE): whenever Algorithm 3 reaches its fixpoint,
 *       the full-edge rule FE of Section 3.1 runs: every hyperedge with
 *       |e| = f(e) goes and its vertices go into the solution (k drops by
 *       one per vertex, see mhs_forced_at); every other hyperedge loses one
 *       unit of demand per such vertex and goes at demand 0.  If FE changed
 *       anything, more rounds follow; the result is a fixpoint of both.
 *
 * Problem input (Problem 1.1, Section 1): hypergraph H = (V, E) with
 * V = {0..n-1}, hyperedges e_0..e_{m-1} in CSR form, demands f(e) >= 1 and
 * the budget k.  DP, SE and MD never change f or k; only FE lowers them.
 *
 * Conventions
 *  - Every function returns an mhs_status; mhs_last_error() gives a message
 *    for the calling thread.
 *  - The library never takes ownership of caller memory.  Input arrays are
 *    read during the call (host arrays) or before the call's stream work
 *    completes (device arrays); output buffers are written by the call.
 *  - Lowest-index tie-breaking makes results deterministic: ids are the
 *    input ids, and the result lists them in ascending order.
 *  - Counts are exact: incidences are 0/1 values in FP8 E4M3 (exact) with
 *    FP32 accumulation (exact below 2^24), or bit-packed with integer
 *    popcounts; n and m must be < 2^24.
 *  - All device work of an instance runs on the stream given at load time
 *    (NULL: the library creates a non-blocking stream for the instance).
 */
#ifndef MHS_H
#define MHS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MHS_OK = 0,
    MHS_EINVAL = 1,    /* invalid argument or malformed instance */
    MHS_ENOMEM = 2,    /* device or host allocation failed, or over budget */
    MHS_ECUDA = 3,     /* CUDA error; see mhs_last_error() */
    MHS_EAGAIN = 4,    /* result not ready yet (serving) */
    MHS_ETIMEDOUT = 5, /* a bounded wait ran out */
    MHS_EBUSY = 6,     /* request queue full (serving) */
    MHS_EDEVICE = 7    /* a kernel reported an internal error status */
} mhs_status;

/* How the pair counts I^E_ij / I^V_ij are contracted. */
typedef enum {
    MHS_CONTRACT_AUTO = 0,     /* library choice by size */
    MHS_CONTRACT_FP8 = 1,      /* tcgen05 tensor cores, E4M3 0/1, FP32 accumulate */
    MHS_CONTRACT_POPCOUNT = 2  /* bit-packed AND + popcount on the integer units */
} mhs_contraction;

/* Order of the rows (and K columns) of the dense operands.  Results never
 * depend on it (ties are broken by input index); performance does. */
typedef enum {
    MHS_LAYOUT_AUTO = 0,    /* library choice (currently MHS_LAYOUT_DEGREE) */
    MHS_LAYOUT_INPUT = 1,   /* input order */
    MHS_LAYOUT_SORTED = 2,  /* hyperedges by their smallest vertex id: interval-like
                               (low Dilworth number) inputs become banded */
    MHS_LAYOUT_DEGREE = 3   /* vertices grouped by degree class floor(log4 deg), ascending,
                               input order inside a class; hyperedges by their smallest
                               vertex position, i.e. by their rarest vertex.  Skewed degrees
                               then concentrate the nonzero blocks; near-uniform degrees keep
                               the input order and its locality */
} mhs_layout;

/* Block-sparse skipping in the tcgen05 contraction.  Exact either way: a
 * skipped K block or tile contributes only zero products. */
typedef enum {
    MHS_SPARSITY_AUTO = 0,  /* skip (currently the same as MHS_SPARSITY_SKIP) */
    MHS_SPARSITY_SKIP = 1,  /* contract only K blocks where both operands hold a nonzero,
                               and only tiles that can change a flag or a count */
    MHS_SPARSITY_DENSE = 2  /* every tile of the upper triangle, every K block */
} mhs_sparsity;

/* The hyperedge rule of each round's first pass. */
typedef enum {
    MHS_RULE_DP = 0,  /* demand pushing, Algorithm 1 (default) */
    MHS_RULE_SE = 1   /* superedge rule SE (the "MD+SE" variant) */
} mhs_edge_rule;

typedef struct {
    int32_t contraction; /* mhs_contraction */
    int32_t max_rounds;  /* mhs_kernelize stops after this many rounds; 0 = fixpoint */
    int32_t use_graphs;  /* 1: replay captured CUDA graphs (the whole fixpoint in one launch) */
    int32_t layout;      /* mhs_layout */
    int32_t sparsity;    /* mhs_sparsity */
    int32_t edge_rule;   /* mhs_edge_rule */
    int32_t full_edges;  /* 1: alternate with rule FE (KernelGPU-FE); needs max_rounds = 0 */
    /* Tile shape of the tcgen05 contraction (FP8).  Every shape gives the same
     * result; 0 takes the autotuner's choice for the instance's size class
     * (see mhs_tile_config). */
    int32_t tile_m;      /* rows per tile: 0 or 128 */
    int32_t tile_n;      /* columns per tile: 0, 128 (four TMEM accumulators) or 256 (two) */
    int32_t group_rows;  /* row blocks per L2 group of the tile order: 0 or 1..4096 */
    int32_t half_stages; /* 0; 1 = a K block shared in one 64-column half loads as that half;
                            2 = whole K blocks only */
    int32_t reserved[1]; /* must be zero */
} mhs_options;

typedef struct {
    int32_t n_alive;    /* vertices left (over all instances for a batch) */
    int32_t m_alive;    /* hyperedges left */
    int32_t rounds;     /* rounds executed so far, incl. a final unchanged one (max over a batch) */
    int32_t changed;    /* 1 if the last executed round deleted something */
    int32_t dp_deleted; /* hyperedges deleted by the last round's DP pass */
    int32_t md_deleted; /* vertices deleted by the last round's MD pass */
    int32_t active;     /* instances not yet at their fixpoint (0: nothing more to do) */
} mhs_round_stats;

typedef struct mhs_instance mhs_instance;

/* Fill *opt with defaults (AUTO contraction, fixpoint, graphs on). */
mhs_status mhs_default_options(mhs_options *opt);

/*
 * Load one instance from HOST arrays (the input encoding of Section 2.2:
 * the library builds the incidence matrix A of Section 2.1 on the device).
 *   n, m          number of vertices / hyperedges, 0 <= n, m < 2^24
 *   edge_ptr      int32[m+1], edge_ptr[0] = 0, non-decreasing
 *   edge_vtx      int32[edge_ptr[m]], vertex ids in [0, n), no id twice in
 *                 one hyperedge (any order)
 *   demand        int32[m], f(e) >= 1 (f(e) > |e| is allowed: the instance
 *                 is then infeasible but the rules stay well defined)
 *   k             the budget, returned unchanged
 *   opt           options (NULL: defaults)
 *   cuda_stream   cudaStream_t for all work of this instance, or NULL
 *   out           receives the new instance handle
 * Errors: MHS_EINVAL for malformed input, MHS_ENOMEM, MHS_ECUDA; on any
 * error no handle is returned and nothing stays allocated.  The pointer
 * array is checked before anything is read from edge_vtx; the incidences
 * are checked on the host (on several threads for a large instance) while
 * the inputs are copied, and no kernel reads them before the checks pass.
 * The call returns after the input is on the device.
 */
mhs_status mhs_load(int32_t n, int32_t m, const int32_t *edge_ptr, const int32_t *edge_vtx,
                    const int32_t *demand, int64_t k, const mhs_options *opt,
                    void *cuda_stream, mhs_instance **out);

/*
 * Same as mhs_load with DEVICE arrays (same layout).  The instance keeps
 * its own copy.  Structural checks run on the device; malformed input
 * gives MHS_EINVAL (one stream synchronisation at load).  Repeated vertex
 * ids inside one hyperedge count once.
 */
mhs_status mhs_load_device(int32_t n, int32_t m, const int32_t *edge_ptr,
                           const int32_t *edge_vtx, const int32_t *demand, int64_t k,
                           const mhs_options *opt, void *cuda_stream, mhs_instance **out);

/*
 * Load a batch of independent instances from HOST arrays, reduced together
 * (each round contracts all unfinished instances in the same launches).
 *   count                 number of instances, 1 .. 65535
 *   n[b], m[b]            sizes of instance b
 *   edge_ptr              int64[sum m + 1]: CSR over the concatenated
 *                         hyperedges of all instances (instance b owns
 *                         hyperedges [sum_{c<b} m[c], sum_{c<=b} m[c]))
 *   edge_vtx              vertex ids local to each instance, in [0, n[b])
 *   demand                int32[sum m]
 *   k                     int64[count]
 * Checks as mhs_load, on several host threads for a large batch while the
 * inputs are copied; MHS_EINVAL names the lowest malformed instance.
 * Results are read per instance with mhs_result_at().
 */
mhs_status mhs_load_batch(int32_t count, const int32_t *n, const int32_t *m,
                          const int64_t *edge_ptr, const int32_t *edge_vtx,
                          const int32_t *demand, const int64_t *k, const mhs_options *opt,
                          void *cuda_stream, mhs_instance **out);

/*
 * mhs_load_batch with the CSR arrays in DEVICE memory (edge_ptr int64,
 * edge_vtx and demand int32, same layout); n, m and k stay host arrays.
 * Structural checks run on the device; a malformed instance gives
 * MHS_EINVAL naming its index.
 */
mhs_status mhs_load_batch_device(int32_t count, const int32_t *n, const int32_t *m,
                                 const int64_t *edge_ptr, const int32_t *edge_vtx,
                                 const int32_t *demand, const int64_t *k,
                                 const mhs_options *opt, void *cuda_stream, mhs_instance **out);

/* Number of instances held by the handle (1 unless loaded as a batch). */
int32_t mhs_count(const mhs_instance *inst);

/*
 * One iteration of Algorithm 3 (one DP pass, then one MD pass on its
 * output) for every unfinished instance.  An instance whose last round
 * deleted nothing is finished and is not run again (with full_edges: FE runs
 * right after such a round, and the instance goes on if FE changed it).
 * stats may be NULL.  Synchronises the instance's stream once.
 */
mhs_status mhs_reduce_round(mhs_instance *inst, mhs_round_stats *stats);

/* Algorithm 3 to the fixpoint (or opt.max_rounds rounds).  stats may be NULL. */
mhs_status mhs_kernelize(mhs_instance *inst, mhs_round_stats *stats);

/*
 * Sharded rounds: one pass of Algorithm 3 split over several replicas of
 * one instance (Section 4.1 computes every pair of a pass independently,
 * so the pairs can be split; the only exchange is the pass's output).
 * Every replica loads the same instance (count 1, same options) and runs,
 * per round and per phase (0: the DP or SE pass, 1: the MD pass):
 *   mhs_pass_begin      plan and encode (identical on every replica);
 *   mhs_pass_contract   its share `shard` of `nshards`: the tile rows of
 *                       the 128-row blocks b with b % nshards == shard
 *                       (may be called for several shares in a row);
 *   mhs_pass_partial    copies this replica's partial result to a DEVICE
 *                       buffer indexed by INPUT id (replicas may lay rows
 *                       out differently): phase 0 the deletion flags
 *                       uint8[m] (1 = superseded, 0 for ids no longer
 *                       alive), phase 1 the dominator counts int32[n] of
 *                       the input's m hyperedges / n vertices
 *                       (*elems_out = m or n);
 *   (the caller combines the replicas' buffers: element-wise maximum of
 *    the flags, sum of the counts -- e.g. one all-reduce each)
 *   mhs_pass_merge      copies the combined buffer back (DEVICE);
 *   mhs_pass_end        the decision and order-preserving compaction
 *                       (identical on every replica); after phase 1 also
 *                       rule FE if enabled, and *stats (may be NULL) as for
 *                       mhs_reduce_round.
 * mhs_pass_partial and mhs_pass_merge run on the instance's stream and
 * return when their copy is done; a buffer written by other streams must
 * be complete before it is passed in.
 * Passes must come in this order; mhs_kernelize / mhs_reduce_round are
 * refused while a sharded round is in progress.  A replica that runs every
 * share itself needs no partial/merge.  Results equal mhs_kernelize's.
 */
mhs_status mhs_pass_begin(mhs_instance *inst, int32_t phase);
mhs_status mhs_pass_contract(mhs_instance *inst, int32_t phase, int32_t shard, int32_t nshards);
mhs_status mhs_pass_partial(const mhs_instance *inst, int32_t phase, void *dev_out,
                            int64_t *elems_out);
mhs_status mhs_pass_merge(mhs_instance *inst, int32_t phase, const void *dev_in);
mhs_status mhs_pass_end(mhs_instance *inst, int32_t phase, mhs_round_stats *stats);

/*
 * Copy the current result of instance `index` to HOST buffers (any may be
 * NULL to skip it; the counts are always returned when their pointer is
 * non-NULL).
 *   vtx_out[vtx_cap]      surviving vertex ids (input ids), ascending
 *   edge_out[edge_cap]    surviving hyperedge ids (input ids), ascending
 *   demand_out[edge_cap]  current f of each surviving hyperedge (the input's
 *                         unless rule FE lowered it)
 *   n_out, m_out          number of surviving vertices / hyperedges
 *   k_out                 current k (the input's minus the vertices FE took)
 *   rounds_out            rounds executed for this instance
 * MHS_EINVAL if a capacity is too small (counts are still returned).
 */
mhs_status mhs_result_at(const mhs_instance *inst, int32_t index, int32_t *vtx_out,
                         int32_t vtx_cap, int32_t *n_out, int32_t *edge_out,
                         int32_t *demand_out, int32_t edge_cap, int32_t *m_out,
                         int64_t *k_out, int32_t *rounds_out);

/*
 * The vertices rule FE put into the solution for instance `index` (input
 * ids, ascending, HOST buffer vtx_out[cap], may be NULL), their number in
 * *count_out and the FE applications run (counting the last, empty one) in
 * *fe_passes_out (either may be NULL).  Without full_edges the list is
 * empty.  MHS_EINVAL if cap is too small (the count is still returned).
 */
mhs_status mhs_forced_at(const mhs_instance *inst, int32_t index, int32_t *vtx_out, int32_t cap,
                         int32_t *count_out, int32_t *fe_passes_out);

/* mhs_result_at for index 0. */
mhs_status mhs_result(const mhs_instance *inst, int32_t *vtx_out, int32_t vtx_cap,
                      int32_t *n_out, int32_t *edge_out, int32_t *demand_out,
                      int32_t edge_cap, int32_t *m_out, int64_t *k_out, int32_t *rounds_out);

/*
 * Device-side result of instance `index`: alive masks over the input ids,
 * written on the instance's stream (no synchronisation).
 *   alive_v   uint8[n] device buffer, 1 = vertex survives
 *   alive_e   uint8[m] device buffer, 1 = hyperedge survives
 */
mhs_status mhs_result_device(const mhs_instance *inst, int32_t index, uint8_t *alive_v,
                             uint8_t *alive_e);

/*
 * Alive masks of every instance of a batch in one launch, over the
 * concatenated input ids: alive_v (uint8[sum n]) and alive_e (uint8[sum m])
 * DEVICE buffers; instance b's vertices start at sum_{c<b} n[c], its
 * hyperedges at sum_{c<b} m[c].  Written on the instance's stream.
 */
mhs_status mhs_result_batch_device(const mhs_instance *inst, uint8_t *alive_v,
                                   uint8_t *alive_e);

/*
 * Per-round sizes recorded by instance `index` (HOST output): for each
 * executed round r < min(cap_rounds, 32), rows_out[3r..3r+2] = hyperedges
 * entering DP, vertices entering DP, hyperedges left after DP (the sizes
 * the two contractions of that round work on).  *rounds_out = rounds run.
 */
mhs_status mhs_trace_at(const mhs_instance *inst, int32_t index, int32_t *rows_out,
                        int32_t cap_rounds, int32_t *rounds_out);

/*
 * Export the current (reduced) instance `index` as a new CSR over the
 * surviving items, renumbered 0..n'-1 / 0..m'-1 in input order, into HOST
 * buffers.  Re-loading it with mhs_load and reducing further reaches the
 * same fixpoint (the output of a round is itself an instance).
 *   edge_ptr_out  int32[m'+1], edge_vtx_out int32[nnz'], demand_out int32[m']
 *   *nnz_out      receives nnz'; MHS_EINVAL if nnz_cap or edge_cap is too small.
 */
mhs_status mhs_export(const mhs_instance *inst, int32_t index, int32_t *edge_ptr_out,
                      int32_t edge_cap, int32_t *edge_vtx_out, int64_t nnz_cap,
                      int32_t *demand_out, int32_t *n_out, int32_t *m_out, int64_t *nnz_out);

/*
 * Per-round device time split of the last mhs_kernelize / mhs_reduce_round
 * call, in milliseconds (CUDA events on the instance's stream):
 * ms[0] DP contraction, ms[1] MD contraction, ms[2] encode + compaction,
 * ms[3] total.  Timing is recorded only if enabled with mhs_set_timing.
 */
mhs_status mhs_set_timing(mhs_instance *inst, int32_t enable);
/*
 * Tensor-core work done since load (tcgen05 contraction): MMA work in units
 * of 128 x 128 x 32 MACs issued, and tiles contracted.  With block-sparse
 * skipping this is below the dense formulation's count.
 */
mhs_status mhs_work_stats(const mhs_instance *inst, int64_t *mma_kblocks, int64_t *mma_tiles);

/*
 * The tile shape the instance's tcgen05 contraction uses (HOST outputs, any
 * may be NULL): columns per tile (128 or 256), row blocks per L2 group,
 * half stages (1 on, 0 off), and whether the autotuner's table gave it
 * (*from_table = 1) rather than explicit options or the defaults.  The
 * table is the file named by the environment variable MHS_TILE_TABLE, or
 * tile_table.txt beside the library, written by the autotuner
 * (paper_2109_06042_gb300/autotune.py), which times every shape on the GPU
 * per size class.  The choice changes speed only, never a result.
 */
mhs_status mhs_tile_config(const mhs_instance *inst, int32_t *tile_n, int32_t *group_rows,
                           int32_t *half_stages, int32_t *from_table);
mhs_status mhs_last_timing(const mhs_instance *inst, float *ms4);

/*
 * Kernelize one small instance without allocating any memory.  The paper has
 * no counterpart: this entry point exists for callers that must not
 * allocate device memory while they run -- for example code running under a
 * fixed-budget or external allocator, real-time loops where cudaMalloc /
 * cudaFree (which may synchronise the device) are not allowed, or plug-ins
 * whose host owns all device memory.
 *
 * Inputs are DEVICE arrays in the layout of mhs_load (edge_ptr[m+1] with
 * edge_ptr[m] == nnz, edge_vtx[nnz], demand[m]); they are read in place and
 * must stay valid until the call returns.  Outputs: alive_v (uint8[n]) and
 * alive_e (uint8[m]) DEVICE buffers receive 1 for surviving vertices /
 * hyperedges (input ids); *rounds_out (host, may be NULL) the round count.
 * Same rules and result as mhs_kernelize (bit-packed popcount contraction).
 * Every array must be device (or managed) memory of the current device; any
 * other pointer gives MHS_EINVAL before a kernel runs.  A malformed instance
 * (bad edge_ptr, vertex id out of range) gives MHS_EINVAL; a kernel error
 * status, or a round cap reached before the fixpoint, gives MHS_EDEVICE.
 *
 * All working memory is one file-scope device array of 6 MiB that every GPU
 * loading the library keeps until the process exits.  Limits: n <= 4096,
 * m <= 4096, nnz <= 65536; larger instances give MHS_EINVAL.  Every call
 * reuses the same array (the call clears what must start at zero), so calls
 * whose GPU work overlaps race and must be serialised by the caller.  Each
 * call looks up the array's address (cudaGetSymbolAddress) on the current
 * device; the first call on a device may load the library's device code and
 * should come before any stream capture.  The call runs on cuda_stream
 * (NULL: the default stream) and returns after the work is done.  Errors
 * are reported through the return value and, if err_buf is non-NULL, a
 * message in err_buf[err_cap] (mhs_last_error is not used, so that no host
 * string is allocated either).
 */
mhs_status mhs_kernelize_noalloc(int32_t n, int32_t m, const int32_t *edge_ptr,
                                 const int32_t *edge_vtx, const int32_t *demand, int32_t nnz,
                                 uint8_t *alive_v, uint8_t *alive_e, int32_t *rounds_out,
                                 void *cuda_stream, char *err_buf, size_t err_cap);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of independent requests on one GPU.          */
/*                                                                          */
/* The paper reduces one instance at a time; the server keeps many in      */
/* flight.  The request loop runs on the device: one CUDA graph per lane   */
/* whose conditional WHILE node repeats admission of the slots the host    */
/* has loaded, one round of Algorithm 3 for all live slots at once, and    */
/* retirement of the instances that reached their fixpoint (published in   */
/* host-mapped memory), with no host step between rounds.  A host thread   */
/* per lane admits queued requests by HBM footprint, loads them into free  */
/* slots beside the running loop, copies finished results out and starts   */
/* the loop again when it has gone idle.  Each result is exactly what      */
/* mhs_kernelize gives for the instance alone.                             */
/* ------------------------------------------------------------------------ */

typedef struct mhs_server mhs_server;

typedef struct {
    int64_t hbm_budget_bytes; /* device bytes the admitted instances may hold (0: 3/4 of free) */
    int32_t max_slots;        /* instances in flight at most, 1..4096 (default 256) */
    int32_t queue_capacity;   /* queued requests at most; beyond it mhs_submit gives MHS_EBUSY */
    int32_t contraction;      /* mhs_contraction */
    int32_t layout;           /* mhs_layout */
    int32_t sparsity;         /* mhs_sparsity */
    int32_t small_items;      /* requests with n + m <= this go to the small-request lane
                                 (0: 8192; < 0: a single lane for all requests) */
    int32_t edge_rule;        /* mhs_edge_rule, for every request */
    int32_t full_edges;       /* 1: KernelGPU-FE for every request (see mhs_options) */
} mhs_server_options;

typedef struct {
    int64_t submitted, admitted, completed, rounds;
    int32_t pending, active;
    int64_t bytes_in_use, peak_bytes, budget_bytes;
} mhs_server_stats;

mhs_status mhs_server_default_options(mhs_server_options *opt);

/* Start a server on the current device.  Requests are split by size into
 * two lanes, each with its own slot table, worker thread and stream: small
 * requests (n + m <= small_items) are batched on a high-priority stream the
 * server creates; large ones run a few at a time on cuda_stream (NULL: a
 * stream of its own).  opt may be NULL (defaults). */
mhs_status mhs_server_create(const mhs_server_options *opt, void *cuda_stream, mhs_server **out);

/*
 * Queue one request (HOST arrays, layout and checks of mhs_load; copied
 * before the call returns).  *ticket identifies it for mhs_poll.
 * MHS_EBUSY: the queue is full; MHS_ENOMEM: the instance alone exceeds the
 * budget; MHS_EINVAL: malformed input.
 */
mhs_status mhs_submit(mhs_server *srv, int32_t n, int32_t m, const int32_t *edge_ptr,
                      const int32_t *edge_vtx, const int32_t *demand, int64_t k,
                      uint64_t *ticket);

/*
 * Wait up to timeout_us (0: do not wait, < 0: no limit) for request
 * `ticket`.  MHS_EAGAIN if it is not finished.  When finished, the outputs
 * are those of mhs_result; times_ns (may be NULL) receives 3 values: time
 * queued, time in service, total (nanoseconds, server clock).  With all of
 * vtx_out, edge_out and demand_out NULL only the counts are returned and
 * the result is kept; otherwise it is copied out and released.
 */
mhs_status mhs_poll(mhs_server *srv, uint64_t ticket, int64_t timeout_us, int32_t *vtx_out,
                    int32_t vtx_cap, int32_t *n_out, int32_t *edge_out, int32_t *demand_out,
                    int32_t edge_cap, int32_t *m_out, int64_t *k_out, int32_t *rounds_out,
                    int64_t *times_ns);

/*
 * The vertices rule FE put into the solution of finished request `ticket`
 * whose result is still held (after a counts-only mhs_poll): input ids
 * ascending into vtx_out[cap] (may be NULL), their number in *count_out.
 * MHS_EAGAIN if the request is not finished, MHS_EINVAL for an unknown or
 * released ticket or a too small cap.
 */
mhs_status mhs_server_forced(mhs_server *srv, uint64_t ticket, int32_t *vtx_out, int32_t cap,
                             int32_t *count_out);

/* Stop (paused != 0) or resume admitting queued requests; running ones finish. */
mhs_status mhs_server_pause(mhs_server *srv, int32_t paused);

mhs_status mhs_server_get_stats(mhs_server *srv, mhs_server_stats *out);

/* Stop the worker, fail unfinished requests and free everything. */
void mhs_server_destroy(mhs_server *srv);

/* Free all device and host memory of the instance (synchronises its stream). */
void mhs_free(mhs_instance *inst);

/*
 * Diagnostic (no counterpart in the paper): run one kernel that waits on a
 * barrier nothing ever arrives at, with the bounded wait every tcgen05 wait
 * uses, limited to limit_ns (<= 2 s).  *status_out receives the kernel's
 * status (4 = the wait timed out, as it must) and *waited_ns_out how long
 * it waited.  The context stays usable afterwards.
 */
mhs_status mhs_selftest_bounded_wait(int64_t limit_ns, int32_t *status_out,
                                     int64_t *waited_ns_out);

/* Thread-local message for the last failing call on this thread. */
const char *mhs_last_error(void);

/* Library version string. */
const char *mhs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MHS_H */

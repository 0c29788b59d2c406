// mhs_internal.h -- device-resident state shared by the kernels and the host driver.
//
// One InstState per instance lives in device memory.  Every kernel reads the
// current sizes from it, so the host never needs them to size a launch: all
// launches use fixed persistent grids and a round can be captured as one
// CUDA graph for any batch.
//
// Ids.  "Original" ids are the input ids.  "Current" ids (positions) number
// the items still alive in the layout order of the dense operands: input
// order; hyperedges sorted by smallest vertex id; or vertices grouped by
// degree class and hyperedges sorted by smallest vertex position.
// Compaction preserves the layout order.  The lowest-index tie-breaks of Algorithms 1 and 2
// always compare ORIGINAL ids (e_c2o / v_c2o), so results do not depend on
// the layout.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace mhs {

// Tile shapes.
constexpr int kPopTile = 64;     // popcount contraction: 64 x 64 pair tiles
constexpr int kTcM = 128;        // tcgen05 contraction: 128 rows (i) x 128 or 256 columns (j)
constexpr int kTcNDefault = 256; // per tile; the wider tile unless chosen otherwise
constexpr int kTcK = 128;        // K bytes per pipeline stage (FP8)
constexpr int kOccK = 64;        // K columns per occupancy bit (half a stage)
constexpr int kRowAlign = 256;   // row capacity rounded to this
constexpr int kTraceRounds = 32; // rounds whose sizes an instance records

enum Contraction : int32_t { kAuto = 0, kFp8 = 1, kPopcount = 2 };

// Status bits written by kernels (OR-ed into InstState::status).
enum : int32_t {
    kErrBadVertex = 1,     // vertex id out of range in the input
    kErrBadPtr = 2,        // edge_ptr not monotone / inconsistent
    kErrTimeout = 4,       // a bounded wait gave up
    kErrCapacity = 8,      // an index exceeded an allocated capacity
    kErrBadDemand = 16,    // a demand f(e) < 1 in the input
    kErrRoundCap = 32,     // the device-side round loop hit its hard cap
};

struct InstState {
    // ---- input (original ids), device copies owned by the instance ----
    int32_t n0, m0;
    int64_t nnz0;
    const int32_t *eptr;   // [m0+1] (int32 offsets into evtx)
    const int32_t *evtx;   // [nnz0] vertex ids
    int32_t *f;            // [m0] current demands (the input's, until FE lowers them)

    int64_t k;             // current budget (FE lowers it)

    // ---- reduction variant ----
    int32_t edge_rule;     // hyperedge pass: 0 = DP (Algorithm 1), 1 = SE (superedge rule)
    int32_t full_edges;    // 1: alternate the DP/SE + MD fixpoint with rule FE
    int32_t fe_stage;      // 1: this round reached the fixpoint; FE runs before the next
    int32_t fe_passes;     // FE applications so far (counting the last, empty one)
    uint8_t *forced;       // [n0] 1 = vertex put into the solution by FE (input ids)

    // ---- round state ----
    int32_t n, m;          // current alive vertices / hyperedges
    int32_t m_dp;          // hyperedges alive after this round's DP pass
    int32_t n_next;        // vertices alive after this round's MD pass
    int32_t rounds;        // executed rounds
    int32_t active;        // 1 while the instance has not reached its fixpoint
    int32_t max_rounds;    // 0 = unbounded
    int32_t changed;       // last round deleted something
    int32_t dp_deleted, md_deleted;
    int32_t status;        // kErr* bits
    int32_t layout_sorted; // 0: input order; 1: hyperedges by smallest vertex id;
                           // 2: vertices by degree class, hyperedges by smallest vertex position

    // id maps (capacity n0 / m0)
    int32_t *v_o2c, *v_c2o;
    int32_t *e_o2c, *e_c2o;
    int32_t *e_prev;       // [m0] input id of each row as DP saw it (before compaction)
    // Compaction of a single instance by several blocks (a chained scan over
    // chunks of 1024 ids, one per block): per chunk a status word
    // {epoch << 34 | flag << 32 | count}; blocks take chunks by ticket, in
    // arrival order.  k_plan resets the ticket and advances the epoch before
    // every phase.  nullptr: one block compacts the instance.
    unsigned long long *scan_status;  // [scan_chunks]
    int32_t scan_chunks;
    uint32_t scan_ticket;
    uint32_t scan_epoch;

    // epilogue inputs, indexed by current id
    int32_t *e_f;          // f of current hyperedge
    int32_t *e_s;          // alive size |e| of current hyperedge (= I^E_ii)
    int32_t *v_deg;        // degree over alive hyperedges (= I^V_jj)   [n0 + 1]
    int32_t *v_maxf;       // max demand over alive hyperedges (0 if none)
    int32_t *v_cnt;        // C_j of Algorithm 2                         [n0 + 1]
    int4 *e_rec;           // tcgen05 path: per current hyperedge {f, f - |e| (SE: |e|), input id},
                           // written by the DP set pass for the epilogue's staging
    uint8_t *e_del;        // DP deletion flags
    uint8_t *v_del;        // MD deletion flags
    // Incremental rounds.  After the first round, a pass can only delete
    // through an item that changed since the previous pass of its kind: a
    // hyperedge that lost a vertex (DP), or a vertex that lost a hyperedge
    // (MD).  e_s keeps each hyperedge's size from the previous DP pass
    // (-1: never tested).  NULL arrays mean every row is a candidate.
    uint8_t *e_dirty_rb;   // per 128 hyperedge rows: some row changed (DP pass)
    uint8_t *v_dirty;      // per current vertex: lost a hyperedge in this round's DP
    uint8_t *v_dirty_rb;   // per 128 vertex rows: some v_dirty set
    int32_t md_full;       // 1: every vertex is an MD candidate (first round, after FE)
    // tcgen05 path, set by the plan of each phase: no candidate can exist in
    // this round's DP pass (the previous MD pass deleted no vertex) or MD pass
    // (this round's DP pass deleted no hyperedge), so its operand is neither
    // written nor cleared and its tile list is empty
    int32_t skip_a, skip_at;

    // dense FP8 operands: rows x pitch bytes (0x38 = 1.0 in E4M3)
    uint8_t *A;            // rows = current hyperedges, K = current vertices
    uint8_t *At;           // rows = current vertices, K = current hyperedges
    int64_t A_pitch, At_pitch;
    int32_t A_rows, At_rows;
    // bit-packed operands: rows x pitch 32-bit words
    uint32_t *Ab, *Atb;
    int32_t Ab_pitch, Atb_pitch;
    // tcgen05 tensor maps for A and At in device memory, each two CUtensorMaps
    // (128 bytes each): full stages, then half stages
    const void *tmap_A;
    const void *tmap_At;
    // block-sparse skipping (tcgen05 path): per row block of 128 rows, one
    // bit per K block of kOccK columns that holds a nonzero of the operand of
    // phase p (0: A, 1: At); occ_words[p] words per row block
    uint32_t *occ[2];
    int32_t occ_words[2];
    int32_t has_loose;     // zero counts matter in this hyperedge pass: DP, some
                           // hyperedge has f > |e|; SE, some hyperedge is empty
    int32_t no_skip;       // 1: contract every tile and K block (dense formulation)
    // offsets of this instance's ids in the concatenated ids of its batch
    int64_t v_base, e_base;
    // per round r < kTraceRounds: hyperedges and vertices entering DP, hyperedges after DP
    int32_t trace[kTraceRounds][3];
};

// Per-phase work plan over a batch, rebuilt on the device before each phase.
struct Plan {
    int32_t count;          // instances
    int32_t any_active;
    int64_t *tile_list;     // tcgen05: packed (instance, row block, column block) to contract
    int32_t list_count;     // entries in tile_list this phase
    int32_t list_cap;
    int32_t total_rows;     // current hyperedges to scatter this phase
    int32_t group_rows;     // tcgen05 tile order: row blocks per L2 group (0: default)
    int64_t total_tiles;    // contraction tiles this phase
    int32_t *row_off;       // [count+1] prefix of current hyperedges of active instances
    int64_t *tile_off;      // [count+1] prefix of tiles
    int32_t list_next;      // tcgen05: next tile_list entry to hand out (dynamic schedule)
    int32_t tile_n;         // tcgen05: columns per tile, 128 or 256 (rows: kTcM)
    int32_t half_stages;    // tcgen05: 1 = load a K block shared in one half as that half
    // tcgen05: the tile list holds two queues, tiles whose MMA work exceeds
    // the epilogue's from the front (list_count entries), the others from
    // the back (list_light entries, the j-th at list_cap - 1 - j)
    int32_t list_light;
    int32_t list_next_light;  // next light entry to hand out
    int32_t two_queues;       // 0: every tile in the front queue (one queue)
};

// Number of pair tiles of an R x R upper triangle.
__host__ __device__ inline int64_t pop_tiles(int32_t R) {
    int64_t t = (R + kPopTile - 1) / kPopTile;
    return R > 1 ? t * (t + 1) / 2 : 0;
}

// Packed tile-list entries.
__host__ __device__ inline int64_t pack_tile(int b, int32_t bi, int32_t bj) {
    return ((int64_t)b << 40) | ((int64_t)bi << 20) | (int64_t)bj;
}
// Flag of a tile-list entry (tcgen05 path): no K block holds a nonzero of
// both operands, so the tile contracts nothing.
constexpr int64_t kTileNoK = (int64_t)1 << 62;
__host__ __device__ inline void unpack_tile(int64_t v, int *b, int32_t *bi, int32_t *bj) {
    *b = (int)((v >> 40) & 0x3FFFFF);
    *bi = (int32_t)((v >> 20) & 0xFFFFF);
    *bj = (int32_t)(v & 0xFFFFF);
}

// tcgen05 tiles: row blocks of kTcM, column blocks of tn = r * kTcM columns
// (r = 1 or 2); tile (bi, bj) is needed iff it holds some pair i < j (j < R),
// i.e. bj >= floor(bi / r).
__host__ __device__ inline int32_t tc_col_blocks(int32_t R, int32_t tn) { return (R + tn - 1) / tn; }
__host__ __device__ inline int32_t tc_row_blocks(int32_t R) { return (R + kTcM - 1) / kTcM; }
// sum over b < bi of floor(b / r), for r = 1 or 2
__host__ __device__ inline int64_t tc_floor_sum(int64_t bi, int32_t r) {
    if (r == 1) return bi * (bi - 1) / 2;
    return (bi / 2) * ((bi - 1) / 2 > 0 ? (bi - 1) / 2 : 0);
}
__host__ __device__ inline int64_t tc_tiles(int32_t R, int32_t tn) {
    if (R <= 1) return 0;
    // sum over row blocks bi of (cb - floor(bi / r))
    const int32_t r = tn / kTcM;
    const int64_t rb = tc_row_blocks(R), cb = tc_col_blocks(R, tn);
    return rb * cb - tc_floor_sum(rb, r);
}

}  // namespace mhs

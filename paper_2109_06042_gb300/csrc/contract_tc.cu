// contract_tc.cu -- tcgen05 tensor-core contraction of the 0/1 incidence
// operands with the fused DP / MD epilogue (sm_103a).
//
// For each tile of 128 rows i x kN columns j of the upper triangle (kN = 256
// or 128, the tile shape of the launch), the kernel computes
// x_ij = sum_k X_ik X_jk, i.e. I^E_ij of Eq. (1) for X = A (phase 0, DP) or
// I^V_ij of Eq. (2) for X = A^T (phase 1, MD), with both operands taken from
// the same K-major FP8 E4M3 matrix (0x38 = 1.0, 0x00 = 0).  Products are 0/1
// and the FP32 accumulator holds integers below 2^24, so x_ij is exact.  The
// counts never leave the SM: the epilogue warps read them with tcgen05.ld
// and apply Algorithm 1 (DP) or Algorithm 2 (MD) directly; the matrix I is
// never written.
//
// Warp roles (352 threads, one CTA per SM, persistent over the tile list):
//   warp 0      TMA producer: 128-byte-swizzled K slices of the i rows
//               (128 x 128 B) and the j rows (kN x 128 B) into a ring of
//               192 KB of stages (4 of 48 KB for kN = 256, 6 of 32 KB for
//               kN = 128).  It reads each tile's shared K blocks from the
//               scheduler's masks in shared memory: no global load on its path.
//   warp 1      TMEM allocation (512 columns = 512 / kN accumulators of
//               128 x kN FP32) and the single-thread tcgen05.mma issuer.
//   warps 2-9   epilogue; warp w reads TMEM lanes 32*(w%4) .. +31, warps 2-5
//               the first kN/2 columns of a tile, warps 6-9 the others.
//   warp 10     tile scheduler: takes tiles from the list ahead of the other
//               roles, ANDs the two operands' occupancy words of each (32
//               lanes in parallel) and publishes tile and masks in a ring of
//               shared-memory slots.
// Tiles whose counts are known to be at most 1024 (every staged size,
// degree and demand is) are drained from TMEM into packed FP16 registers
// right away, so their accumulator goes back to the MMA thread before the
// pair tests run.
// Every mbarrier wait is bounded: on timeout the kernel records
// kErrTimeout, stops issuing work, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>

#include "bounded_wait.cuh"
#include "kernels.h"
#include "mhs_internal.h"

namespace mhs {

namespace {

constexpr int kABytes = kTcM * kTcK;            // 16 KB: the i rows of a stage
// A stage whose K block shares a nonzero in only one of its two halves
// loads just that half (kOccK columns of each operand, 64-byte swizzle,
// 8 KB per 128-row box) into the front of the same slots.
constexpr int kHalfBox = kTcM * kOccK;          // 8 KB
static_assert(2 * kOccK == kTcK, "a stage is two occupancy blocks");
constexpr int kStageBudget = 192 * 1024;        // shared memory for stages
// An operand's tensor maps: the full-stage map, then the half-stage map.
constexpr int kTmapBytes = 128;
constexpr int kTmemCols = 512;
constexpr int kEpiWarps = 8;                    // two per TMEM lane quarter
constexpr int kSchedWarp = 2 + kEpiWarps;       // the tile scheduler's warp
constexpr int kThreads = 32 * (kSchedWarp + 1); // producer, MMA, epilogue, scheduler
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kMaskWords = 64;                  // occupancy words kept per ring slot
                                                // (K up to 131,072; beyond, the producer
                                                // reads the rest from global memory)
constexpr int kGroupRows = 16;                  // default row blocks per L2 group
constexpr uint64_t kWaitNs = 4000000000ull;     // 4 s bound on any wait
constexpr int kRing = 8;                        // tile-list entries in flight
constexpr float kSmallMax = 1024.f;             // FP16 paired tests: |values| <= this

// Compile-time shape of a launch: tiles of 128 x kN.
template <int kN>
struct Shape {
    static_assert(kN == 128 || kN == 256, "tile widths of 128 or 256 columns");
    static constexpr int kBBytes = kN * kTcK;                 // the j rows of a stage
    static constexpr int kStageBytes = kABytes + kBBytes;     // 48 or 32 KB
    static constexpr int kStages = kStageBudget / kStageBytes;  // 4 or 6
    static constexpr int kHalfStageBytes = kHalfBox * (1 + kN / kTcM);
    static constexpr int kAcc = kTmemCols / kN;               // accumulators: 2 or 4
    static constexpr int kRatio = kN / kTcM;                  // row blocks per column block
    static constexpr int kCols = kN / 2;                      // columns per epilogue warp
    static constexpr int kChunks = kCols / 32;                // 32-column chunks per warp
    // Instruction descriptor, kind::f8f6f4: D = F32, A = B = E4M3, both
    // K-major, N = kN, M = 128.
    static constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) |
                                       ((uint32_t)(kN >> 3) << 17) |
                                       ((uint32_t)(kTcM >> 4) << 24);
};

// ------------------------------------------------------------- PTX glue --

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int32_t x, int32_t y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(tmap), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptors, K-major, version 1 (bits 46-48), the
// leading byte offset unused (1): a full stage has 128-byte swizzled rows in
// 8-row atoms of 1024 bytes (stride byte offset, layout type 2); a half
// stage 64-byte swizzled rows in atoms of 512 bytes (layout type 4).  The
// start address (bits 0-13, in 16-byte units) is OR-ed in per MMA.
constexpr uint64_t kDescFull =
    ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
constexpr uint64_t kDescHalf =
    ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
__device__ __forceinline__ uint64_t smem_desc(uint64_t layout, uint32_t addr) {
    return layout | (uint64_t)((addr & 0x3FFFFu) >> 4);
}

template <uint32_t kIdesc>
__device__ __forceinline__ void mma_f8(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}
// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per
// lane); the load is asynchronous until tmem_wait.
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
// Wait for this thread's outstanding TMEM loads.  The registers of the
// loads are in-out operands, so no use of them is scheduled before the wait.
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                   "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                   "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}
// Orders the registers of a second load after an earlier tmem_wait (which
// waited for every outstanding load of the thread).
__device__ __forceinline__ void tmem_after_wait(uint32_t (&r)[32]) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                   "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                   "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    tmem_ld32_issue(taddr, r);
    tmem_wait(r);
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}
// Two FP32 counts (exact integers <= 2048) as one FP16x2 word.
__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ __half2 as_h2(uint32_t w) { return *reinterpret_cast<__half2 *>(&w); }
// Named barrier of the epilogue warps that also ANDs a flag over them.
__device__ __forceinline__ bool epi_bar_and(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kEpiThreads)
        : "memory");
    return r != 0;
}

// ------------------------------------------------------ tile scheduling --

// Tiles of one instance: row block bi (128 rows) x column block bj (kN =
// r * 128 columns), kept iff it holds a pair i < j, i.e. bj >= floor(bi / r).
// prefix(bi) = number of tiles in row blocks < bi.
__device__ __forceinline__ int64_t tc_prefix(int64_t bi, int64_t cb, int32_t r) {
    return bi * cb - tc_floor_sum(bi, r);
}

// Order: groups of G row blocks; inside a group, column block by column
// block, and inside a column block the group's row blocks.  With G = 16,
// the ~152 tiles in flight share 16 row blocks and a few column blocks,
// which keeps their K slices in L2.
__device__ void tc_tile_coords(int64_t t, int32_t R, int32_t G, int32_t r, int32_t *bi_out,
                               int32_t *bj_out) {
    const int32_t rb = tc_row_blocks(R), cb = tc_col_blocks(R, r * kTcM);
    const int32_t ng = (rb + G - 1) / G;
    int32_t lo = 0, hi = ng;  // find group g: prefix(g*G) <= t < prefix((g+1)*G)
    while (hi - lo > 1) {
        int32_t mid = (lo + hi) >> 1;
        if (tc_prefix((int64_t)mid * G, cb, r) <= t) lo = mid; else hi = mid;
    }
    const int32_t g = lo;
    const int32_t r0 = g * G;
    const int32_t gsz = min(G, rb - r0);
    int64_t p = t - tc_prefix(r0, cb, r);
    int32_t bj = r0 / r;  // first column block of the group
    for (;;) {
        // row blocks bi in [r0, r0+gsz) with floor(bi/r) <= bj
        int32_t c = r * bj + r - r0;
        c = c < 0 ? 0 : (c > gsz ? gsz : c);
        if (c == gsz) {
            *bj_out = bj + (int32_t)(p / gsz);
            *bi_out = r0 + (int32_t)(p % gsz);
            return;
        }
        if (p < c) { *bj_out = bj; *bi_out = r0 + (int32_t)p; return; }
        p -= c;
        ++bj;
    }
}

struct TileInfo {
    int b;
    int32_t bi, bj, R, nk;
};

// Sizes of the tile a packed tile-list entry names.
__device__ __forceinline__ void tile_info(const InstState *st, int phase, int64_t entry,
                                          TileInfo *ti) {
    unpack_tile(entry, &ti->b, &ti->bi, &ti->bj);
    const InstState &s = st[ti->b];
    ti->R = phase == 0 ? s.m : s.n;
    const int32_t K = phase == 0 ? s.n : s.m_dp;
    ti->nk = ((K > 0 ? K : 1) + kTcK - 1) / kTcK;
}

// The epilogue's per-row record of row or column j (zero past R): DP / SE
// {f, f - |e| (SE: |e|), input id}; MD {deg, 0, input id}, with a degree
// of 0 staged as -1.  A vertex in no hyperedge is deleted whatever its
// dominator count (its maximum demand is 0), and the only counts equal to
// its degree 0 are the zero counts with other such vertices; staged as -1
// it matches no count, so zero counts never set a flag in MD and a chunk of
// them needs no test.
__device__ __forceinline__ int4 epi_record(const InstState &s, int phase, int32_t j, int32_t R) {
    if (j >= R) return make_int4(0, 0, 0, 0);
    if (phase == 0) return s.e_rec[j];
    const int32_t d = s.v_deg[j];
    return make_int4(d > 0 ? d : -1, 0, s.v_c2o[j], 0);
}
// True if a record's values bound every count it takes part in by
// kSmallMax: |a|, |b| and the size a - b (DP; SE and MD stage the size or
// degree itself) are all at most kSmallMax.
__device__ __forceinline__ bool record_small(int4 rec) {
    const float a = (float)rec.x, b = (float)rec.y;
    return fabsf(a) <= kSmallMax && fabsf(b) <= kSmallMax && fabsf(a - b) <= kSmallMax;
}

// K blocks of a tile where both operands hold a nonzero: the occupancy
// bits of row block bi AND those of the r row blocks of column block bj.
// A bit covers kOccK = 64 columns, half a K block: a K block is loaded when
// either of its halves is shared, so a nonzero of one operand in the low
// half and one of the other in the high half do not cost a load; kit_next
// leaves in `halves` which halves are shared (1: low, 2: high, 3: both).
// Every role walks the same sequence.
struct KIter {
    const uint32_t *a, *b0, *b1;
    int32_t nkw, w, nk;
    uint32_t mask;
    uint32_t halves;
    bool all;
};
__device__ __forceinline__ void kit_init(KIter &k, const InstState &s, int phase,
                                         const TileInfo &ti, int32_t r) {
    const uint32_t *base = s.occ[phase];
    const int64_t W = s.occ_words[phase];
    k.a = base + (int64_t)ti.bi * W;
    k.b0 = base + (int64_t)(r * ti.bj) * W;
    k.b1 = r == 2 ? k.b0 + W : nullptr;
    k.nk = 2 * ti.nk;  // occupancy bits
    k.nkw = (k.nk + 31) / 32;
    k.w = -1;
    k.mask = 0;
    k.all = s.no_skip != 0;
}
__device__ __forceinline__ int32_t kit_next(KIter &k) {
    while (k.mask == 0) {
        if (++k.w >= k.nkw) return -1;
        if (k.all) {
            const int32_t left = k.nk - 32 * k.w;
            k.mask = left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
        } else {
            uint32_t bm = __ldg(k.b0 + k.w);
            if (k.b1) bm |= __ldg(k.b1 + k.w);
            k.mask = __ldg(k.a + k.w) & bm;
        }
    }
    const int32_t bit = (__ffs(k.mask) - 1) & ~1;  // the K block's two bits
    k.halves = (k.mask >> bit) & 3u;
    k.mask &= ~(3u << bit);
    return (k.w * 32 + bit) >> 1;
}

// Shared K-block halves of a tile (its MMA work in half stages): the set
// bits of the ANDed occupancy words over its K range.
__device__ __forceinline__ int32_t kit_weight(const KIter &k) {
    if (k.all) return 2 * k.nk;
    int32_t w = 0;
    for (int32_t i = 0; i < k.nkw; ++i) {
        uint32_t bm = __ldg(k.b0 + i);
        if (k.b1) bm |= __ldg(k.b1 + i);
        w += __popc(__ldg(k.a + i) & bm);
    }
    return w;
}

// A tile whose MMA work exceeds about what the epilogue spends on a tile
// (~5,000 cycles: 18 half stages of 128 x 256 x 64 at the FP8 rate) is
// heavy; the scheduler alternates heavy and light tiles so that the MMA
// thread and the epilogue warps stay busy together.  Measured on one GB300:
// power-law 20,000 x 40,000 +2.8 % per kernelization, the batch of 4,096
// -1.1 % (its two frontiers of the tile order share L2 less well), so a load
// of one instance uses two queues and a batch one (Plan::two_queues).
constexpr int32_t kHeavyHalves = 18;

// Build this phase's tile list: every tile of the upper triangle (in the
// grouped order of tc_tile_coords, tiles 128 x plan->tile_n) that holds a
// candidate row or column (incremental rounds) and shares a nonzero K block
// -- or, in a DP pass of an instance with a hyperedge f > |e|, every such
// tile, since zero counts can then supersede.  Zero tiles otherwise change
// nothing: in DP a zero count supersedes only from a hyperedge with
// f > |e|, and in MD a zero count only adds dominators of a vertex in no
// hyperedge, which is deleted anyway (its maximum demand is 0).
// Warp-aggregated appends keep runs of 32 consecutive tiles together.
__global__ void k_tile_list(InstState *st, Plan *plan, int phase, int shard, int nshards) {
    const int lane = threadIdx.x & 31;
    const int64_t total = plan->total_tiles;
    const int32_t G = plan->group_rows > 0 ? plan->group_rows : kGroupRows;
    const int32_t r = plan->tile_n / kTcM;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane); base < total;
         base += nw * 32) {
        const int64_t t = base + lane;
        bool keep = false;
        int64_t packed = 0;
        int32_t weight = kHeavyHalves;  // (the dense formulation: every tile heavy)
        if (t < total) {
            int lo = 0, hi = plan->count;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (plan->tile_off[mid] <= t) lo = mid; else hi = mid;
            }
            const InstState &s = st[lo];
            TileInfo ti;
            ti.b = lo;
            ti.R = phase == 0 ? s.m : s.n;
            const int32_t K = phase == 0 ? s.n : s.m_dp;
            ti.nk = ((K > 0 ? K : 1) + kTcK - 1) / kTcK;
            tc_tile_coords(t - plan->tile_off[lo], ti.R, G, r, &ti.bi, &ti.bj);
            bool has_k = true;
            if (nshards > 1 && ti.bi % nshards != shard) {
                keep = false;  // another share's row block
            } else if (s.no_skip) {
                keep = true;  // the dense formulation: every tile, every round
            } else {
                // only tiles that hold a candidate row (incremental rounds) ...
                const uint8_t *drb = phase == 0 ? s.e_dirty_rb : s.v_dirty_rb;
                keep = !drb || (phase == 1 && s.md_full) || drb[ti.bi] || drb[r * ti.bj] ||
                       (r == 2 && drb[r * ti.bj + 1]);
                // ... and share a nonzero K block, unless zero counts matter
                if (keep) {
                    KIter k;
                    kit_init(k, s, phase, ti, r);
                    weight = kit_weight(k);
                    has_k = weight > 0;
                    keep = has_k || (phase == 0 && s.has_loose);
                }
            }
            packed = pack_tile(lo, ti.bi, ti.bj) | (has_k ? 0 : kTileNoK);
        }
        // heavy tiles from the front of the list, light ones from the back
        // (a 128 x 128 tile halves both sides, so the threshold holds for both widths)
        const bool heavy = !plan->two_queues || weight >= kHeavyHalves;
        const uint32_t bh = __ballot_sync(0xffffffffu, keep && heavy);
        const uint32_t bl = __ballot_sync(0xffffffffu, keep && !heavy);
        int32_t sh = 0, sl = 0;
        if (lane == 0 && bh) sh = atomicAdd(&plan->list_count, __popc(bh));
        if (lane == 0 && bl) sl = atomicAdd(&plan->list_light, __popc(bl));
        sh = __shfl_sync(0xffffffffu, sh, 0);
        sl = __shfl_sync(0xffffffffu, sl, 0);
        const uint32_t below = (1u << lane) - 1u;
        if (keep && heavy) plan->tile_list[sh + __popc(bh & below)] = packed;
        if (keep && !heavy) plan->tile_list[plan->list_cap - 1 - (sl + __popc(bl & below))] = packed;
    }
}

// Tiles are handed out dynamically: the scheduler warp takes the next
// tile-list entry with an atomic and publishes it in a ring of shared slots
// that the producer, the MMA thread and the epilogue warps read in the same
// order.  CTAs that draw cheap tiles take more of them, so the tiles in
// flight at any time stay a narrow window of the (L2-grouped) list.
// One published tile: its list entry, coordinates, and the AND of both
// operands' occupancy words over its K range (bit: 64 shared columns).
struct TileSlot {
    int64_t entry;  // packed tile-list entry, -1 = no more tiles
    int32_t b, bi, bj, R, nk, nkw;
    uint32_t mask[kMaskWords];
};

// The column records of a tile, staged by the epilogue (one column per
// thread), double-buffered so that a warp can stage the next tile while
// slower warps still test this one.
template <int kN>
struct __align__(16) TileCols {
    __half a16[kN];  // ab as FP16 (exact when |value| <= 1024): the paired tests
    __half b16[kN];
    float2 ab[kN];   // DP: (f_j, f_j - s_j)   SE: (f_j, s_j)   MD: (d_j, 0)
    int32_t o[kN];   // input index of column j (tie-breaks)
};

template <int kN>
struct __align__(16) SharedCtl {
    using S = Shape<kN>;
    TileCols<kN> cols[2];
    uint64_t full[S::kStages];
    uint64_t empty[S::kStages];
    uint64_t tmem_full[S::kAcc];
    uint64_t tmem_empty[S::kAcc];
    uint64_t ring_full[kRing];   // slot published (the scheduler's 32 lanes arrive)
    uint64_t ring_empty[kRing];  // slot read by the producer, the MMA thread and the epilogue
    TileSlot slot[kRing];
    uint32_t stage_last[S::kStages];  // bit 0: the stage ends its tile; bit 1: a half stage
                                      // (written by the producer)
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

template <int kN>
constexpr size_t smem_bytes() {
    return 1024 + (size_t)Shape<kN>::kStages * Shape<kN>::kStageBytes + sizeof(SharedCtl<kN>);
}
static_assert(smem_bytes<256>() <= 232448 && smem_bytes<128>() <= 232448,
              "stages and control fit one CTA's shared memory");

// Transpose the 32 x 32 bit matrix held by a warp (lane r holds row r, bit
// c = column c): afterwards lane c holds column c (bit r = row r).  Five
// butterfly stages, each swapping the off-diagonal w x w blocks of every
// 2w x 2w block.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int w = 16 >> st;
        const uint32_t m = masks[st];
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, w);
        x = (lane & w) ? ((x & ~m) | ((y & ~m) >> w)) : ((x & m) | ((y & m) << w));
    }
    return x;
}

// Paired FP16 tests of one 32 x 32 chunk whose pairs are all valid (i < j
// < R for every row of the warp and every column) and whose counts, staged
// values and sums are integers FP16 holds exactly: two counts per
// HADD2/HSET2.  Leaves in *cm the D_ij bits and in *rm the D_ji bits of
// this lane's row (bit k: column 2k, bit 16 + k: column 2k + 1).  Without a
// mutual pair (both bits set at one position) the tie-breaks reduce to D_ij
// for column j and D_ji for row i.
// kMode 0: DP  D_ij = [x + f_i - s_i >= f_j], D_ji = [x + f_j - s_j >= f_i]
//       1: SE  D_ij = [x = s_i and f_i >= f_j], D_ji = [x = s_j and f_j >= f_i]
//       2: MD  D_ij = [x = d_j], D_ji = [x = d_i]
template <int kMode>
__device__ __forceinline__ void paired_masks(const uint32_t *x, const __half *colA,
                                             const __half *colB, __half2 rf2, __half2 ra2,
                                             uint32_t *cm_out, uint32_t *rm_out) {
    uint4 av[4], bv[4];  // the chunk's 32 column values (broadcast loads)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        av[q] = reinterpret_cast<const uint4 *>(colA)[q];
        bv[q] = reinterpret_cast<const uint4 *>(colB)[q];
    }
    const uint32_t *aw = reinterpret_cast<const uint32_t *>(av);
    const uint32_t *bw = reinterpret_cast<const uint32_t *>(bv);
    uint32_t cm = 0, rm = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const __half2 x2 = as_h2(x[k]);
        const __half2 a2 = as_h2(aw[k]), b2 = as_h2(bw[k]);
        const uint32_t sel = (1u << k) | (1u << (16 + k));
        uint32_t mij, mji;
        if (kMode == 0) {
            mij = __hge2_mask(__hadd2(x2, ra2), a2);  // x + f_i - s_i >= f_j
            mji = __hge2_mask(__hadd2(x2, b2), rf2);  // x + f_j - s_j >= f_i
        } else if (kMode == 1) {
            mij = __heq2_mask(x2, ra2) & __hge2_mask(rf2, a2);  // x = s_i, f_i >= f_j
            mji = __heq2_mask(x2, b2) & __hge2_mask(a2, rf2);   // x = s_j, f_j >= f_i
        } else {
            mij = __heq2_mask(x2, a2);   // x = d_j
            mji = __heq2_mask(x2, rf2);  // x = d_i
        }
        cm |= mij & sel;
        rm |= mji & sel;
    }
    *cm_out = cm;
    *rm_out = rm;
}

// The paired bit order (bit k: column 2k, bit 16 + k: column 2k + 1) back to
// bit c = column c.
__device__ __forceinline__ uint32_t unpair(uint32_t m) {
    auto spread = [](uint32_t v) {
        v = (v | (v << 8)) & 0x00FF00FFu;
        v = (v | (v << 4)) & 0x0F0F0F0Fu;
        v = (v | (v << 2)) & 0x33333333u;
        return (v | (v << 1)) & 0x55555555u;
    };
    return spread(m & 0xFFFFu) | (spread(m >> 16) << 1);
}

// All interior chunks of a drained tile, without a branch or a vote between
// them, so that their tests overlap; the votes come after.
template <int kMode, int kChunks>
__device__ __forceinline__ void paired_tile(const uint32_t *pk, const __half *colA,
                                            const __half *colB, __half2 rf2, __half2 ra2,
                                            uint32_t inter, uint32_t *cm, uint32_t *rm) {
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
        cm[c] = rm[c] = 0u;
        if ((inter >> c) & 1u)
            paired_masks<kMode>(pk + c * 16, colA + c * 32, colB + c * 32, rf2, ra2, &cm[c],
                                &rm[c]);
    }
}

template <int kN, int kPhase>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_contract(InstState *st, const Plan *plan, BatchCounters *ctr, int32_t *kerr) {
    using S = Shape<kN>;
    constexpr int phase = kPhase;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte alignment for the swizzle atoms
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    SharedCtl<kN> *ctl = reinterpret_cast<SharedCtl<kN> *>(smem + S::kStages * S::kStageBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort = &ctl->abort;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S::kStages; ++s) {
            mbar_init(smem_u32(&ctl->full[s]), 1);
            mbar_init(smem_u32(&ctl->empty[s]), 1);
        }
        for (int a = 0; a < S::kAcc; ++a) {
            mbar_init(smem_u32(&ctl->tmem_full[a]), 1);
            mbar_init(smem_u32(&ctl->tmem_empty[a]), kEpiThreads);
        }
        // a slot is written by the scheduler's 32 lanes and read by the
        // producer, the MMA thread and each epilogue warp
        for (int r = 0; r < kRing; ++r) {
            mbar_init(smem_u32(&ctl->ring_full[r]), 32);
            mbar_init(smem_u32(&ctl->ring_empty[r]), 3);
        }
        mbar_init(smem_u32(&ctl->drain), 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&ctl->tmem_base)),
                     "n"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;
    // A reader is done with ring entry k.
    auto ring_release = [&](int k) { mbar_arrive(smem_u32(&ctl->ring_empty[k % kRing])); };
    // Wait for ring entry k (false on abort).
    auto ring_wait = [&](int k) -> bool {
        const uint32_t bar = smem_u32(&ctl->ring_full[k % kRing]);
        const uint32_t par = (k / kRing) & 1;
        return mbar_wait(bar, par, abort, kWaitNs);
    };

    if (warp == 0) {
        // ------------------------------------------------ TMA producer --
        if (lane == 0) {
            int stage = 0;
            uint32_t phase_bit = 0;
            int64_t issued = 0;
            bool aborted = false;
            const bool halves_on = plan->half_stages != 0;
            const void *tmap = nullptr, *tmap64 = nullptr;
            int tmap_b = -1;
            for (int it = 0;; ++it) {
                if (!ring_wait(it)) {
                    aborted = true;
                    break;
                }
                const TileSlot &ts = ctl->slot[it % kRing];
                const int64_t entry = *reinterpret_cast<const volatile int64_t *>(&ts.entry);
                if (entry < 0) {
                    ring_release(it);
                    break;
                }
                if (entry & kTileNoK) {  // nothing to load; the MMA thread skips it too
                    ring_release(it);
                    continue;
                }
                const int b = ts.b;
                if (b != tmap_b) {  // the maps were written to global memory by a copy
                    const InstState &s = st[b];
                    tmap = phase == 0 ? s.tmap_A : s.tmap_At;  // full map, then half map
                    tmap64 = static_cast<const uint8_t *>(tmap) + kTmapBytes;
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap)
                                 : "memory");
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap64)
                                 : "memory");
                    tmap_b = b;
                }
                const int32_t yi = ts.bi * kTcM, yj = ts.bj * kN;
                const int32_t nkw = ts.nkw;
                // The shared K blocks, from the slot's masks (words past
                // kMaskWords, for K > 131,072, straight from global memory).
                int32_t w = -1;
                uint32_t mask = 0;
                auto next_kb = [&](uint32_t *halves) -> int32_t {
                    while (mask == 0) {
                        if (++w >= nkw) return -1;
                        if (w < kMaskWords) {
                            mask = ts.mask[w];
                        } else {
                            KIter k;
                            TileInfo t2;
                            t2.b = b; t2.bi = ts.bi; t2.bj = ts.bj; t2.R = ts.R; t2.nk = ts.nk;
                            kit_init(k, st[b], phase, t2, S::kRatio);
                            mask = k.all ? (2 * ts.nk - 32 * w >= 32 ? 0xffffffffu
                                                                      : ((1u << (2 * ts.nk - 32 * w)) - 1u))
                                         : (__ldg(k.a + w) & (__ldg(k.b0 + w) |
                                                               (k.b1 ? __ldg(k.b1 + w) : 0u)));
                        }
                    }
                    const int32_t bit = (__ffs(mask) - 1) & ~1;  // the K block's two bits
                    *halves = (mask >> bit) & 3u;
                    mask &= ~(3u << bit);
                    return (w * 32 + bit) >> 1;
                };
                uint32_t hv = 3u;
                int32_t kb = next_kb(&hv);
                while (kb >= 0) {
                    // one K block ahead: the MMA thread learns from the stage
                    // whether it ends the tile, and walks no occupancy bits
                    uint32_t hv_next = 3u;
                    const int32_t kb_next = next_kb(&hv_next);
                    if (!mbar_wait(smem_u32(&ctl->empty[stage]), phase_bit ^ 1, abort, kWaitNs)) {
                        aborted = true;
                        break;
                    }
                    // a whole K block, or one shared half: kOccK columns at x (a
                    // multiple of 64 bytes) through the half map, into the front
                    // of each slot; the flag tells the MMA thread which, and
                    // whether the stage ends its tile (published by the arrive)
                    const bool whole = hv == 3u || !halves_on;
                    ctl->stage_last[stage] = (kb_next < 0 ? 1u : 0u) | (whole ? 0u : 2u);
                    const uint32_t full = smem_u32(&ctl->full[stage]);
                    const uint32_t sa = smem_u32(smem + stage * S::kStageBytes);
                    const uint32_t sb = sa + kABytes;
                    const void *map = whole ? tmap : tmap64;
                    const int32_t x = kb * kTcK + (whole ? 0 : (hv == 2u ? kOccK : 0));
                    const uint32_t box = whole ? (uint32_t)kABytes : (uint32_t)kHalfBox;
                    mbar_expect_tx(full, whole ? S::kStageBytes : S::kHalfStageBytes);
                    tma_load_2d(sa, map, x, yi, full);
#pragma unroll
                    for (int q = 0; q < S::kRatio; ++q)
                        tma_load_2d(sb + q * box, map, x, yj + q * kTcM, full);
                    ++issued;
                    if (++stage == S::kStages) { stage = 0; phase_bit ^= 1; }
                    kb = kb_next;
                    hv = hv_next;
                }
                ring_release(it);  // done with the slot's masks
                if (aborted) break;
            }
            if (aborted) {  // let the loads still in flight land before exiting
                for (int64_t k = issued > S::kStages ? issued - S::kStages : 0; k < issued; ++k)
                    mbar_wait_ns(smem_u32(&ctl->full[k % S::kStages]),
                                 (uint32_t)((k / S::kStages) & 1), 100000000ull);
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------- MMA issuer --
        if (lane == 0) {
            int stage = 0;
            uint32_t phase_bit = 0;
            int it = 0;
            bool aborted = false;
            unsigned long long n_kblocks = 0, n_tiles = 0;
            // The tile list flags tiles without a shared K block; the
            // producer flags the last stage of every other tile.
            for (;; ++it) {
                if (!ring_wait(it)) {
                    aborted = true;
                    break;
                }
                const int64_t cur =
                    *reinterpret_cast<const volatile int64_t *>(&ctl->slot[it % kRing].entry);
                ring_release(it);  // done with entry `it`
                if (cur < 0) break;
                const bool has_k = (cur & kTileNoK) == 0;
                const int acc = it % S::kAcc;
                const uint32_t acc_phase = (it / S::kAcc) & 1;
                if (!mbar_wait(smem_u32(&ctl->tmem_empty[acc]), acc_phase ^ 1, abort, kWaitNs)) {
                    aborted = true;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + acc * kN;
                bool first = true;
                ++n_tiles;
                for (bool last = !has_k; !last;) {
                    if (!mbar_wait(smem_u32(&ctl->full[stage]), phase_bit, abort, kWaitNs)) {
                        aborted = true;
                        break;
                    }
                    tc_fence_after();
                    // The flag must be read before this stage goes back to the
                    // producer: the first MMA's accumulate flag depends on the
                    // loaded word (which is below 4), so the MMAs, and the
                    // commit that releases the stage, issue after the load.
                    const uint32_t lastw =
                        *reinterpret_cast<volatile uint32_t *>(&ctl->stage_last[stage]);
                    last = (lastw & 1u) != 0;
                    const uint32_t sa = smem_u32(smem + stage * S::kStageBytes);
                    const uint32_t sb = sa + kABytes;
                    // K = 32 per MMA: four for a whole K block, two for a half
                    const bool half_st = (lastw & 2u) != 0;
                    const uint64_t layout = half_st ? kDescHalf : kDescFull;
                    const int nmma = half_st ? kOccK / 32 : kTcK / 32;
#pragma unroll
                    for (int k = 0; k < kTcK / 32; ++k)
                        if (k < nmma)
                            mma_f8<S::kIdesc>(d, smem_desc(layout, sa + 32 * k),
                                              smem_desc(layout, sb + 32 * k),
                                              (!first || k > 0 || lastw == 4u) ? 1u : 0u);
                    first = false;
                    // work counter in units of 128 x 128 x 32 MACs
                    n_kblocks += (unsigned long long)nmma * S::kRatio;
                    mma_commit(smem_u32(&ctl->empty[stage]));
                    if (++stage == S::kStages) { stage = 0; phase_bit ^= 1; }
                }
                if (aborted) break;
                mma_commit(smem_u32(&ctl->tmem_full[acc]));
            }
            if (aborted) {  // wait for the MMAs already issued before freeing TMEM
                mma_commit(smem_u32(&ctl->drain));
                mbar_wait_ns(smem_u32(&ctl->drain), 0, 100000000ull);
            }
            if (ctr && n_tiles) {
                atomicAdd(&ctr->mma_kblocks, n_kblocks);
                atomicAdd(&ctr->mma_tiles, n_tiles);
            }
        }
    } else if (warp < kSchedWarp) {
        // ------------------------------------------------------ epilogue --
        // Warp w tests 32 rows (TMEM lane quarter q) by kN / 2 columns
        // (half) of every tile.  The epilogue threads stage one column
        // record each and meet once per tile.
        const int q = warp & 3;             // TMEM lane quarter
        const int half = (warp - 2) >> 2;   // which kN/2 columns of the tile
        const int et = threadIdx.x - 64;
        const bool stages_col = et < kN;    // this thread stages column j0 + et
        // The next tile's records, loaded into registers while this tile
        // waits for its accumulator and is tested (the records do not
        // change during a launch): the entry they belong to, or -1.
        int64_t pre_entry = -1;
        int4 pre_col = make_int4(0, 0, 0, 0), pre_row = make_int4(0, 0, 0, 0);
        for (int it = 0;; ++it) {
            const int slot = it % kRing;
            // every exit below is decided by a barrier's result, the same for
            // all epilogue threads: none may leave while others still wait
            // at a barrier (which has no time limit)
            const bool ok = ring_wait(it);
            const TileSlot &ts = ctl->slot[slot];
            const int64_t entry = *reinterpret_cast<const volatile int64_t *>(&ts.entry);
            const int b = ts.b;
            const int32_t R = ts.R;
            const int32_t j0 = ts.bj * kN;              // first column of the tile
            const int32_t jw = j0 + half * S::kCols;    // first column of this warp
            const int32_t wi0 = ts.bi * kTcM + 32 * q;  // first row of this warp
            const int32_t i = wi0 + lane;
            TileCols<kN> &C = ctl->cols[it & 1];
            const bool have = pre_entry == entry;
            bool vals_small = true;  // every staged value bounds its counts by kSmallMax
            int4 rrec = make_int4(0, 0, 0, 0);
            const InstState *sp = ok && entry >= 0 ? &st[b] : nullptr;
            if (sp) {
                if (stages_col) {  // column j0 + et
                    const int4 rec = have ? pre_col : epi_record(*sp, phase, j0 + et, R);
                    const float a = (float)rec.x, bb = (float)rec.y;
                    C.ab[et] = make_float2(a, bb);
                    C.o[et] = rec.z;
                    C.a16[et] = __float2half_rn(a);
                    C.b16[et] = __float2half_rn(bb);
                    vals_small = record_small(rec);
                }
                // DP: f_i, f_i - s_i ; SE: f_i, s_i ; MD: d_i ; and the input index of row i
                rrec = have ? pre_row : epi_record(*sp, phase, i, R);
                vals_small = vals_small && record_small(rrec);
            }
            // Every count of a tile is at most the size (DP, SE) or degree
            // (MD) of its row and of its column, so a tile whose staged
            // values are all small has only counts <= kSmallMax, which FP16
            // holds exactly, as it does every sum the tests form.  The one
            // barrier per tile also publishes the staged columns, and orders
            // every read of the slot before its release.
            bool tile_small = epi_bar_and(ok && vals_small);
            if (!tile_small && !epi_bar_and(ok)) {  // a second barrier only if not small
                *abort = 1;
                break;
            }
            if (entry < 0) break;  // read after a successful wait by every thread
            if (et == 0) ring_release(it);
            // fields of the tile's instance, read once per tile
            uint8_t *const e_del = sp->e_del;
            int32_t *const v_cnt = sp->v_cnt;
            const bool se = phase == 0 && sp->edge_rule != 0;  // DP stages f, f - s; SE f, s
            // A count of 0 changes nothing unless some hyperedge has f > |e| (DP)
            // or is empty (SE): only from such a hyperedge does x = 0 delete; in
            // MD a zero count matches no staged degree (see epi_record).
            const bool zero_matters = phase == 0 && sp->has_loose;
            const float ri_f = (float)rrec.x, ri_a = (float)rrec.y;
            const int32_t ri_o = rrec.z;
            const int acc = it % S::kAcc;
            const uint32_t acc_phase = (it / S::kAcc) & 1;
            // Load the next tile's records if its slot is published (it
            // usually is: the scheduler runs ahead).
            pre_entry = -1;
            {
                const int nk = it + 1;
                const uint32_t nbar = smem_u32(&ctl->ring_full[nk % kRing]);
                const uint32_t npar = (nk / kRing) & 1;
                if (mbar_try(nbar, npar)) {
                    const TileSlot &ns_ = ctl->slot[nk % kRing];
                    const int64_t ne = *reinterpret_cast<const volatile int64_t *>(&ns_.entry);
                    if (ne >= 0) {
                        const InstState &ns = st[ns_.b];
                        if (stages_col) pre_col = epi_record(ns, phase, ns_.bj * kN + et, ns_.R);
                        pre_row = epi_record(ns, phase, ns_.bi * kTcM + 32 * q + lane, ns_.R);
                        pre_entry = ne;
                    }
                }
            }
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&ctl->tmem_full[acc]), acc_phase,
                                                   abort, kWaitNs))) {
                // the next tile's barrier takes every epilogue thread out
                *abort = 1;
                continue;
            }
            tc_fence_after();
            bool rowflag = false;
            int32_t rowcnt = 0;
            // A tile contracts at least one K block, so its accumulator holds
            // its counts -- except a tile the list flags as having no shared K
            // block (kept only in a DP pass where zero counts matter), which
            // the MMA thread skips, leaving the accumulator stale.
            const bool nonzero = (entry & kTileNoK) == 0;
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + acc * kN + half * S::kCols;
            const int cw = half * S::kCols;  // this warp's first column in C
            // Publish the column flags of this warp's chunk c: DP marks the
            // columns for deletion, MD adds to each column the number of this
            // warp's rows that dominate it (a bit-matrix transpose gives lane
            // l the column l).
            auto put_cols = [&](uint32_t colmask, int c) {
                if (phase == 0) {
                    const uint32_t any = __reduce_or_sync(0xffffffffu, colmask);
                    if ((any >> lane) & 1u) e_del[jw + c * 32 + lane] = 1;
                } else if (__any_sync(0xffffffffu, colmask != 0)) {
                    const int n1 = __popc(warp_transpose32(colmask, lane));
                    if (n1) atomicAdd(&v_cnt[jw + c * 32 + lane], n1);
                }
            };
            // chunk c of this warp holds only pairs i < j < R
            auto interior = [&](int c) {
                const int32_t jc0 = jw + c * 32;
                return wi0 + 31 < R && jc0 + 31 < R && jc0 > wi0 + 31;
            };
            uint32_t slow_chunks = 0;  // chunks that need the full test (bit c)
            // drained counts of this thread's row, two per FP16x2 word
            uint32_t pk[S::kChunks * 16];
            if (tile_small) {
                // Drain, then give the accumulator back before testing.
                if (nonzero) {
#pragma unroll
                    for (int c = 0; c < S::kChunks; c += 2) {
                        uint32_t r0[32], r1[32];
                        tmem_ld32_issue(taddr + c * 32, r0);
                        tmem_ld32_issue(taddr + (c + 1) * 32, r1);
                        tmem_wait(r0);
                        tmem_after_wait(r1);
#pragma unroll
                        for (int k = 0; k < 16; ++k) {
                            pk[c * 16 + k] = pack_h2(__uint_as_float(r0[2 * k]),
                                                     __uint_as_float(r0[2 * k + 1]));
                            pk[(c + 1) * 16 + k] = pack_h2(__uint_as_float(r1[2 * k]),
                                                           __uint_as_float(r1[2 * k + 1]));
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < S::kChunks * 16; ++k) pk[k] = 0u;
                }
                tc_fence_before();
                mbar_arrive(smem_u32(&ctl->tmem_empty[acc]));
                const __half2 rf2 = __float2half2_rn(ri_f), ra2 = __float2half2_rn(ri_a);
                // Interior chunks take the paired tests.  Running them on a
                // chunk of zero counts sets nothing: without a hyperedge of
                // f > |e| (DP) or an empty one (SE) a zero count supersedes
                // nothing, and in MD no staged degree is 0 (see epi_record).
                uint32_t inter = 0;
#pragma unroll
                for (int c = 0; c < S::kChunks; ++c) inter |= (interior(c) ? 1u : 0u) << c;
                uint32_t cm[S::kChunks], rm[S::kChunks];
                const __half *ca = C.a16 + cw, *cb = C.b16 + cw;
                if (phase == 1)
                    paired_tile<2, S::kChunks>(pk, ca, cb, rf2, ra2, inter, cm, rm);
                else if (se)
                    paired_tile<1, S::kChunks>(pk, ca, cb, rf2, ra2, inter, cm, rm);
                else
                    paired_tile<0, S::kChunks>(pk, ca, cb, rf2, ra2, inter, cm, rm);
#pragma unroll
                for (int c = 0; c < S::kChunks; ++c) {
                    if ((inter >> c) & 1u) {
                        if (__any_sync(0xffffffffu, (cm[c] & rm[c]) != 0)) {
                            slow_chunks |= 1u << c;  // a mutual pair: the tie-breaks decide
                        } else {
                            if (phase == 0) rowflag |= rm[c] != 0;
                            else rowcnt += __popc(rm[c]);
                            put_cols(unpair(cm[c]), c);
                        }
                    } else {
                        // diagonal or ragged chunk: the full test, unless all its
                        // counts are zero and zero counts cannot matter
                        uint32_t nz = 0;
#pragma unroll
                        for (int k = 0; k < 16; ++k) nz |= pk[c * 16 + k];
                        if (zero_matters || __any_sync(0xffffffffu, nz != 0))
                            slow_chunks |= 1u << c;
                    }
                }
            } else {
                // Large values: FP32 tests straight from TMEM, chunk by chunk.
#pragma unroll 1
                for (int c = 0; c < S::kChunks; ++c) {
                    float v[32];
                    if (nonzero) {
                        tmem_ld32(taddr + c * 32, v);
                    } else {
#pragma unroll
                        for (int k = 0; k < 32; ++k) v[k] = 0.f;
                    }
                    float m16[16];  // the chunk's maximum count, as a tree
#pragma unroll
                    for (int k = 0; k < 16; ++k) m16[k] = fmaxf(v[k], v[k + 16]);
#pragma unroll
                    for (int w = 8; w > 0; w >>= 1)
#pragma unroll
                        for (int k = 0; k < w; ++k) m16[k] = fmaxf(m16[k], m16[k + w]);
                    // skip 32 x 32 blocks of zero counts (counts are >= 0)
                    if (!zero_matters && !__any_sync(0xffffffffu, m16[0] > 0.f)) continue;
                    bool slow = !interior(c);
                    if (!slow) {
                        const float2 *cab = C.ab + cw + c * 32;
                        uint32_t cm = 0, rm = 0;
#pragma unroll
                        for (int k = 0; k < 32; ++k) {
                            const float x = v[k];
                            const float2 ab = cab[k];
                            bool dij, dji;
                            if (phase == 0) {
                                dij = se ? (x == ri_a && ri_f >= ab.x) : x + ri_a >= ab.x;
                                dji = se ? (x == ab.y && ab.x >= ri_f) : x + ab.y >= ri_f;
                            } else {
                                dij = x == ab.x;  // x = d_j
                                dji = x == ri_f;  // x = d_i
                            }
                            cm |= (uint32_t)dij << k;
                            rm |= (uint32_t)dji << k;
                        }
                        slow = __any_sync(0xffffffffu, (cm & rm) != 0);
                        if (!slow) {
                            if (phase == 0) rowflag |= rm != 0;
                            else rowcnt += __popc(rm);
                            put_cols(cm, c);
                        }
                    }
                    if (slow) slow_chunks |= 1u << c;
                }
            }
            // Full test (diagonal / ragged chunks, or a mutual pair present):
            // validity mask and the input-index tie-breaks of Algorithms 1
            // and 2.  The counts come back from the packed registers (drained
            // tiles; static register indices through the chunk selection) or
            // again from TMEM.
#pragma unroll 1
            for (uint32_t sc = slow_chunks; sc;) {
                const int c = __ffs(sc) - 1;
                sc &= sc - 1;
                float v[32];
                if (tile_small) {
                    uint32_t w[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) w[k] = pk[k];
#pragma unroll
                    for (int cc = 1; cc < S::kChunks; ++cc)
                        if (cc == c)
#pragma unroll
                            for (int k = 0; k < 16; ++k) w[k] = pk[cc * 16 + k];
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const __half2 h = as_h2(w[k]);
                        v[2 * k] = __low2float(h);
                        v[2 * k + 1] = __high2float(h);
                    }
                } else if (nonzero) {
                    tmem_ld32(taddr + c * 32, v);
                } else {
#pragma unroll
                    for (int k = 0; k < 32; ++k) v[k] = 0.f;
                }
                uint32_t colmask = 0;
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const int cc = cw + c * 32 + k;
                    const int32_t j = j0 + cc;
                    const bool valid = (i < j) && (j < R);
                    const float x = v[k];
                    const float2 ab = C.ab[cc];
                    const bool i_first = ri_o < C.o[cc];  // input-index tie-break
                    if (phase == 0) {
                        // Algorithm 1: D_ij = [f_i - (s_i - x) >= f_j] (rule SE:
                        // [x = s_i and f_i >= f_j]); e_j goes iff D_ij and
                        // (not D_ji or i before j)
                        const bool dij = se ? (x == ri_a && ri_f >= ab.x) : x + ri_a >= ab.x;
                        const bool dji = se ? (x == ab.y && ab.x >= ri_f) : x + ab.y >= ri_f;
                        colmask |= (uint32_t)(valid && dij && (!dji || i_first)) << k;
                        rowflag |= valid && dji && (!dij || !i_first);
                    } else {
                        // Algorithm 2: D_ij = [x = d_j and (x != d_i or i before j)]
                        const bool eqj = x == ab.x;
                        const bool eqi = x == ri_f;
                        colmask |= (uint32_t)(valid && eqj && (!eqi || i_first)) << k;
                        rowcnt += (int32_t)(valid && eqi && (!eqj || !i_first));
                    }
                }
                put_cols(colmask, c);
            }
            if (!tile_small) {  // a drained tile gave its accumulator back already
                tc_fence_before();
                mbar_arrive(smem_u32(&ctl->tmem_empty[acc]));
            }
            if (phase == 0) {
                if (rowflag) e_del[i] = 1;
            } else {
                if (rowcnt) atomicAdd(&v_cnt[i], rowcnt);
            }
        }
    }
    if (warp == kSchedWarp) {
        // ---------------------------------------------- tile scheduler --
        // Takes the next tile-list entry, ANDs the occupancy words of its
        // row block and column block (lane w: words w, w + 32, ...) into the
        // slot and publishes it; every lane arrives on the slot's barrier
        // after its own writes.  Runs at most kRing slots ahead of the
        // slowest reader.
        bool heavy_left = true, light_left = true;  // (lane 0: a queue once empty stays so)
        for (int k = 0;; ++k) {
            const int sl = k % kRing;
            bool ok = true;
            if (lane == 0)
                ok = mbar_wait(smem_u32(&ctl->ring_empty[sl]), ((k / kRing) & 1) ^ 1, abort,
                               kWaitNs);
            if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
            int64_t e = -1;
            if (lane == 0) {
                // alternate the heavy (front) and light (back) queues; when one
                // is empty, take from the other (a list of one queue: only it)
                const int first = plan->list_light == 0 ? 0 : (int)((k + blockIdx.x) & 1);
                for (int q = 0; q < 2 && e < 0; ++q) {
                    if (((first + q) & 1) == 0) {
                        if (heavy_left) {
                            const int32_t t =
                                atomicAdd(const_cast<int32_t *>(&plan->list_next), 1);
                            if (t < plan->list_count) e = plan->tile_list[t];
                            else heavy_left = false;
                        }
                    } else if (light_left) {
                        const int32_t t =
                            atomicAdd(const_cast<int32_t *>(&plan->list_next_light), 1);
                        if (t < plan->list_light) e = plan->tile_list[plan->list_cap - 1 - t];
                        else light_left = false;
                    }
                }
            }
            e = __shfl_sync(0xffffffffu, e, 0);
            TileSlot &ts = ctl->slot[sl];
            if (e >= 0) {
                TileInfo ti;
                tile_info(st, phase, e, &ti);
                const int32_t nbits = 2 * ti.nk;  // occupancy bits of the K range
                const int32_t nkw = (nbits + 31) / 32;
                if ((e & kTileNoK) == 0) {
                    KIter kt;
                    kit_init(kt, st[ti.b], phase, ti, S::kRatio);
                    for (int w = lane; w < nkw && w < kMaskWords; w += 32) {
                        uint32_t m;
                        if (kt.all) {
                            const int32_t left = nbits - 32 * w;
                            m = left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
                        } else {
                            uint32_t bm = __ldg(kt.b0 + w);
                            if (kt.b1) bm |= __ldg(kt.b1 + w);
                            m = __ldg(kt.a + w) & bm;
                        }
                        ts.mask[w] = m;
                    }
                }
                if (lane == 0) {
                    ts.b = ti.b;
                    ts.bi = ti.bi;
                    ts.bj = ti.bj;
                    ts.R = ti.R;
                    ts.nk = ti.nk;
                    ts.nkw = nkw;
                }
            }
            if (lane == 0) ts.entry = e;
            mbar_arrive(smem_u32(&ctl->ring_full[sl]));
            if (e < 0) break;
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort) atomicOr(kerr, kErrTimeout);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "n"(kTmemCols)
                     : "memory");
    }
}

}  // namespace

// Host side ----------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Two 2D uint8 tensor maps over a rows x pitch byte matrix, 128-row boxes;
// out-of-range rows read as zero: a full stage (box 128 bytes wide, 128-byte
// swizzle), then a half stage (box 64 bytes wide, 64-byte swizzle).
static_assert(sizeof(CUtensorMap) == kTmapBytes, "tensor map size");
bool make_operand_tmap(void *out, const void *base, int64_t pitch, int64_t rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = get_encode_fn();
    if (!fn) return false;
    for (int h = 0; h < 2; ++h) {
        CUtensorMap m;
        std::memset(&m, 0, sizeof(m));
        cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
        cuuint64_t strides[1] = {(cuuint64_t)pitch};
        cuuint32_t box[2] = {(cuuint32_t)(h ? kOccK : kTcK), (cuuint32_t)kTcM};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        h ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
        std::memcpy(static_cast<uint8_t *>(out) + h * kTmapBytes, &m, sizeof(m));
    }
    return true;
}

size_t tmap_bytes() { return 2 * sizeof(CUtensorMap); }

cudaError_t prepare_tc_contract() {
    static cudaError_t once = [] {
        cudaError_t e = cudaSuccess;
        auto set = [&](const void *fn, size_t bytes) {
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
        };
        set((const void *)k_tc_contract<256, 0>, smem_bytes<256>());
        set((const void *)k_tc_contract<256, 1>, smem_bytes<256>());
        set((const void *)k_tc_contract<128, 0>, smem_bytes<128>());
        set((const void *)k_tc_contract<128, 1>, smem_bytes<128>());
        return e;
    }();
    return once;
}

cudaError_t launch_tc_contract(InstState *st, Plan *plan, BatchCounters *ctr, int phase, int sms,
                               int tile_n, int32_t *kerr, cudaStream_t s) {
    if (tile_n == 128) {
        if (phase == 0)
            k_tc_contract<128, 0><<<sms, kThreads, smem_bytes<128>(), s>>>(st, plan, ctr, kerr);
        else
            k_tc_contract<128, 1><<<sms, kThreads, smem_bytes<128>(), s>>>(st, plan, ctr, kerr);
    } else {
        if (phase == 0)
            k_tc_contract<256, 0><<<sms, kThreads, smem_bytes<256>(), s>>>(st, plan, ctr, kerr);
        else
            k_tc_contract<256, 1><<<sms, kThreads, smem_bytes<256>(), s>>>(st, plan, ctr, kerr);
    }
    return cudaGetLastError();
}

int32_t tile_group_rows() {
    static int32_t g = [] {
        const char *e = std::getenv("MHS_TILE_GROUP_ROWS");
        const int v = e ? std::atoi(e) : 0;
        return (int32_t)(v >= 1 && v <= 4096 ? v : kGroupRows);
    }();
    return g;
}

cudaError_t launch_tc_tile_list(InstState *st, Plan *plan, int phase, int sms, cudaStream_t s,
                                int shard, int nshards) {
    k_tile_list<<<sms * 4, 256, 0, s>>>(st, plan, phase, shard, nshards);
    return cudaGetLastError();
}

}  // namespace mhs

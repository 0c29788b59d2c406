// contract_tc.cu -- tcgen05 tensor-core contraction of the 0/1 incidence
// operands with the fused DP / MD epilogue (sm_103a).
//
// For each tile of 128 rows i x 256 columns j of the upper triangle, the
// kernel computes x_ij = sum_k X_ik X_jk, i.e. I^E_ij of Eq. (1) for
// X = A (phase 0, DP) or I^V_ij of Eq. (2) for X = A^T (phase 1, MD), with
// both operands taken from the same K-major FP8 E4M3 matrix (0x38 = 1.0,
// 0x00 = 0).  Products are 0/1 and the FP32 accumulator holds integers
// below 2^24, so x_ij is exact.  The counts stay in TMEM: the epilogue warps
// read them with tcgen05.ld and apply Algorithm 1 (DP) or Algorithm 2 (MD)
// directly; the matrix I is never written.
//
// Warp roles (320 threads, one CTA per SM, persistent over the tile list):
//   warp 0      TMA producer: 128-byte-swizzled K slices of the i rows
//               (128 x 128 B) and j rows (2 x 128 x 128 B) into a 4-stage
//               shared-memory ring.
//   warp 1      TMEM allocation (512 columns = two 128 x 256 FP32
//               accumulators) and the single-thread tcgen05.mma issuer.
//   warps 2-9   epilogue; warp w reads TMEM lanes 32*(w%4) .. +31, warps
//               2-5 columns 0-127 and warps 6-9 columns 128-255 of a tile.
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

constexpr int kStages = 4;
constexpr int kABytes = kTcM * kTcK;            // 16 KB
constexpr int kBBytes = kTcN * kTcK;            // 32 KB
constexpr int kStageBytes = kABytes + kBBytes;  // 48 KB
// A stage whose K block shares a nonzero in only one of its two halves
// loads just that half (kOccK columns of each operand, 64-byte swizzle,
// 8 KB per 128-row box) into the front of the same slots.
constexpr int kHalfBox = kTcM * kOccK;          // 8 KB
constexpr int kHalfStageBytes = 3 * kHalfBox;   // 24 KB
static_assert(2 * kOccK == kTcK, "a stage is two occupancy blocks");
// An operand's tensor maps: the full-stage map, then the half-stage map.
constexpr int kTmapBytes = 128;
constexpr int kAccCols = kTcN;                  // FP32 columns per accumulator
constexpr int kTmemCols = 2 * kAccCols;         // 512
constexpr int kEpiWarps = 8;                    // two per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;   // producer + MMA + epilogue
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kGroupRows = 16;                  // default row blocks per L2 group
constexpr uint64_t kWaitNs = 4000000000ull;     // 4 s bound on any wait

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
// Instruction descriptor, kind::f8f6f4: D = F32, A = B = E4M3, both K-major,
// N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

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
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}
__device__ __forceinline__ void epi_bar() {  // named barrier among the 4 epilogue warps
    asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
}
// Named barrier among the epilogue warps that also ANDs a flag, so that all
// four take the same branch after a wait.
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

// Tiles of one instance: row block bi (128 rows) x column block bj (256
// columns), kept iff it holds a pair i < j, i.e. bj >= floor(bi / 2).
// prefix(bi) = number of tiles in row blocks < bi.
__device__ __forceinline__ int64_t tc_prefix(int64_t bi, int64_t cb) {
    return bi * cb - (bi / 2) * ((bi - 1) / 2 > 0 ? (bi - 1) / 2 : 0);
}

// Order: groups of G row blocks; inside a group, column block by column
// block, and inside a column block the group's row blocks.  With G = 16,
// about 152 concurrent tiles share 16 row blocks and ~10 column blocks,
// which keeps their K slices in L2.
__device__ void tc_tile_coords(int64_t t, int32_t R, int32_t G, int32_t *bi_out,
                               int32_t *bj_out) {
    const int32_t rb = tc_row_blocks(R), cb = tc_col_blocks(R);
    const int32_t ng = (rb + G - 1) / G;
    int32_t lo = 0, hi = ng;  // find group g: prefix(g*G) <= t < prefix((g+1)*G)
    while (hi - lo > 1) {
        int32_t mid = (lo + hi) >> 1;
        if (tc_prefix((int64_t)mid * G, cb) <= t) lo = mid; else hi = mid;
    }
    const int32_t g = lo;
    const int32_t r0 = g * G;
    const int32_t gsz = min(G, rb - r0);
    int64_t p = t - tc_prefix(r0, cb);
    int32_t bj = r0 / 2;  // first column block of the group
    for (;;) {
        // row blocks bi in [r0, r0+gsz) with floor(bi/2) <= bj
        int32_t c = 2 * bj + 2 - r0;
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
// {f, f - |e| (SE: |e|), input id}; MD {deg, 0, input id}.
__device__ __forceinline__ int4 epi_record(const InstState &s, int phase, int32_t j, int32_t R) {
    if (j >= R) return make_int4(0, 0, 0, 0);
    if (phase == 0) return s.e_rec[j];
    return make_int4(s.v_deg[j], 0, s.v_c2o[j], 0);
}

// K blocks of a tile where both operands hold a nonzero: the occupancy
// bits of row block bi AND those of the two row blocks of column block bj.
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
                                         const TileInfo &ti) {
    const uint32_t *base = s.occ[phase];
    const int64_t W = s.occ_words[phase];
    k.a = base + (int64_t)ti.bi * W;
    k.b0 = base + (int64_t)(2 * ti.bj) * W;
    k.b1 = k.b0 + W;
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
            k.mask = __ldg(k.a + k.w) & (__ldg(k.b0 + k.w) | __ldg(k.b1 + k.w));
        }
    }
    const int32_t bit = (__ffs(k.mask) - 1) & ~1;  // the K block's two bits
    k.halves = (k.mask >> bit) & 3u;
    k.mask &= ~(3u << bit);
    return (k.w * 32 + bit) >> 1;
}

// Build this phase's tile list: every tile of the upper triangle (in the
// grouped order of tc_tile_coords) that holds a candidate row or column
// (incremental rounds) and shares a nonzero K block -- or, in a DP pass of
// an instance with a hyperedge f > |e|, every such tile, since zero counts
// can then supersede.  Zero tiles otherwise change nothing: in DP a
// zero count supersedes only from a hyperedge with f > |e|, and in MD a
// zero count only adds dominators of a vertex in no hyperedge, which is
// deleted anyway (its maximum demand is 0).  Warp-aggregated appends keep
// runs of 32 consecutive tiles together.
__global__ void k_tile_list(InstState *st, Plan *plan, int phase) {
    const int lane = threadIdx.x & 31;
    const int64_t total = plan->total_tiles;
    const int32_t G = plan->group_rows > 0 ? plan->group_rows : kGroupRows;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane); base < total;
         base += nw * 32) {
        const int64_t t = base + lane;
        bool keep = false;
        int64_t packed = 0;
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
            tc_tile_coords(t - plan->tile_off[lo], ti.R, G, &ti.bi, &ti.bj);
            bool has_k = true;
            if (s.no_skip) {
                keep = true;  // the dense formulation: every tile, every round
            } else {
                // only tiles that hold a candidate row (incremental rounds) ...
                const uint8_t *drb = phase == 0 ? s.e_dirty_rb : s.v_dirty_rb;
                keep = !drb || (phase == 1 && s.md_full) || drb[ti.bi] || drb[2 * ti.bj] ||
                       drb[2 * ti.bj + 1];
                // ... and share a nonzero K block, unless zero counts matter
                if (keep) {
                    KIter k;
                    kit_init(k, s, phase, ti);
                    has_k = kit_next(k) >= 0;
                    keep = has_k || (phase == 0 && s.has_loose);
                }
            }
            packed = pack_tile(lo, ti.bi, ti.bj) | (has_k ? 0 : kTileNoK);
        }
        const uint32_t ballot = __ballot_sync(0xffffffffu, keep);
        int32_t start = 0;
        if (lane == 0 && ballot) start = atomicAdd(&plan->list_count, __popc(ballot));
        start = __shfl_sync(0xffffffffu, start, 0);
        if (keep) plan->tile_list[start + __popc(ballot & ((1u << lane) - 1))] = packed;
    }
}

// Tiles are handed out dynamically: the producer thread takes the next
// tile-list entry with an atomic and publishes it in a shared ring that the
// MMA thread and the epilogue warps read in the same order.  CTAs that draw
// cheap tiles take more of them, so the tiles in flight at any time stay a
// narrow window of the (L2-grouped) list.
constexpr int kRing = 8;

struct __align__(8) SharedCtl {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t tmem_full[2];
    uint64_t tmem_empty[2];
    uint64_t ring_full[kRing];   // entry published (producer arrives)
    uint64_t ring_empty[kRing];  // entry read by the MMA thread and the epilogue (2 arrivals)
    int64_t ring[kRing];         // packed tile entry, -1 = no more tiles
    uint32_t stage_last[kStages];  // bit 0: the stage ends its tile; bit 1: a half stage
                                   // (written by the producer)
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
    float2 colAB[kTcN];  // DP: (f_j, f_j - s_j)   MD: (d_j, 0)
    int32_t colO[kTcN];  // input index of column j (tie-breaks)
    __half colA16[kTcN];  // colAB as FP16 (exact when |value| <= 1024): the paired fast path
    __half colB16[kTcN];
    int32_t ccnt[kTcN];
};

__global__ void __launch_bounds__(kThreads, 1)
    k_tc_contract(InstState *st, const Plan *plan, BatchCounters *ctr, int phase, int32_t *kerr) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte alignment for the swizzle atoms
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    SharedCtl *ctl = reinterpret_cast<SharedCtl *>(smem + kStages * kStageBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort = &ctl->abort;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&ctl->full[s]), 1);
            mbar_init(smem_u32(&ctl->empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&ctl->tmem_full[a]), 1);
            mbar_init(smem_u32(&ctl->tmem_empty[a]), kEpiThreads);
        }
        // readers of a ring entry: the MMA thread and the epilogue
        for (int r = 0; r < kRing; ++r) {
            mbar_init(smem_u32(&ctl->ring_full[r]), 1);
            mbar_init(smem_u32(&ctl->ring_empty[r]), 2);
        }
        mbar_init(smem_u32(&ctl->drain), 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x >= 64) {
        for (int c = threadIdx.x - 64; c < kTcN; c += kEpiThreads) ctl->ccnt[c] = 0;
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
            const void *fenced = nullptr;
            // Publish ring entry k: wait until both readers are done with the
            // slot's previous entry, take the next list entry, and release it.
            // Returns the entry (-1: the list is exhausted), or -2 on abort.
            auto publish = [&](int k) -> int64_t {
                const int slot = k % kRing;
                if (!mbar_wait(smem_u32(&ctl->ring_empty[slot]), ((k / kRing) & 1) ^ 1, abort,
                               kWaitNs))
                    return -2;
                const int32_t t = atomicAdd(const_cast<int32_t *>(&plan->list_next), 1);
                const int64_t e = t < plan->list_count ? plan->tile_list[t] : -1;
                ctl->ring[slot] = e;
                mbar_arrive(smem_u32(&ctl->ring_full[slot]));
                return e;
            };
            // The next tile (list entry and first shared K block) is fetched
            // while the current one is issued, so a tile start does not wait
            // on global-memory latency.
            TileInfo ti, nx;
            KIter kit, nkit;
            int32_t kb = -1, nkb = -1;
            uint32_t hv = 3u, nhv = 3u;
            int it = 0;
            int64_t cur = publish(0);
            aborted = cur == -2;
            if (cur >= 0) {
                tile_info(st, phase, cur, &ti);
                kit_init(kit, st[ti.b], phase, ti);
                kb = kit_next(kit);
                hv = kit.halves;
            }
            while (cur >= 0 && !aborted) {
                const int64_t nxt = publish(it + 1);
                if (nxt == -2) {
                    aborted = true;
                    break;
                }
                if (nxt >= 0) {
                    tile_info(st, phase, nxt, &nx);
                    kit_init(nkit, st[nx.b], phase, nx);
                    nkb = kit_next(nkit);
                    nhv = nkit.halves;
                }
                const InstState &s = st[ti.b];
                const void *tmap = phase == 0 ? s.tmap_A : s.tmap_At;  // full map, then half map
                const void *tmap64 = static_cast<const uint8_t *>(tmap) + kTmapBytes;
                if (tmap != fenced) {  // the maps were written to global memory by a copy
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap)
                                 : "memory");
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap64)
                                 : "memory");
                    fenced = tmap;
                }
                const int32_t yi = ti.bi * kTcM, yj = ti.bj * kTcN;
                while (kb >= 0) {
                    // one K block ahead: the MMA thread learns from the stage
                    // whether it ends the tile, and walks no occupancy bits
                    const int32_t kb_next = kit_next(kit);
                    const uint32_t hv_next = kit.halves;
                    if (!mbar_wait(smem_u32(&ctl->empty[stage]), phase_bit ^ 1, abort, kWaitNs)) {
                        aborted = true;
                        break;
                    }
                    // a whole K block, or one shared half: kOccK columns at x (a
                    // multiple of 64 bytes) through the half map, into the front
                    // of each slot; the flag tells the MMA thread which, and
                    // whether the stage ends its tile (published by the arrive)
                    const bool whole = hv == 3u;
                    ctl->stage_last[stage] = (kb_next < 0 ? 1u : 0u) | (whole ? 0u : 2u);
                    const uint32_t full = smem_u32(&ctl->full[stage]);
                    const uint32_t sa = smem_u32(smem + stage * kStageBytes);
                    const uint32_t sb = sa + kABytes;
                    const void *map = whole ? tmap : tmap64;
                    const int32_t x = kb * kTcK + (hv == 2u ? kOccK : 0);
                    const uint32_t box = whole ? (uint32_t)kABytes : (uint32_t)kHalfBox;
                    mbar_expect_tx(full, whole ? kStageBytes : kHalfStageBytes);
                    tma_load_2d(sa, map, x, yi, full);
                    tma_load_2d(sb, map, x, yj, full);
                    tma_load_2d(sb + box, map, x, yj + kTcM, full);
                    ++issued;
                    if (++stage == kStages) { stage = 0; phase_bit ^= 1; }
                    kb = kb_next;
                    hv = hv_next;
                }
                cur = nxt;
                ti = nx;
                kit = nkit;
                kb = nkb;
                hv = nhv;
                ++it;
            }
            if (aborted) {  // let the loads still in flight land before exiting
                for (int64_t k = issued > kStages ? issued - kStages : 0; k < issued; ++k)
                    mbar_wait_ns(smem_u32(&ctl->full[k % kStages]), (uint32_t)((k / kStages) & 1),
                                 100000000ull);
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
            // ring entry k (false on abort)
            auto take = [&](int k, int64_t *e) -> bool {
                if (!ring_wait(k)) return false;
                *e = *reinterpret_cast<volatile int64_t *>(&ctl->ring[k % kRing]);
                return true;
            };
            // The tile list flags tiles without a shared K block; the
            // producer flags the last stage of every other tile.
            int64_t cur = -1;
            aborted = !take(0, &cur);
            while (cur >= 0 && !aborted) {
                ring_release(it);  // done with entry `it`
                int64_t nxt = -1;
                if (!take(it + 1, &nxt)) {  // published before tile `it` was loaded
                    aborted = true;
                    break;
                }
                const bool has_k = (cur & kTileNoK) == 0;
                const int acc = it & 1;
                const uint32_t acc_phase = (it >> 1) & 1;
                if (!mbar_wait(smem_u32(&ctl->tmem_empty[acc]), acc_phase ^ 1, abort, kWaitNs)) {
                    aborted = true;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + acc * kAccCols;
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
                    const uint32_t sa = smem_u32(smem + stage * kStageBytes);
                    const uint32_t sb = sa + kABytes;
                    // K = 32 per MMA: four for a whole K block, two for a half
                    const bool half_st = (lastw & 2u) != 0;
                    const uint64_t layout = half_st ? kDescHalf : kDescFull;
                    const int nmma = half_st ? kOccK / 32 : kTcK / 32;
#pragma unroll
                    for (int k = 0; k < kTcK / 32; ++k)
                        if (k < nmma)
                            mma_f8(d, smem_desc(layout, sa + 32 * k), smem_desc(layout, sb + 32 * k),
                                   (!first || k > 0 || lastw == 4u) ? 1u : 0u);
                    first = false;
                    n_kblocks += nmma / 2;
                    mma_commit(smem_u32(&ctl->empty[stage]));
                    if (++stage == kStages) { stage = 0; phase_bit ^= 1; }
                }
                if (!aborted) mma_commit(smem_u32(&ctl->tmem_full[acc]));
                cur = nxt;
                ++it;
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
    } else {
        // ------------------------------------------------------ epilogue --
        const int q = warp & 3;             // TMEM lane quarter
        const int half = (warp - 2) >> 2;   // which 128 columns of the tile
        const int et = threadIdx.x - 64;
        TileInfo ti;
        // The next tile's records, loaded into registers while this tile
        // waits for its accumulator and is tested (the records do not
        // change during a launch): the entry they belong to, or -1.
        int64_t pre_entry = -1;
        int4 pre_col = make_int4(0, 0, 0, 0), pre_row = make_int4(0, 0, 0, 0);
        static_assert(kEpiThreads == kTcN, "one staged column per epilogue thread");
        for (int it = 0;; ++it) {
            const int slot = it % kRing;
            if (!epi_bar_and(ring_wait(it))) {
                *abort = 1;
                break;
            }
            const int64_t entry = *reinterpret_cast<volatile int64_t *>(&ctl->ring[slot]);
            if (entry < 0) break;
            tile_info(st, phase, entry, &ti);
            InstState &s = st[ti.b];
            const int acc = it & 1;
            const uint32_t acc_phase = (it >> 1) & 1;
            const int32_t R = ti.R;
            const int32_t j0 = ti.bj * kTcN;
            const int32_t i = ti.bi * kTcM + 32 * q + lane;
            // DP stages f and f - s per hyperedge, SE stages f and s
            const bool se = phase == 0 && s.edge_rule != 0;
            // stage the column data of this tile
            bool vals_small = true;  // every staged value fits FP16 exactly, with room for a sum
            epi_bar();  // every epilogue thread has read the entry
            if (et == 0) ring_release(it);
            const bool have = pre_entry == entry;
            {  // column j0 + et
                const int4 rec = have ? pre_col : epi_record(s, phase, j0 + et, R);
                const float a = (float)rec.x, bb = (float)rec.y;
                ctl->colAB[et] = make_float2(a, bb);
                ctl->colO[et] = rec.z;
                ctl->colA16[et] = __float2half_rn(a);
                ctl->colB16[et] = __float2half_rn(bb);
                vals_small = fabsf(a) <= 1024.f && fabsf(bb) <= 1024.f;
            }
            // DP: f_i, f_i - s_i ; SE: f_i, s_i ; MD: d_i ; and the input index of row i
            const int4 rrec = have ? pre_row : epi_record(s, phase, i, R);
            const float ri_f = (float)rrec.x, ri_a = (float)rrec.y;
            const int32_t ri_o = rrec.z;
            vals_small = vals_small && fabsf(ri_f) <= 1024.f && fabsf(ri_a) <= 1024.f;
            const bool tile_small = epi_bar_and(vals_small);  // also publishes the staged columns
            // Load the next tile's records if its entry is published (it
            // usually is: the producer publishes one entry ahead).
            pre_entry = -1;
            {
                const int nk = it + 1;
                const uint32_t nbar = smem_u32(&ctl->ring_full[nk % kRing]);
                const uint32_t npar = (nk / kRing) & 1;
                if (mbar_try(nbar, npar)) {
                    const int64_t ne = *reinterpret_cast<volatile int64_t *>(&ctl->ring[nk % kRing]);
                    if (ne >= 0) {
                        TileInfo nt;
                        tile_info(st, phase, ne, &nt);
                        const InstState &ns = st[nt.b];
                        pre_col = epi_record(ns, phase, nt.bj * kTcN + et, nt.R);
                        pre_row = epi_record(ns, phase, nt.bi * kTcM + 32 * q + lane, nt.R);
                        pre_entry = ne;
                    }
                }
            }
            const bool ok = epi_bar_and(mbar_wait(smem_u32(&ctl->tmem_full[acc]), acc_phase, abort, kWaitNs));
            if (!ok) { *abort = 1; break; }
            tc_fence_after();
            bool rowflag = false;
            int32_t rowcnt = 0;
            // A tile contracts at least one K block, so its accumulator holds
            // its counts -- except a tile the list flags as having no shared K
            // block (kept only in a DP pass where zero counts matter), which
            // the MMA thread skips, leaving the accumulator stale.
            const bool nonzero = (entry & kTileNoK) == 0;
            // A count of 0 changes nothing unless some hyperedge has f > |e| (DP)
            // or is empty (SE): only from such a hyperedge does x = 0 delete; in
            // MD it only adds dominators of a vertex in no hyperedge, deleted anyway.
            const bool zero_matters = phase == 0 && s.has_loose;
            {
                const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + acc * kAccCols;
#pragma unroll 1
                for (int ch = half * (kTcN / 64); ch < (half + 1) * (kTcN / 64); ++ch) {
                    float v[32];
                    if (nonzero) {
                        tmem_ld32(taddr + ch * 32, v);
                    } else {
#pragma unroll
                        for (int c = 0; c < 32; ++c) v[c] = 0.f;
                    }
                    float vmax = 0.f;  // counts are >= 0
#pragma unroll
                    for (int c = 0; c < 32; ++c) vmax = fmaxf(vmax, v[c]);
                    // skip 32 x 32 blocks of zero counts
                    if (!zero_matters && !__any_sync(0xffffffffu, vmax > 0.f)) continue;
                    uint32_t colmask = 0;
                    const float2 *cab = ctl->colAB + ch * 32;
                    // Fast path for a chunk whose pairs are all valid (i < j < R for
                    // every row of the warp and every column): without a mutual
                    // pair (both D_ij and D_ji) the tie-breaks reduce to D_ij for
                    // column j and D_ji for row i.
                    const int32_t jc0 = j0 + ch * 32;
                    const int32_t wi0 = ti.bi * kTcM + 32 * q;  // first row of this warp
                    bool slow = !(wi0 + 31 < R && jc0 + 31 < R && jc0 > wi0 + 31);
                    // Paired form of the fast path: two counts per FP16x2 instruction.
                    // Counts and staged values up to 1024 and their sums (<= 2048)
                    // are integers FP16 holds exactly, so every test is exact.
                    bool paired = !slow && tile_small && __all_sync(0xffffffffu, vmax <= 1024.f);
                    if (paired) {
                        const __half2 *ca2 = reinterpret_cast<const __half2 *>(ctl->colA16 + ch * 32);
                        const __half2 *cb2 = reinterpret_cast<const __half2 *>(ctl->colB16 + ch * 32);
                        const __half2 rf2 = __float2half2_rn(ri_f), ra2 = __float2half2_rn(ri_a);
                        // bit k: column 2k, bit 16 + k: column 2k + 1
                        uint32_t cm = 0, rm = 0, mm = 0;
#pragma unroll
                        for (int k = 0; k < 16; ++k) {
                            const __half2 x2 = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
                            const __half2 a2 = ca2[k], b2 = cb2[k];
                            const uint32_t sel = (1u << k) | (1u << (16 + k));
                            uint32_t mij, mji;
                            if (phase == 0 && !se) {
                                mij = __hge2_mask(__hadd2(x2, ra2), a2);  // x + f_i - s_i >= f_j
                                mji = __hge2_mask(__hadd2(x2, b2), rf2);  // x + f_j - s_j >= f_i
                            } else if (phase == 0) {
                                mij = __heq2_mask(x2, ra2) & __hge2_mask(rf2, a2);  // x = s_i, f_i >= f_j
                                mji = __heq2_mask(x2, b2) & __hge2_mask(a2, rf2);   // x = s_j, f_j >= f_i
                            } else {
                                mij = __heq2_mask(x2, a2);   // x = d_j
                                mji = __heq2_mask(x2, rf2);  // x = d_i
                            }
                            cm |= mij & sel;
                            rm |= mji & sel;
                            mm |= mij & mji;
                        }
                        if (!__any_sync(0xffffffffu, mm != 0)) {
                            // back to bit c = column c (interleave the two halves)
                            auto spread = [](uint32_t x) {
                                x = (x | (x << 8)) & 0x00FF00FFu;
                                x = (x | (x << 4)) & 0x0F0F0F0Fu;
                                x = (x | (x << 2)) & 0x33333333u;
                                return (x | (x << 1)) & 0x55555555u;
                            };
                            colmask = spread(cm & 0xFFFFu) | (spread(cm >> 16) << 1);
                            if (phase == 0) rowflag |= rm != 0;
                            else rowcnt += __popc(rm);
                        } else {
                            slow = true;  // a mutual pair: the tie-breaks decide
                        }
                    }
                    if (!slow && !paired) {
                        uint32_t cm = 0;
                        bool rf = false, mut = false;
                        int32_t rc = 0;
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            const float x = v[c];
                            const float2 ab = cab[c];
                            if (phase == 0) {
                                // DP: f_i - (s_i - x) >= f_j ; SE: x = s_i and f_i >= f_j
                                const bool dij = se ? (x == ri_a && ri_f >= ab.x)
                                                    : x + ri_a >= ab.x;
                                const bool dji = se ? (x == ab.y && ab.x >= ri_f)
                                                    : x + ab.y >= ri_f;
                                cm |= (uint32_t)dij << c;
                                rf |= dji;
                                mut |= dij && dji;
                            } else {
                                const bool eqj = x == ab.x;  // x = d_j
                                const bool eqi = x == ri_f;  // x = d_i
                                cm |= (uint32_t)eqj << c;
                                rc += (int32_t)eqi;
                                mut |= eqj && eqi;
                            }
                        }
                        slow = __any_sync(0xffffffffu, mut);
                        if (!slow) {
                            colmask = cm;
                            rowflag |= rf;
                            rowcnt += rc;
                        }
                    }
                    if (slow) {  // diagonal / ragged chunks, or a mutual pair present
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            const int cc = ch * 32 + c;
                            const int32_t j = j0 + cc;
                            const bool valid = (i < j) && (j < R);
                            const float x = v[c];
                            const float2 ab = cab[c];
                            const bool i_first = ri_o < ctl->colO[cc];  // input-index tie-break
                            if (phase == 0) {
                                // Algorithm 1: D_ij = [f_i - (s_i - x) >= f_j] (rule SE:
                                // [x = s_i and f_i >= f_j]); e_j goes iff D_ij and
                                // (not D_ji or i before j)
                                const bool dij = se ? (x == ri_a && ri_f >= ab.x)
                                                    : x + ri_a >= ab.x;
                                const bool dji = se ? (x == ab.y && ab.x >= ri_f)
                                                    : x + ab.y >= ri_f;
                                colmask |= (uint32_t)(valid && dij && (!dji || i_first)) << c;
                                rowflag |= valid && dji && (!dij || !i_first);
                            } else {
                                // Algorithm 2: D_ij = [x = d_j and (x != d_i or i before j)]
                                const bool eqj = x == ab.x;
                                const bool eqi = x == ri_f;
                                colmask |= (uint32_t)(valid && eqj && (!eqi || i_first)) << c;
                                rowcnt += (int32_t)(valid && eqi && (!eqj || !i_first));
                            }
                        }
                    }
                    const uint32_t any = __reduce_or_sync(0xffffffffu, colmask);
                    if (any) {
                        if (phase == 0) {
                            if ((any >> lane) & 1u) s.e_del[j0 + ch * 32 + lane] = 1;
                        } else {
                            uint32_t m = any;
                            while (m) {
                                const int c = __ffs(m) - 1;
                                m &= m - 1;
                                const int n1 = __popc(__ballot_sync(0xffffffffu, (colmask >> c) & 1u));
                                if (lane == 0) atomicAdd(&ctl->ccnt[ch * 32 + c], n1);
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&ctl->tmem_empty[acc]));
            if (phase == 0) {
                if (rowflag) s.e_del[i] = 1;
            } else {
                if (rowcnt) atomicAdd(&s.v_cnt[i], rowcnt);
                epi_bar();
                for (int c = et; c < kTcN; c += kEpiThreads) {
                    const int32_t cnt = ctl->ccnt[c];
                    if (cnt) { atomicAdd(&s.v_cnt[j0 + c], cnt); ctl->ccnt[c] = 0; }
                }
            }
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

constexpr size_t kSmemBytes = 1024 + kStages * kStageBytes + sizeof(SharedCtl);

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
    static cudaError_t once = cudaFuncSetAttribute(
        k_tc_contract, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    return once;
}

cudaError_t launch_tc_contract(InstState *st, Plan *plan, BatchCounters *ctr, int phase, int sms,
                               int32_t *kerr, cudaStream_t s) {
    k_tc_contract<<<sms, kThreads, kSmemBytes, s>>>(st, plan, ctr, phase, kerr);
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

cudaError_t launch_tc_tile_list(InstState *st, Plan *plan, int phase, int sms, cudaStream_t s) {
    k_tile_list<<<sms * 4, 256, 0, s>>>(st, plan, phase);
    return cudaGetLastError();
}

}  // namespace mhs

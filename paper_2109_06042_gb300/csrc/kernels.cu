// kernels.cu -- encode, compaction, planning and the bit-packed popcount
// contraction with the fused DP / MD epilogue.
//
// Round structure (Algorithm 3, Section 4.1), all on the device:
//   plan(phase 0) -> encode A -> contract(DP or SE) -> compact_edges
//   plan(phase 1) -> clear A + encode A^T -> contract(MD) -> clear A^T -> compact_vertices
//   [rule FE at a fixpoint, fe.cu]
// The contraction of either kind (this file: popcount; contract_tc.cu:
// tcgen05 FP8) computes the pair counts of Eq. (1) / Eq. (2) tile by tile
// and never writes them out: the epilogue turns each count into the
// deletion flags of Algorithm 1 or the dominator counts of Algorithm 2.
#include <algorithm>

#include <cuda_runtime.h>

#include "bounded_wait.cuh"
#include "kernels.h"
#include "mhs_internal.h"

namespace mhs {

namespace {

constexpr uint8_t kFp8One = 0x38;  // 1.0 in E4M3


// Exclusive block scan of one value per thread (blockDim.x a multiple of
// 32, at most 1024).  *total receives the block total.
template <typename T>
__device__ T block_exclusive_scan(T x, T *total, T *sh /*[33]*/) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    T inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nwarps ? sh[lane] : T(0);
        T winc = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, winc, o);
            if (lane >= o) winc += y;
        }
        if (lane < nwarps) sh[lane] = winc - w;
        if (lane == 31) sh[32] = winc;
    }
    __syncthreads();
    T r = inc - x + sh[warp];
    *total = sh[32];
    __syncthreads();
    return r;
}

// Locate the instance owning global item `g` in a prefix array off[0..count].
template <typename T>
__device__ __forceinline__ int find_owner(const T *off, int count, T g) {
    int lo = 0, hi = count;  // off[lo] <= g < off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- setup --

// Structural checks of device-resident inputs (blockIdx.y = instance):
// edge_ptr starts at 0, is non-decreasing and ends at nnz; vertex ids lie in
// [0, n); demands are >= 1.
__global__ void k_validate(InstState *st, int count) {
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (tid == 0) {
        if (s.eptr[0] != 0 || (int64_t)s.eptr[s.m0] != s.nnz0) atomicOr(&s.status, kErrBadPtr);
    }
    for (int64_t e = tid; e < s.m0; e += stride) {
        if (s.eptr[e + 1] < s.eptr[e]) atomicOr(&s.status, kErrBadPtr);
        if (s.f[e] < 1) atomicOr(&s.status, kErrBadDemand);
    }
    for (int64_t p = tid; p < s.nnz0; p += stride) {
        int32_t v = s.evtx[p];
        if (v < 0 || v >= s.n0) atomicOr(&s.status, kErrBadVertex);
    }
}

// OR of the instances' status words, so that a batch load reads back one
// word instead of every instance's state.
__global__ void k_status_or(const InstState *st, int count, int32_t *out) {
    int32_t x = 0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < count; b += gridDim.x * blockDim.x)
        x |= st[b].status;
    x = __reduce_or_sync(0xffffffffu, x);
    if ((threadIdx.x & 31) == 0 && x) atomicOr(out, x);
}

// Batch inputs from device arrays: convert the global int64 CSR offsets of
// instance b (hyperedges [e0[b], e0[b] + m0)) to its local int32 offsets.
__global__ void k_localize_ptr(InstState *st, int count, const int64_t *gptr, const int64_t *e0) {
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    int32_t *eptr = const_cast<int32_t *>(s.eptr);
    const int64_t base = gptr[e0[b]];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= s.m0;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = gptr[e0[b] + i] - base;
        eptr[i] = (x >= 0 && x <= s.nnz0) ? (int32_t)x : -1;
    }
}

// Gather gptr[e0[b]] for b in [0, count] (instance boundaries of a batch).
__global__ void k_gather_bounds(const int64_t *gptr, const int64_t *e0, int64_t *out, int count) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= count; b += gridDim.x * blockDim.x)
        out[b] = gptr[e0[b]];
}

// Chained-scan compaction of a single instance (see k_compact_edges): status
// word epochs (30 bits) and the time limit of a wait on a predecessor chunk.
constexpr uint32_t kEpochMask = (1u << 30) - 1;
constexpr uint64_t kChainWaitNs = 2000000000ull;  // 2 s

// Zero the occupancy bits of phase p's operand for its first R rows (all
// row blocks a tile over R rows can touch).  Block-cooperative.
__device__ __forceinline__ void zero_occupancy(InstState &s, int p, int32_t R, int64_t first,
                                               int64_t stride) {
    if (!s.occ[p]) return;
    const int64_t words = (int64_t)((R + 255) / 256) * 2 * s.occ_words[p];
    for (int64_t w = first; w < words; w += stride) s.occ[p][w] = 0;
}

// Round state and vertex id maps (one block per instance).  In input
// layout the hyperedge maps are the identity too; in sorted layout they are
// filled by the k_layout_* kernels below, whose buckets (v_cnt) and cursors
// (v_deg) are zeroed here.
// (blockIdx.y = instance; the blocks of an instance split its ranges)
__global__ void k_init(InstState *st, int count, int32_t max_rounds) {
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    const int32_t t0 = blockIdx.x * blockDim.x + threadIdx.x, ts = gridDim.x * blockDim.x;
    for (int32_t v = t0; v < s.n0; v += ts) { s.v_o2c[v] = v; s.v_c2o[v] = v; }
    if (s.layout_sorted == 2)  // degrees for the vertex layout (v_maxf is free until MD)
        for (int32_t v = t0; v < s.n0; v += ts) s.v_maxf[v] = 0;
    if (s.layout_sorted) {
        for (int32_t v = t0; v <= s.n0; v += ts) { s.v_cnt[v] = 0; s.v_deg[v] = 0; }
    } else {
        for (int32_t e = t0; e < s.m0; e += ts) { s.e_o2c[e] = e; s.e_c2o[e] = e; }
    }
    if (s.forced)
        for (int32_t v = t0; v < s.n0; v += ts) s.forced[v] = 0;
    if (s.v_dirty)
        for (int32_t v = t0; v < s.n0; v += ts) s.v_dirty[v] = 0;
    if (s.v_dirty_rb)
        for (int32_t w = t0; w < s.At_rows / 128; w += ts) s.v_dirty_rb[w] = 0;
    if (s.e_dirty_rb)
        for (int32_t w = t0; w < s.A_rows / 128; w += ts) s.e_dirty_rb[w] = 0;
    zero_occupancy(s, 0, s.m0, t0, ts);
    if (s.scan_status)
        for (int32_t c = t0; c < s.scan_chunks; c += ts) s.scan_status[c] = 0;
    if (t0 == 0) {
        s.n = s.n0; s.m = s.m0; s.m_dp = s.m0; s.n_next = s.n0;
        s.rounds = 0; s.active = s.status == 0; s.max_rounds = max_rounds; s.changed = 0;
        s.dp_deleted = 0; s.md_deleted = 0; s.has_loose = 0;
        s.fe_stage = 0; s.fe_passes = 0; s.md_full = 1; s.skip_a = 0; s.skip_at = 0;
    }
}

// Degree layout, step 1 (blockIdx.y = instance): vertex degrees into v_maxf.
__global__ void k_vertex_degrees(InstState *st, int count) {
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    if (s.layout_sorted != 2 || s.status) return;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < s.nnz0;
         p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&s.v_maxf[s.evtx[p]], 1);
}

// Degree layout, step 2 (one block of 1024 threads per instance): vertices
// grouped by degree class floor(log4(deg)) in ascending order, input order
// inside a class (a stable counting sort).  With skewed degrees, sorting
// hyperedges by their smallest position then places each hyperedge by its
// rarest vertex: the rows of a row block share rare vertices, and their
// popular vertices fall in the few K blocks at the end, so far fewer
// (row block, K block) pairs are occupied.  Near-uniform degrees keep the
// input order (one or two classes), and with it any locality.
constexpr int kDegClasses = 16;
__device__ __forceinline__ int deg_class(int32_t d) {
    return d <= 1 ? 0 : min((31 - __clz(d)) / 2, kDegClasses - 1);
}
__global__ void __launch_bounds__(1024) k_vertex_layout(InstState *st, int count) {
    __shared__ int32_t start[kDegClasses];
    __shared__ int32_t wcnt[32][kDegClasses];  // this chunk: per warp, per class
    const int b = blockIdx.x;
    if (b >= count) return;
    InstState &s = st[b];
    if (s.layout_sorted != 2 || s.status) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < kDegClasses) start[threadIdx.x] = 0;
    __syncthreads();
    for (int32_t v = threadIdx.x; v < s.n0; v += blockDim.x) atomicAdd(&start[deg_class(s.v_maxf[v])], 1);
    __syncthreads();
    if (threadIdx.x == 0) {  // exclusive prefix over the classes
        int32_t acc = 0;
        for (int c = 0; c < kDegClasses; ++c) { const int32_t x = start[c]; start[c] = acc; acc += x; }
    }
    __syncthreads();
    for (int32_t base = 0; base < s.n0; base += blockDim.x) {
        const int32_t v = base + threadIdx.x;
        const int c = v < s.n0 ? deg_class(s.v_maxf[v]) : -1;
        const uint32_t peers = __match_any_sync(0xffffffffu, c);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (lane < kDegClasses) wcnt[warp][lane] = 0;
        __syncwarp();
        if (c >= 0 && rank == 0) wcnt[warp][c] = __popc(peers);
        __syncthreads();
        if (threadIdx.x < kDegClasses) {  // per class: prefix over the warps, then advance
            int32_t acc = start[threadIdx.x];
            for (int w = 0; w < 32; ++w) { const int32_t x = wcnt[w][threadIdx.x]; wcnt[w][threadIdx.x] = acc; acc += x; }
            start[threadIdx.x] = acc;
        }
        __syncthreads();
        if (c >= 0) {
            const int32_t pos = wcnt[warp][c] + rank;
            s.v_c2o[pos] = v;
            s.v_o2c[v] = pos;
        }
        __syncthreads();
    }
}

// Sorted layouts, step 1 (blockIdx.y = instance): key of each hyperedge =
// its smallest vertex id (layout 1) or position (layout 2), n0 if empty,
// kept in e_s; bucket counts in v_cnt.
__global__ void k_layout_keys(InstState *st, int count) {
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    if (!s.layout_sorted || s.status) return;
    const bool by_pos = s.layout_sorted == 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.m0;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t key = s.n0;
        for (int32_t p = s.eptr[e]; p < s.eptr[e + 1]; ++p)
            key = min(key, by_pos ? s.v_o2c[s.evtx[p]] : s.evtx[p]);
        s.e_s[e] = key;
        atomicAdd(&s.v_cnt[key], 1);
    }
}

// Sorted layout, step 2 (one block per instance): bucket starts in v_deg,
// an exclusive scan of the n0 + 1 bucket counts, 8 consecutive buckets per
// thread.
__global__ void k_layout_scan(InstState *st, int count) {
    __shared__ int32_t sh[33];
    constexpr int kPer = 8;
    const int b = blockIdx.x;
    if (b >= count) return;
    InstState &s = st[b];
    if (!s.layout_sorted || s.status) return;
    const int32_t nb = s.n0 + 1;
    int32_t carry = 0;
    for (int32_t base = 0; base < nb; base += blockDim.x * kPer) {
        const int32_t i0 = base + threadIdx.x * kPer;
        int32_t x[kPer], sum = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            x[k] = i0 + k < nb ? s.v_cnt[i0 + k] : 0;
            sum += x[k];
        }
        int32_t tot;
        int32_t ex = carry + block_exclusive_scan<int32_t>(sum, &tot, sh);
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            if (i0 + k < nb) s.v_deg[i0 + k] = ex;
            ex += x[k];
        }
        carry += tot;
    }
}

// Sorted layout, step 3: place every hyperedge at the next slot of its
// bucket, in arbitrary order (steps 4 and 5 sort each bucket by input id,
// so that every load of an instance gets the same layout: sharded passes
// split the tile rows of replicas that must agree on it).
__global__ void k_layout_place(InstState *st, int count) {
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    if (!s.layout_sorted || s.status) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.m0;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t pos = atomicAdd(&s.v_deg[s.e_s[e]], 1);
        s.e_c2o[pos] = (int32_t)e;
        s.e_o2c[e] = pos;
    }
}

// Sorted layout, step 4: each hyperedge's final position is its bucket's
// start plus the number of hyperedges of the bucket with a smaller input id
// (after step 3, v_deg[key] is the bucket's end and v_cnt[key] its size).
// The cost is the sum of the squared bucket sizes; buckets hold the
// hyperedges sharing their smallest vertex (id or position).
__global__ void k_layout_rank(InstState *st, int count) {
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    if (!s.layout_sorted || s.status) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.m0;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t key = s.e_s[e];
        const int32_t hi = s.v_deg[key], lo = hi - s.v_cnt[key];
        int32_t rank = 0;
        for (int32_t p = lo; p < hi; ++p) rank += s.e_c2o[p] < (int32_t)e;
        s.e_o2c[e] = lo + rank;
    }
}

// Sorted layout, step 5: the position -> id map from the final positions.
__global__ void k_layout_commit(InstState *st, int count) {
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    if (!s.layout_sorted || s.status) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.m0;
         e += (int64_t)gridDim.x * blockDim.x)
        s.e_c2o[s.e_o2c[e]] = (int32_t)e;
}

// Hyperedge rows of round 1, by position.
__global__ void k_edge_rows(InstState *st, int count) {
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    if (s.status) return;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s.m0;
         r += (int64_t)gridDim.x * blockDim.x) {
        s.e_f[r] = s.f[s.e_c2o[r]];
        s.e_s[r] = -1;  // never tested: every hyperedge is a DP candidate
        s.e_del[r] = 0;
    }
}

// ------------------------------------------------------------- planning --

// phase 0: rows = current hyperedges (DP); phase 1: rows = current vertices (MD).
// tc: 0 popcount tiles, 1 tcgen05 tiles (128 x plan->tile_n).
__global__ void k_plan(InstState *st, Plan *plan, int phase, int tc, BatchCounters *ctr) {
    __shared__ int32_t sh[33];
    __shared__ int64_t sh64[33];
    const int count = plan->count;
    int32_t rcarry = 0;
    int64_t tcarry = 0;
    int32_t act_any = 0;
    for (int base = 0; base < count; base += blockDim.x) {
        int b = base + threadIdx.x;
        int32_t rows = 0;
        int64_t tiles = 0;
        if (b < count) {
            const InstState &s = st[b];
            if (s.scan_status) {  // this phase's compaction: tickets from 0, a new epoch
                st[b].scan_ticket = 0;
                st[b].scan_epoch = (s.scan_epoch + 1) & kEpochMask;
            }
            if (s.active && s.status == 0) {
                // Incremental rounds (tcgen05 path): a pass without candidates
                // deletes nothing, so its operand is not needed.  DP: no
                // hyperedge lost a vertex since the previous DP pass, i.e. the
                // previous MD pass deleted none (FE sets md_full).  MD: this
                // round's DP pass deleted no hyperedge.
                int32_t skip = 0;
                if (tc && !s.no_skip && !s.md_full) {
                    if (phase == 0) skip = s.e_dirty_rb && s.md_deleted == 0;
                    else skip = s.v_dirty && s.dp_deleted == 0;
                }
                if (phase == 0) st[b].skip_a = skip;
                else st[b].skip_at = skip;
                // hyperedges to scatter: phase 0 the current ones; phase 1 the
                // rows DP saw (the fused pass clears A at those rows and sets
                // A^T for the ones DP kept)
                // (tcgen05 path: rounded up to a multiple of 32, so a warp's
                // group of 32 rows lies in one instance and starts at a
                // 32-aligned position: k_set_a_tc, k_set_md_tc, k_clear_at_tc)
                const bool none = phase == 0 ? skip : skip && s.skip_a;
                rows = !tc ? s.m : none ? 0 : (s.m + 31) & ~31;
                const int32_t R = phase == 0 ? s.m : s.n;
                tiles = tc ? tc_tiles(R, plan->tile_n) : pop_tiles(R);
                act_any = 1;
            }
        }
        int32_t rtot;
        int32_t rex = block_exclusive_scan<int32_t>(rows, &rtot, sh);
        if (b < count) plan->row_off[b] = rcarry + rex;
        rcarry += rtot;
        int64_t ttot;
        int64_t tex = block_exclusive_scan<int64_t>(tiles, &ttot, sh64);
        if (b < count) plan->tile_off[b] = tcarry + tex;
        tcarry += ttot;
    }
    act_any = __syncthreads_or(act_any);
    if (threadIdx.x == 0) {
        plan->row_off[count] = rcarry;
        plan->tile_off[count] = tcarry;
        plan->total_rows = rcarry;
        plan->list_count = 0;
        plan->list_next = 0;
        plan->list_light = 0;
        plan->list_next_light = 0;
        plan->total_tiles = tcarry;
        plan->any_active = act_any;
        if (phase == 0 && ctr) {
            ctr->active = 0; ctr->n_alive = 0; ctr->m_alive = 0; ctr->dp_deleted = 0;
            ctr->md_deleted = 0; ctr->max_rounds_seen = 0; ctr->changed_any = 0;
            ctr->status_any = 0; ctr->n_done = 0;
        }
    }
}

// --------------------------------------------------------------- encode --

// Bit-packed operands (popcount path).  One hyperedge row per lane, a warp
// walking the original vertex lists of its 32 hyperedges together.  Phase 0
// (rows = current hyperedges) sets A[e'][v'] (K = current vertices) and
// counts |e| (= I^E_ii).  Phase 1 walks the rows the DP pass saw (e_prev):
// its set pass clears their entries of A (the DP pass's clear, fused in since
// it walks the same incidences), marks the vertices of the hyperedges DP
// deleted as MD candidates, and for the kept ones sets At[v'][e''] (rows =
// current vertices, K = the hyperedges' positions after DP) and counts deg(v)
// (= I^V_jj) and the maximum demand; its clear pass clears At after the MD
// contraction.  So the operands are all-zero between rounds, and A^T between
// phases.  A set counts only incidences that were not already set, so a
// repeated id inside one hyperedge counts once.
template <int kPhase, bool kSet>
__global__ void __launch_bounds__(256) k_scatter(InstState *st, const Plan *plan) {
    // Each warp takes 32 consecutive rows and walks the incidences of all of
    // them together, 32 at a time, so a hyperedge of 64 vertices does not
    // hold its warp 64 dependent atomics long.
    __shared__ int32_t wfresh[8][32];  // fresh incidences per row of each warp
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int32_t total = plan->total_rows;
    const int32_t nw = gridDim.x * (blockDim.x >> 5);
    for (int32_t g0 = (blockIdx.x * (blockDim.x >> 5) + wib) * 32; g0 < total; g0 += nw * 32) {
        const int32_t g = g0 + lane;
        int b = 0;
        int32_t ce = 0, e = 0, p0 = 0, len = 0;
        bool mark = false;
        int32_t cnew = 0;  // phase 1: the row's position after DP, -1 if DP deleted it
        if (g < total) {
            b = find_owner(plan->row_off, plan->count, g);
            const InstState &s = st[b];
            ce = g - plan->row_off[b];
            e = kPhase == 0 ? s.e_c2o[ce] : s.e_prev[ce];
            if (kPhase == 1) cnew = s.e_o2c[e];
            p0 = s.eptr[e];
            len = s.eptr[e + 1] - p0;
            // phase 1 set: a hyperedge the DP pass deleted makes its
            // vertices MD candidates of this round
            mark = kPhase == 1 && kSet && s.v_dirty && cnew < 0;
            // phase 1 clear: A^T holds only the rows DP kept
            if (kPhase == 1 && !kSet && cnew < 0) len = 0;
        }
        int32_t incl = len;  // inclusive prefix of the row lengths over the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int32_t start = incl - len;
        const int32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        if (kSet && kPhase == 0) wfresh[wib][lane] = 0;
        __syncwarp();
        for (int32_t f0 = 0; f0 < tot; f0 += 32) {
            const int32_t f = f0 + lane;
            // owner row: the last lane whose run starts at or before f
            int r = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int c = r + step;
                const int32_t sc = __shfl_sync(0xffffffffu, start, c & 31);
                if (c < 32 && sc <= f) r = c;
            }
            const int rb = __shfl_sync(0xffffffffu, b, r);
            const int32_t rce = __shfl_sync(0xffffffffu, ce, r);
            const int32_t rnew = __shfl_sync(0xffffffffu, cnew, r);
            const int32_t re = __shfl_sync(0xffffffffu, e, r);
            const int32_t rp = __shfl_sync(0xffffffffu, p0, r) + f - __shfl_sync(0xffffffffu, start, r);
            const bool rmark = __shfl_sync(0xffffffffu, mark, r);
            if (f >= tot) continue;
            InstState &s = st[rb];
            const int32_t cv = s.v_o2c[s.evtx[rp]];
            if (cv < 0) continue;
            if (rmark && cv < s.n) {
                s.v_dirty[cv] = 1;
                s.v_dirty_rb[cv >> 7] = 1;
            }
            if (kPhase == 1 && kSet) {  // the DP pass's clear of A, fused in
                s.Ab[(int64_t)rce * s.Ab_pitch + (cv >> 5)] = 0;
                if (rnew < 0) continue;  // deleted by DP: nothing in A^T
            }
            const int32_t R = kPhase == 0 ? s.m : s.n;
            const int32_t K = kPhase == 0 ? s.n : s.m_dp;
            const int32_t rr = kPhase == 0 ? rce : cv;
            const int32_t cc = kPhase == 0 ? cv : rnew;
            if (rr >= R || cc >= K) { atomicOr(&s.status, kErrCapacity); continue; }
            bool fresh = false;
            uint32_t *row = (kPhase == 0 ? s.Ab : s.Atb) +
                            (int64_t)rr * (kPhase == 0 ? s.Ab_pitch : s.Atb_pitch);
            if (kSet) {
                const uint32_t bit = 1u << (cc & 31);
                fresh = (atomicOr(&row[cc >> 5], bit) & bit) == 0;
            } else {
                row[cc >> 5] = 0;  // every set bit of this word is cleared by some thread
            }
            if (kSet && fresh) {
                if (kPhase == 0) {
                    atomicAdd(&wfresh[wib][r], 1);
                } else {
                    atomicAdd(&s.v_deg[cv], 1);
                    atomicMax(&s.v_maxf[cv], s.f[re]);
                }
            }
        }
        if (kSet && kPhase == 0) {
            __syncwarp();
            if (g < total) {
                InstState &s = st[b];
                const int32_t fresh_cnt = wfresh[wib][lane];
                // a hyperedge whose size changed since the previous DP pass (or
                // never tested) makes its row block a DP candidate
                if (s.e_dirty_rb && s.e_s[ce] != fresh_cnt) s.e_dirty_rb[ce >> 7] = 1;
                s.e_s[ce] = fresh_cnt;  // one lane owns the row
                if (s.e_rec) {  // the tcgen05 epilogue stages this one record per row
                    const int32_t fe = s.e_f[ce];
                    s.e_rec[ce] = make_int4(fe, s.edge_rule ? fresh_cnt : fe - fresh_cnt, e, 0);
                }
            }
            __syncwarp();  // wfresh is reused by the next group of rows
        }
    }
}

// ------------------------------------------ dense operands (tcgen05) --
//
// The FP8 operands hold one byte per incidence, and DRAM and L2 move them in
// 32-byte sectors.  A byte store or a byte atomic into a sector L2 does not
// hold makes L2 read the sector from DRAM first; a store that covers the
// whole sector does not.  So the set and clear passes of the dense operands
// write whole sectors, and each sector has one writer:
//  * A (rows = hyperedges): a sector lies in one row; the warp that owns the
//    row builds the sector's byte mask in a shared-memory table from the
//    row's incidences and writes the sector once.
//  * A^T (rows = vertices, K = hyperedge positions after DP): the warp that
//    owns positions [32w, 32w + 32) owns sector w of every vertex row, so it
//    builds those sectors from its hyperedges' incidences.
//  * A clear writes the zero sector: every nonzero byte in it belongs to the
//    row being cleared (A) or to the same all-clearing pass (A^T).
// Warps take groups of 32 rows; the plan rounds every instance's rows up to
// a multiple of 32, so a group lies in one instance at a 32-aligned
// position.  A group whose incidences exceed its table sets its bytes with
// atomics instead, for all of its sectors, so no sector is written both
// ways.  The table also deduplicates: a vertex listed twice in a hyperedge
// sets one bit, so sizes and degrees count it once.

constexpr int kSecWarps = 4;          // warps per block
constexpr int kSecTab = 512;          // table entries per warp (a power of two)
constexpr int kSecTabLog = 9;

// One entry per sector: key << 32 | byte mask (bit b: byte b is 1.0).
struct SecTable {
    unsigned long long e[kSecTab];
};
constexpr unsigned long long kSecFree = ~0ull;

// Sets `bit` in the entry of `key`, inserting the key if absent: one shared
// atomic in the common cases (the key present: an OR; its slot free: a
// compare-and-swap).  False if the table is full (callers insert at most
// kSecTab keys, so it never is).
__device__ __forceinline__ bool sec_set(SecTable &t, uint32_t key, uint32_t bit) {
    uint32_t h = (key * 2654435761u) >> (32 - kSecTabLog);
    const unsigned long long mine = (unsigned long long)key << 32;
    for (int p = 0; p < kSecTab; ++p) {
        const unsigned long long cur = *reinterpret_cast<volatile unsigned long long *>(&t.e[h]);
        if (cur != kSecFree && (cur >> 32) == key) {
            atomicOr(&t.e[h], (unsigned long long)bit);
            return true;
        }
        if (cur == kSecFree) {
            const unsigned long long old = atomicCAS(&t.e[h], kSecFree, mine | bit);
            if (old == kSecFree) return true;
            if ((old >> 32) == key) {
                atomicOr(&t.e[h], (unsigned long long)bit);
                return true;
            }
        }
        h = (h + 1) & (kSecTab - 1);
    }
    return false;
}

// Four mask bits -> four bytes of 0 or 1.0 (bit i -> byte i).
__device__ __forceinline__ uint32_t fp8_bytes(uint32_t nib) {
    return ((nib * 0x00204081u) & 0x01010101u) * kFp8One;
}

__device__ __forceinline__ void store_sector(uint8_t *p, uint32_t m) {
    uint4 *q = reinterpret_cast<uint4 *>(p);
    q[0] = make_uint4(fp8_bytes(m & 15u), fp8_bytes((m >> 4) & 15u), fp8_bytes((m >> 8) & 15u),
                      fp8_bytes((m >> 12) & 15u));
    q[1] = make_uint4(fp8_bytes((m >> 16) & 15u), fp8_bytes((m >> 20) & 15u),
                      fp8_bytes((m >> 24) & 15u), fp8_bytes(m >> 28));
}

__device__ __forceinline__ void zero_sector(uint8_t *p) {
    uint4 *q = reinterpret_cast<uint4 *>(p);
    q[0] = make_uint4(0u, 0u, 0u, 0u);
    q[1] = make_uint4(0u, 0u, 0u, 0u);
}

// Occupancy bit of (row block rr / 128, K block cc / kOccK) of phase p's operand.
__device__ __forceinline__ void set_occupancy(InstState &s, int p, int32_t rr, int32_t cc) {
    const int32_t kblk = cc / kOccK;
    uint32_t *ow = s.occ[p] + (int64_t)(rr >> 7) * s.occ_words[p] + (kblk >> 5);
    const uint32_t ob = 1u << (kblk & 31);
    if (!(*reinterpret_cast<volatile uint32_t *>(ow) & ob)) atomicOr(ow, ob);
}

// Byte atomic (groups whose incidences exceed the table); true if the byte was 0.
__device__ __forceinline__ bool set_byte(uint8_t *row, int32_t cc) {
    uint32_t *w = reinterpret_cast<uint32_t *>(row + (cc & ~3));
    const uint32_t sh = 8u * (cc & 3);
    const uint32_t old = atomicOr(w, (uint32_t)kFp8One << sh);
    return ((old >> sh) & 0xffu) == 0;
}

// The incidences of a warp's 32 rows (lane l: row l, its list at p0, len
// entries), flattened: *start = the lane's first flat index, returns the total.
__device__ __forceinline__ int32_t rows_prefix(int lane, int32_t len, int32_t *start) {
    int32_t incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    *start = incl - len;
    return __shfl_sync(0xffffffffu, incl, 31);
}

// Flat index f -> its row (the last lane whose run starts at or before f).
__device__ __forceinline__ int flat_owner(int32_t start, int32_t f) {
    int r = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int c = r + step;
        const int32_t sc = __shfl_sync(0xffffffffu, start, c & 31);
        if (c < 32 && sc <= f) r = c;
    }
    return r;
}

// Walks the incidences of a warp's 32 rows whose vertices are alive (lane l:
// row l, its vertex list at p0, flattened from *start, tot in all), calling
// fn(r, cv, x_r) with the row r, the vertex's current position cv and row
// r's payload x.  The loads of kWalkU chunks of 32 incidences are issued
// before any is used, so a warp has that many dependent pairs in flight.
constexpr int kWalkU = 4;
template <typename F>
__device__ __forceinline__ void walk_live(const InstState &s, int lane, int32_t p0,
                                          int32_t start, int32_t tot, int32_t x, F &&fn) {
    const int32_t *evtx = s.evtx;
    const int32_t *o2c = s.v_o2c;
    for (int32_t f0 = 0; f0 < tot; f0 += 32 * kWalkU) {
        int r[kWalkU];
        int32_t v[kWalkU], xr[kWalkU];
#pragma unroll
        for (int u = 0; u < kWalkU; ++u) {
            const int32_t f = f0 + 32 * u + lane;
            r[u] = flat_owner(start, f);
            const int32_t rp = __shfl_sync(0xffffffffu, p0, r[u]) + f -
                               __shfl_sync(0xffffffffu, start, r[u]);
            xr[u] = __shfl_sync(0xffffffffu, x, r[u]);
            v[u] = f < tot ? __ldg(evtx + rp) : -1;
        }
#pragma unroll
        for (int u = 0; u < kWalkU; ++u) v[u] = v[u] >= 0 ? __ldg(o2c + v[u]) : -1;
#pragma unroll
        for (int u = 0; u < kWalkU; ++u)
            if (v[u] >= 0) fn(r[u], v[u], xr[u]);
    }
}

// Empties the table entries the warp has written: fn(key, mask) writes an
// entry's sector and returns, through *ow / *ob, the occupancy word and bit
// it sets.  The lanes of one pass over 32 slots set each distinct word with
// one atomic.
template <typename F>
__device__ __forceinline__ void drain_table(SecTable &t, int lane, F &&fn) {
    __syncwarp();
    for (int base = 0; base < kSecTab; base += 32) {
        const int i = base + lane;
        const unsigned long long ent = t.e[i];
        uint32_t *ow = nullptr;
        uint32_t ob = 0;
        if (ent != kSecFree) {
            t.e[i] = kSecFree;
            fn((uint32_t)(ent >> 32), (uint32_t)ent, &ow, &ob);
        }
        const unsigned grp = __match_any_sync(0xffffffffu, (unsigned long long)(uintptr_t)ow);
        const uint32_t bits = __reduce_or_sync(grp, ob);
        if (ow && lane == __ffs(grp) - 1) atomicOr(ow, bits);
    }
    __syncwarp();
}

__device__ __forceinline__ void init_table(SecTable &t, int lane) {
    for (int i = lane; i < kSecTab; i += 32) t.e[i] = kSecFree;
    __syncwarp();
}

// Occupancy word and bit of (row block rr / 128, K block cc / kOccK) of
// phase p's operand.
__device__ __forceinline__ uint32_t *occ_word(InstState &s, int p, int32_t rr, int32_t cc,
                                              uint32_t *ob) {
    const int32_t kblk = cc / kOccK;
    *ob = 1u << (kblk & 31);
    return s.occ[p] + (int64_t)(rr >> 7) * s.occ_words[p] + (kblk >> 5);
}

// Phase 0 set: A[e'][v'] = 1.0 for the current hyperedges' live incidences,
// |e| (= I^E_ii), the epilogue's row records and the occupancy bits of A.
__global__ void __launch_bounds__(32 * kSecWarps) k_set_a_tc(InstState *st, const Plan *plan) {
    __shared__ SecTable tab[kSecWarps];
    __shared__ int32_t wfresh[kSecWarps][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    SecTable &t = tab[wib];
    init_table(t, lane);
    const int32_t total = plan->total_rows;
    const int32_t nw = gridDim.x * kSecWarps;
    for (int32_t g0 = (blockIdx.x * kSecWarps + wib) * 32; g0 < total; g0 += nw * 32) {
        const int b = find_owner(plan->row_off, plan->count, g0);
        InstState &s = st[b];
        const int32_t ce0 = g0 - plan->row_off[b];
        const int32_t ce = ce0 + lane;
        const bool row = ce < s.m;
        int32_t e = 0, p0 = 0, len = 0;
        if (row) {
            e = __ldg(s.e_c2o + ce);
            p0 = __ldg(s.eptr + e);
            len = __ldg(s.eptr + e + 1) - p0;
        }
        int32_t start;
        const int32_t tot = rows_prefix(lane, len, &start);
        const bool table = tot <= kSecTab;
        const int32_t K = s.n;
        uint8_t *const A = s.A;
        const int64_t pitch = s.A_pitch;
        wfresh[wib][lane] = 0;
        __syncwarp();
        walk_live(s, lane, p0, start, tot, 0, [&](int r, int32_t cv, int32_t) {
            if (cv >= K) { atomicOr(&s.status, kErrCapacity); return; }
            if (table) {
                if (!sec_set(t, ((uint32_t)r << 26) | (uint32_t)(cv >> 5), 1u << (cv & 31)))
                    atomicOr(&s.status, kErrCapacity);
            } else {
                const int32_t rr = ce0 + r;
                if (set_byte(A + (int64_t)rr * pitch, cv)) atomicAdd(&wfresh[wib][r], 1);
                set_occupancy(s, 0, rr, cv);
            }
        });
        if (table) {
            drain_table(t, lane, [&](uint32_t key, uint32_t m, uint32_t **ow, uint32_t *ob) {
                const int r = (int)(key >> 26);
                const int32_t c0 = (int32_t)(key & 0x3ffffffu) * 32;
                const int32_t rr = ce0 + r;
                store_sector(A + (int64_t)rr * pitch + c0, m);
                atomicAdd(&wfresh[wib][r], __popc(m));
                *ow = occ_word(s, 0, rr, c0, ob);
            });
        } else {
            __syncwarp();
        }
        if (row) {
            const int32_t size = wfresh[wib][lane];
            // a hyperedge whose size changed since the previous DP pass (or
            // never tested) makes its row block a DP candidate
            if (s.e_dirty_rb && s.e_s[ce] != size) s.e_dirty_rb[ce >> 7] = 1;
            s.e_s[ce] = size;
            const int32_t fe = s.e_f[ce];
            if (s.e_rec) s.e_rec[ce] = make_int4(fe, s.edge_rule ? size : fe - size, e, 0);
            // a count of 0 decides a pair only from a hyperedge with f > |e|
            // (DP) or an empty one (SE)
            if (s.edge_rule ? size == 0 : fe > size) s.has_loose = 1;
        }
        __syncwarp();  // wfresh is reused by the next group
    }
}

// Phase 1 set, two walks per group of 32 positions [c0, c0 + 32):
//  (a) the rows the DP pass saw there (e_prev): zero their sectors of A (the
//      DP pass's clear), and mark the vertices of the hyperedges DP deleted
//      as MD candidates;
//  (b) the hyperedges DP kept there (e_c2o after DP): sector c0 / 32 of
//      A^T's vertex rows, deg(v) (= I^V_jj), the maximum demand over E(v),
//      and the occupancy bits of A^T.
__global__ void __launch_bounds__(32 * kSecWarps) k_set_md_tc(InstState *st, const Plan *plan) {
    __shared__ SecTable tab[kSecWarps];
    __shared__ int32_t wdem[kSecWarps][32];  // demands of the group's hyperedges
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    SecTable &t = tab[wib];
    init_table(t, lane);
    const int32_t total = plan->total_rows;
    const int32_t nw = gridDim.x * kSecWarps;
    for (int32_t g0 = (blockIdx.x * kSecWarps + wib) * 32; g0 < total; g0 += nw * 32) {
        const int b = find_owner(plan->row_off, plan->count, g0);
        InstState &s = st[b];
        const int32_t c0 = g0 - plan->row_off[b];
        const int32_t n = s.n;
        if (!s.skip_a) {  // (a)
            const int32_t ce = c0 + lane;
            int32_t p0 = 0, len = 0, mark = 0;
            if (ce < s.m) {
                const int32_t e = __ldg(s.e_prev + ce);
                p0 = __ldg(s.eptr + e);
                len = __ldg(s.eptr + e + 1) - p0;
                mark = s.v_dirty && __ldg(s.e_o2c + e) < 0;
            }
            int32_t start;
            const int32_t tot = rows_prefix(lane, len, &start);
            uint8_t *const A = s.A;
            const int64_t pitch = s.A_pitch;
            uint8_t *const vd = s.v_dirty;
            uint8_t *const vdrb = s.v_dirty_rb;
            walk_live(s, lane, p0, start, tot, mark, [&](int r, int32_t cv, int32_t rmark) {
                if (rmark && cv < n) {
                    vd[cv] = 1;
                    vdrb[cv >> 7] = 1;
                }
                zero_sector(A + (int64_t)(c0 + r) * pitch + (cv & ~31));
            });
        }
        if (!s.skip_at) {  // (b)
            const int32_t cn = c0 + lane;
            int32_t p0 = 0, len = 0, fe = 0;
            if (cn < s.m_dp) {
                const int32_t e = __ldg(s.e_c2o + cn);
                p0 = __ldg(s.eptr + e);
                len = __ldg(s.eptr + e + 1) - p0;
                fe = __ldg(s.f + e);
            }
            int32_t start;
            const int32_t tot = rows_prefix(lane, len, &start);
            const bool table = tot <= kSecTab;
            wdem[wib][lane] = fe;
            __syncwarp();
            uint8_t *const At = s.At;
            const int64_t pitch = s.At_pitch;
            int32_t *const deg = s.v_deg;
            int32_t *const maxf = s.v_maxf;
            walk_live(s, lane, p0, start, tot, fe, [&](int r, int32_t cv, int32_t rfe) {
                if (cv >= n) { atomicOr(&s.status, kErrCapacity); return; }
                if (table) {
                    if (!sec_set(t, (uint32_t)cv, 1u << r)) atomicOr(&s.status, kErrCapacity);
                } else {
                    if (set_byte(At + (int64_t)cv * pitch, c0 + r)) {
                        atomicAdd(&deg[cv], 1);
                        atomicMax(&maxf[cv], rfe);
                    }
                    set_occupancy(s, 1, cv, c0);
                }
            });
            if (table) {
                drain_table(t, lane, [&](uint32_t cv, uint32_t m, uint32_t **ow, uint32_t *ob) {
                    int32_t mf = 0;  // the largest demand among the sector's hyperedges
                    for (uint32_t bits = m; bits; bits &= bits - 1)
                        mf = max(mf, wdem[wib][__ffs(bits) - 1]);
                    store_sector(At + (int64_t)cv * pitch + c0, m);
                    atomicAdd(&deg[cv], __popc(m));
                    atomicMax(&maxf[cv], mf);
                    *ow = occ_word(s, 1, (int32_t)cv, c0, ob);
                });
            } else {
                __syncwarp();
            }
        }
    }
}

// Phase 1 clear, after the MD contraction: zero the sectors of A^T that the
// set pass wrote (group [c0, c0 + 32): sector c0 / 32 of its vertices' rows).
__global__ void __launch_bounds__(32 * kSecWarps) k_clear_at_tc(InstState *st,
                                                              const Plan *plan) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int32_t total = plan->total_rows;
    const int32_t nw = gridDim.x * kSecWarps;
    for (int32_t g0 = (blockIdx.x * kSecWarps + wib) * 32; g0 < total; g0 += nw * 32) {
        const int b = find_owner(plan->row_off, plan->count, g0);
        InstState &s = st[b];
        const int32_t c0 = g0 - plan->row_off[b];
        if (s.skip_at) continue;
        const int32_t cn = c0 + lane;
        int32_t p0 = 0, len = 0;
        if (cn < s.m_dp) {
            const int32_t e = __ldg(s.e_c2o + cn);
            p0 = __ldg(s.eptr + e);
            len = __ldg(s.eptr + e + 1) - p0;
        }
        int32_t start;
        const int32_t tot = rows_prefix(lane, len, &start);
        uint8_t *const At = s.At;
        const int64_t pitch = s.At_pitch;
        const int32_t n = s.n;
        walk_live(s, lane, p0, start, tot, 0, [&](int, int32_t cv, int32_t) {
            if (cv < n) zero_sector(At + (int64_t)cv * pitch + c0);
        });
    }
}

// ----------------------------------------------------------- compaction --

// Chained scan across the blocks compacting one instance: the exclusive
// prefix, over chunks 0..c-1 of this launch, of the kept counts, given
// chunk c's own count `agg` (decoupled look-back, one thread per block).
// Chunk c first publishes its count, then walks back over its
// predecessors until one has published its inclusive prefix, and
// publishes its own.  Returns -1 if a predecessor published nothing within
// the time limit.  Every predecessor belongs to a block that took its
// ticket earlier, so it is running.
__device__ int32_t chain_exclusive(unsigned long long *status, uint32_t epoch, int32_t c,
                                   int32_t agg) {
    const unsigned long long tag = (unsigned long long)epoch << 34;
    if (c == 0) {
        atomicExch(&status[0], tag | (2ull << 32) | (uint32_t)agg);
        return 0;
    }
    atomicExch(&status[c], tag | (1ull << 32) | (uint32_t)agg);
    int32_t excl = 0;
    uint64_t t0 = 0;
    for (int32_t p = c - 1; p >= 0;) {
        const unsigned long long w = *reinterpret_cast<volatile unsigned long long *>(&status[p]);
        const uint32_t flag = (uint32_t)(w >> 32) & 3u;
        if ((uint32_t)(w >> 34) != epoch || flag == 0) {  // not published in this launch yet
            const uint64_t t = globaltimer();
            if (t0 == 0) t0 = t;
            else if (t - t0 > kChainWaitNs) return -1;
            continue;
        }
        excl += (int32_t)(uint32_t)w;
        if (flag == 2) break;
        --p;
    }
    atomicExch(&status[c], tag | (2ull << 32) | (uint32_t)(excl + agg));
    return excl;
}

// Order-preserving compaction of the hyperedges that DP kept (Algorithm 1's
// returned rows), and the zeroed vertex rows of this round's MD pass.  With
// one block per instance (blockIdx.y), chunked so the in-place update of
// e_c2o never overwrites an entry not yet read.  With several blocks (a
// single instance), block t of the ticket order takes chunk t of 1024 rows:
// it writes only after every earlier chunk has published its count, which
// each does after reading its rows, and never beyond its own chunk.
__global__ void k_compact_edges(InstState *st, int count) {
    __shared__ int32_t sh[33];
    __shared__ int32_t sh_x[2];
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    const bool chained = gridDim.x > 1;
    int32_t c = 0;  // this block's chunk (chained)
    if (chained) {
        if (threadIdx.x == 0) sh_x[0] = (int32_t)atomicAdd(&s.scan_ticket, 1u);
        __syncthreads();
        c = sh_x[0];
    }
    if (!s.active || s.status) return;
    const int32_t m = s.m;
    int32_t kept = 0;  // rows kept before this block's chunk (chained: of chunk c)
    bool last_chunk = false;
    for (int32_t base = chained ? c * 1024 : 0; base < m; base += blockDim.x) {
        int32_t r = base + threadIdx.x;
        int32_t keep = 0, orig = -1, size = 0;
        if (r < m) {
            keep = s.e_del[r] == 0;
            orig = s.e_c2o[r];
            size = s.e_s[r];
            s.e_prev[r] = orig;  // row r of A as this DP pass saw it
        }
        int32_t tot;
        int32_t ex = block_exclusive_scan<int32_t>(keep, &tot, sh);  // syncs after reads
        if (chained) {
            if (threadIdx.x == 0)
                sh_x[1] = chain_exclusive(s.scan_status, s.scan_epoch, c, tot);
            __syncthreads();
            kept = sh_x[1];
            if (kept < 0) {
                if (threadIdx.x == 0) atomicOr(&s.status, kErrTimeout);
                return;
            }
        }
        if (r < m) {
            s.e_o2c[orig] = keep ? kept + ex : -1;
            if (keep) {
                s.e_c2o[kept + ex] = orig;
                s.e_s[kept + ex] = size;  // the size this DP pass saw moves with the row
            }
        }
        kept += tot;
        if (chained) {
            last_chunk = base + 1024 >= m;
            break;
        }
        __syncthreads();
    }
    if (m == 0 && c == 0) last_chunk = true;
    if (threadIdx.x == 0 && (chained ? last_chunk : true)) {
        s.m_dp = kept;
        s.dp_deleted = m - kept;
        if (s.rounds < kTraceRounds) {
            s.trace[s.rounds][0] = m;
            s.trace[s.rounds][1] = s.n;
            s.trace[s.rounds][2] = kept;
        }
    }
    // vertex rows of this round's MD pass (s.n is not changed here)
    const int32_t first = chained ? c * 1024 + (int32_t)threadIdx.x : (int32_t)threadIdx.x;
    const int32_t stride = chained ? (int32_t)gridDim.x * 1024 : (int32_t)blockDim.x;
    const int32_t nv = s.n;
    zero_occupancy(s, 1, nv, first, stride);
    for (int32_t r = first; r < nv; r += stride) {
        s.v_deg[r] = 0;
        s.v_maxf[r] = 0;
        s.v_cnt[r] = 0;
        s.v_del[r] = 0;
    }
}

// MD decision (Algorithm 2: delete v_j iff C_j >= max f over E(v_j)),
// order-preserving compaction of the vertices, and round bookkeeping.  One
// block per instance, or (a single instance) one block per chunk of 1024
// vertices as in k_compact_edges; then the block of the last chunk keeps
// the books, and each block clears the next round's rows in its own range.
__global__ void k_compact_vertices(InstState *st, int count, BatchCounters *ctr,
                                   int32_t *done_list) {
    __shared__ int32_t sh[33];
    __shared__ int32_t sh_x[2];
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    const bool chained = gridDim.x > 1;
    int32_t c = 0;
    if (chained) {
        if (threadIdx.x == 0) sh_x[0] = (int32_t)atomicAdd(&s.scan_ticket, 1u);
        __syncthreads();
        c = sh_x[0];
    }
    // The state is read before any block can finish the books: the block
    // of chunk 0 reads it before publishing, and the last chunk waits for
    // that.  A block without a chunk does only the clears of its range.
    const bool run = s.active && s.status == 0;
    const int32_t n = s.n, m_dp = s.m_dp;
    bool books = !chained;  // this block keeps the books
    if (run) {
        int32_t kept = 0;
        // (chained: chunk 0 runs even when n = 0, so that some block keeps the books)
        for (int32_t base = chained ? c * 1024 : 0; base < n || (chained && base == 0);
             base += blockDim.x) {
            int32_t r = base + threadIdx.x;
            int32_t keep = 0, orig = -1;
            if (r < n) {
                // a vertex that lost no hyperedge since it last survived MD
                // survives again: its dominator count can only have dropped
                const bool cand = s.md_full || !s.v_dirty || s.v_dirty[r];
                keep = !cand || s.v_cnt[r] < s.v_maxf[r];
                orig = s.v_c2o[r];
                s.v_del[r] = !keep;
            }
            int32_t tot;
            int32_t ex = block_exclusive_scan<int32_t>(keep, &tot, sh);
            if (chained) {
                if (threadIdx.x == 0)
                    sh_x[1] = chain_exclusive(s.scan_status, s.scan_epoch, c, tot);
                __syncthreads();
                kept = sh_x[1];
                if (kept < 0) {
                    if (threadIdx.x == 0) atomicOr(&s.status, kErrTimeout);
                    return;
                }
            }
            if (r < n) {
                s.v_o2c[orig] = keep ? kept + ex : -1;
                if (keep) s.v_c2o[kept + ex] = orig;
            }
            kept += tot;
            if (chained) {
                books = base + 1024 >= n;
                break;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0 && books) {
            s.n_next = kept;
            s.md_deleted = n - kept;
            s.changed = (s.dp_deleted + s.md_deleted) > 0;
            s.m = m_dp;
            s.n = kept;
            s.rounds += 1;
            s.md_full = 0;
            if (!s.changed && s.full_edges && s.max_rounds == 0) {
                // fixpoint: rule FE decides (fe.cu) whether it goes on; no
                // vertex was deleted, so v_del is already all zero
                s.fe_stage = 1;
            } else if (!s.changed || (s.max_rounds > 0 && s.rounds >= s.max_rounds)) {
                s.active = 0;
                if (done_list && ctr) done_list[atomicAdd(&ctr->n_done, 1)] = b;
            }
        }
        // the next round's rows: MD candidates start empty; hyperedge rows
        // of the DP pass (e_s keeps the sizes).  One block skips them once
        // the instance has finished; several blocks cannot know that and
        // clear them anyway, which is harmless.
        bool next_rows = true;
        int32_t nv = n;  // vertex rows to clear
        if (!chained) {
            __syncthreads();  // the books are kept
            next_rows = s.active != 0;
            nv = s.n;
        }
        if (next_rows) {  // (32 bits suffice: blocks x 1024 < max(n0, m0) + 1024)
            const int32_t first = chained ? c * 1024 + (int32_t)threadIdx.x : (int32_t)threadIdx.x;
            const int32_t stride = chained ? (int32_t)gridDim.x * 1024 : (int32_t)blockDim.x;
            if (s.v_dirty) {
                for (int32_t r = first; r < nv; r += stride) s.v_dirty[r] = 0;
                for (int32_t w = first; w < (nv + 127) / 128; w += stride) s.v_dirty_rb[w] = 0;
            }
            for (int32_t r = first; r < m_dp; r += stride) {
                s.e_f[r] = s.f[s.e_c2o[r]];
                s.e_del[r] = 0;
            }
            if (s.e_dirty_rb)
                for (int32_t w = first; w < (m_dp + 127) / 128; w += stride) s.e_dirty_rb[w] = 0;
            zero_occupancy(s, 0, m_dp, first, stride);
            if (first == 0) s.has_loose = 0;
        }
    } else {
        books = !chained || c == 0;  // nothing changes: one block reports it
    }
    if (threadIdx.x == 0 && ctr && books) {  // read by a later kernel
        atomicAdd(&ctr->active, s.active);
        atomicAdd(&ctr->n_alive, s.n);
        atomicAdd(&ctr->m_alive, s.m);
        atomicAdd(&ctr->dp_deleted, s.dp_deleted);
        atomicAdd(&ctr->md_deleted, s.md_deleted);
        atomicMax(&ctr->max_rounds_seen, s.rounds);
        atomicOr(&ctr->changed_any, s.changed);
        atomicOr(&ctr->status_any, s.status);
    }
}

// ------------------------------------------------ popcount contraction --

// Map a tile index of the upper triangle of an nt x nt tile grid (ti <= tj,
// row-major) to (ti, tj).
__device__ __forceinline__ void tri_tile(int64_t t, int32_t nt, int32_t *ti, int32_t *tj) {
    // off(i) = i*nt - i*(i-1)/2 ; find the largest i with off(i) <= t
    double a = 2.0 * nt + 1.0;
    double disc = a * a - 8.0 * (double)t;
    int32_t i = (int32_t)((a - sqrt(disc > 0 ? disc : 0)) * 0.5);
    if (i < 0) i = 0;
    if (i > nt - 1) i = nt - 1;
    auto off = [nt](int64_t x) { return x * nt - x * (x - 1) / 2; };
    while (i > 0 && off(i) > t) --i;
    while (i + 1 < nt && off(i + 1) <= t) ++i;
    *ti = i;
    *tj = i + (int32_t)(t - off(i));
}

constexpr int kPopKW = 32;  // K words staged per step

// phase 0: DP on Ab (rows = hyperedges); phase 1: MD on Atb (rows = vertices).
// With nshards > 1 only the tiles whose rows lie in a 128-row block b with
// b % nshards == shard are contracted (one share of a sharded pass).
__global__ void __launch_bounds__(256) k_pop_contract(InstState *st, const Plan *plan, int phase,
                                                      int shard, int nshards) {
    __shared__ uint32_t As[kPopTile][kPopKW + 1];
    __shared__ uint32_t Bs[kPopTile][kPopKW + 1];
    __shared__ int32_t rcnt[kPopTile], ccnt[kPopTile];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t total = plan->total_tiles;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const int b = find_owner(plan->tile_off, plan->count, t);
        InstState &s = st[b];
        const int64_t local = t - plan->tile_off[b];
        const int32_t R = phase == 0 ? s.m : s.n;
        const int32_t W = phase == 0 ? (s.n + 31) / 32 : (s.m_dp + 31) / 32;
        const uint32_t *X = phase == 0 ? s.Ab : s.Atb;
        const int64_t pitch = phase == 0 ? s.Ab_pitch : s.Atb_pitch;
        const int32_t nt = (R + kPopTile - 1) / kPopTile;
        int32_t ti, tj;
        tri_tile(local, nt, &ti, &tj);
        const int32_t i0 = ti * kPopTile, j0 = tj * kPopTile;
        if (nshards > 1 && (i0 / kTcM) % nshards != shard) continue;  // another share's tile
        {  // incremental rounds: only tiles that hold a candidate row or column
            const uint8_t *drb = phase == 0 ? s.e_dirty_rb : s.v_dirty_rb;
            if (drb && !(phase == 1 && s.md_full) && !drb[i0 >> 7] && !drb[j0 >> 7]) continue;
        }
        int32_t acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] = 0;
        for (int32_t k0 = 0; k0 < W; k0 += kPopKW) {
            for (int idx = threadIdx.x; idx < kPopTile * kPopKW; idx += blockDim.x) {
                int row = idx / kPopKW, w = idx % kPopKW;
                int32_t kw = k0 + w;
                uint32_t va = 0, vb = 0;
                if (kw < W) {
                    if (i0 + row < R) va = X[(int64_t)(i0 + row) * pitch + kw];
                    if (j0 + row < R) vb = X[(int64_t)(j0 + row) * pitch + kw];
                }
                As[row][w] = va;
                Bs[row][w] = vb;
            }
            __syncthreads();
#pragma unroll 8
            for (int w = 0; w < kPopKW; ++w) {
                uint32_t av[4], bv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) av[a] = As[ty + 16 * a][w];
#pragma unroll
                for (int c = 0; c < 4; ++c) bv[c] = Bs[tx + 16 * c][w];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][c] += __popc(av[a] & bv[c]);
            }
            __syncthreads();
        }
        // ---- fused epilogue: pairs i < j < R ----
        if (phase == 0) {
            // Algorithm 1: D_ij = [f_i - (s_i - x) >= f_j]; delete j iff
            // D_ij and (not D_ji or i < j), i < j comparing input indices.
            // Rule SE instead: D_ij = [x = s_i and f_i >= f_j] (e_i within e_j).
            const bool se = s.edge_rule != 0;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int32_t i = i0 + ty + 16 * a;
                if (i >= R) continue;
                const int32_t fi = s.e_f[i], si = s.e_s[i], oi = s.e_c2o[i];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int32_t j = j0 + tx + 16 * c;
                    if (j <= i || j >= R) continue;
                    const int32_t x = acc[a][c];
                    const int32_t fj = s.e_f[j], sj = s.e_s[j];
                    const bool dij = se ? (x == si && fi >= fj) : fi - (si - x) >= fj;
                    const bool dji = se ? (x == sj && fj >= fi) : fj - (sj - x) >= fi;
                    const bool i_first = oi < s.e_c2o[j];  // tie-break by input index
                    if (dij && (!dji || i_first)) s.e_del[j] = 1;   // same-value stores
                    if (dji && (!dij || !i_first)) s.e_del[i] = 1;
                }
            }
        } else {
            // Algorithm 2: D_ij = [x = d_j and (x != d_i or i < j)], i < j
            // comparing input indices.
            if (threadIdx.x < kPopTile) { rcnt[threadIdx.x] = 0; ccnt[threadIdx.x] = 0; }
            __syncthreads();
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int32_t i = i0 + ty + 16 * a;
                if (i >= R) continue;
                const int32_t di = s.v_deg[i], oi = s.v_c2o[i];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int32_t j = j0 + tx + 16 * c;
                    if (j <= i || j >= R) continue;
                    const int32_t x = acc[a][c];
                    const int32_t dj = s.v_deg[j];
                    const bool i_first = oi < s.v_c2o[j];  // tie-break by input index
                    if (x == dj && (x != di || i_first)) atomicAdd(&ccnt[tx + 16 * c], 1);
                    if (x == di && (x != dj || !i_first)) atomicAdd(&rcnt[ty + 16 * a], 1);
                }
            }
            __syncthreads();
            if (threadIdx.x < kPopTile) {
                int32_t v = ccnt[threadIdx.x];
                if (v) atomicAdd(&s.v_cnt[j0 + threadIdx.x], v);
            } else if (threadIdx.x < 2 * kPopTile) {
                int32_t v = rcnt[threadIdx.x - kPopTile];
                if (v) atomicAdd(&s.v_cnt[i0 + threadIdx.x - kPopTile], v);
            }
            __syncthreads();
        }
    }
}

// --------------------------------------------------------------- results --

// Alive masks over the input ids; blockIdx.y = instance.  With `batch`
// set, instance b writes at its offsets v_base / e_base of the
// concatenated masks; otherwise at 0.
__global__ void k_alive_masks(const InstState *st, int count, bool batch, uint8_t *alive_v,
                              uint8_t *alive_e) {
    const int b = blockIdx.y;
    if (b >= count) return;
    const InstState &s = st[b];
    if (batch) {
        alive_v += s.v_base;
        alive_e += s.e_base;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)s.n0 + s.m0;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < s.n0) alive_v[i] = s.v_o2c[i] >= 0;
        else alive_e[i - s.n0] = s.e_o2c[i - s.n0] >= 0;
    }
}

// ---- serving loop (device-resident; see server.cpp) ----

// One block per slot at a time.  The ready flag is read once per slot (by
// thread 0): the host may set it while this kernel runs.
__global__ void k_server_admit(InstState *live, const InstState *staged, volatile int32_t *ready,
                               int count) {
    __shared__ int32_t go;
    constexpr int kWords = (int)(sizeof(InstState) / 4);
    static_assert(sizeof(InstState) % 4 == 0, "state copied in words");
    for (int si = blockIdx.x; si < count; si += gridDim.x) {
        if (threadIdx.x == 0) go = ready[si];
        __syncthreads();
        if (go) {
            const int32_t *src = reinterpret_cast<const int32_t *>(staged + si);
            int32_t *dst = reinterpret_cast<int32_t *>(live + si);
            for (int w = threadIdx.x; w < kWords; w += blockDim.x) dst[w] = src[w];
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                ready[si] = 0;
                __threadfence_system();
            }
        }
        __syncthreads();
    }
}

// One block.  A slot is retired once: a finished instance is inactive (and
// its live slot zeroed here), a failed one is taken while still active.
__global__ void __launch_bounds__(256) k_server_retire(InstState *live, InstState *out,
                                                       const int32_t *done,
                                                       const BatchCounters *ctr,
                                                       volatile int32_t *ring,
                                                       volatile ServerFlags *flags,
                                                       ServerDev *dev, int count) {
    __shared__ int32_t fin[4096];  // max_slots <= 4096
    __shared__ int32_t nfin;
    constexpr int kWords = (int)(sizeof(InstState) / 4);
    if (threadIdx.x == 0) nfin = 0;
    __syncthreads();
    const int nd = min(ctr->n_done, count);
    for (int i = threadIdx.x; i < nd; i += blockDim.x) {
        const int si = done[i];
        if (si >= 0 && si < count) fin[atomicAdd(&nfin, 1) & 4095] = si;
    }
    for (int si = threadIdx.x; si < count; si += blockDim.x)
        if (live[si].active && live[si].status) fin[atomicAdd(&nfin, 1) & 4095] = si;
    __syncthreads();
    const int nf = min(nfin, count);  // each slot at most once
    for (int i = 0; i < nf; ++i) {
        const int si = fin[i];
        int32_t *src = reinterpret_cast<int32_t *>(live + si);
        int32_t *dst = reinterpret_cast<int32_t *>(out + si);
        for (int w = threadIdx.x; w < kWords; w += blockDim.x) dst[w] = src[w];
        __syncthreads();
        for (int w = threadIdx.x; w < kWords; w += blockDim.x) src[w] = 0;
        __syncthreads();
    }
    if (threadIdx.x == 0 && nf > 0) {
        __threadfence_system();  // the states in `out` before the ring entries
        const uint32_t head = dev->head;
        for (int i = 0; i < nf; ++i) ring[(head + (uint32_t)i) % (uint32_t)count] = fin[i];
        __threadfence_system();  // the entries before the head
        dev->head = head + (uint32_t)nf;
        flags->head = head + (uint32_t)nf;
        __threadfence_system();
    }
}

__global__ void k_server_cond(cudaGraphConditionalHandle h, const BatchCounters *ctr,
                              const int32_t *kerr, const Plan *plan, ServerDev *dev,
                              volatile ServerFlags *flags, volatile const int32_t *ready,
                              int count, int32_t cap) {
    __shared__ int32_t pending;
    if (threadIdx.x == 0) pending = 0;
    __syncthreads();
    for (int si = threadIdx.x; si < count; si += blockDim.x)
        if (ready[si]) pending = 1;
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (plan->any_active) dev->rounds += 1;
    const int32_t it = ++dev->iters;
    const int32_t err = *kerr;
    flags->rounds = dev->rounds;
    flags->kerr = err;
    __threadfence_system();
    const bool go = !flags->stop && err == 0 && it < cap && (ctr->active > 0 || pending);
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_loop_cond(cudaGraphConditionalHandle h, BatchCounters *ctr, int32_t *kerr,
                            int32_t round_cap) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int32_t it = ++ctr->loop_iters;
    bool go = ctr->active > 0 && *kerr == 0 && ctr->status_any == 0;
    if (go && it >= round_cap) {
        atomicOr(kerr, kErrRoundCap);
        go = false;
    }
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

}  // namespace

// ------------------------------------------------------- host launchers --

cudaError_t launch_loop_cond(cudaGraphConditionalHandle h, BatchCounters *ctr, int32_t *kerr,
                             int32_t round_cap, cudaStream_t s) {
    k_loop_cond<<<1, 32, 0, s>>>(h, ctr, kerr, round_cap);
    return cudaGetLastError();
}

cudaError_t launch_server_admit(InstState *live, const InstState *staged, int32_t *ready,
                                int count, cudaStream_t s) {
    k_server_admit<<<count < 152 ? count : 152, 128, 0, s>>>(live, staged, ready, count);
    return cudaGetLastError();
}

cudaError_t launch_server_retire(InstState *live, InstState *out, const int32_t *done,
                                 const BatchCounters *ctr, int32_t *ring, ServerFlags *flags,
                                 ServerDev *dev, int count, cudaStream_t s) {
    if (count > 4096) return cudaErrorInvalidValue;  // one block lists the retirements
    k_server_retire<<<1, 256, 0, s>>>(live, out, done, ctr, ring, flags, dev, count);
    return cudaGetLastError();
}

cudaError_t launch_server_cond(cudaGraphConditionalHandle h, const BatchCounters *ctr,
                               const int32_t *kerr, const Plan *plan, ServerDev *dev,
                               ServerFlags *flags, const int32_t *ready, int count, int32_t cap,
                               cudaStream_t s) {
    k_server_cond<<<1, 256, 0, s>>>(h, ctr, kerr, plan, dev, flags, ready, count, cap);
    return cudaGetLastError();
}

static int grid_for(int sms, int per_sm) { return sms * per_sm; }

// Blocks per instance for a grid-stride kernel over `items` per instance:
// enough for the largest instance, but for a batch no more than about 16
// blocks per SM in all (a block that finds no work still costs a launch).
static int per_instance_grid(int64_t items, int count) {
    int64_t g = (items + 255) / 256;
    const int64_t cap = count > 1 ? (152 * 16 + count - 1) / count : 256;
    if (g > cap) g = cap;
    if (g > 256) g = 256;
    return g < 1 ? 1 : (int)g;
}

cudaError_t launch_validate(InstState *st, int count, cudaStream_t s) {
    k_validate<<<dim3(count > 1 ? per_instance_grid(1 << 20, count) : 256, count), 256, 0, s>>>(
        st, count);
    return cudaGetLastError();
}

cudaError_t launch_status_or(const InstState *st, int count, int32_t *out, cudaStream_t s) {
    k_status_or<<<(count + 255) / 256 < 64 ? (count + 255) / 256 : 64, 256, 0, s>>>(st, count, out);
    return cudaGetLastError();
}

cudaError_t launch_localize_ptr(InstState *st, int count, const int64_t *gptr, const int64_t *e0,
                                cudaStream_t s) {
    k_localize_ptr<<<dim3(16, count), 256, 0, s>>>(st, count, gptr, e0);
    return cudaGetLastError();
}

cudaError_t launch_gather_bounds(const int64_t *gptr, const int64_t *e0, int64_t *out, int count,
                                 cudaStream_t s) {
    k_gather_bounds<<<(count + 256) / 256, 256, 0, s>>>(gptr, e0, out, count);
    return cudaGetLastError();
}

cudaError_t launch_build(InstState *st, int count, int32_t max_rounds, int64_t max_nnz,
                         int64_t max_m, int64_t max_n, cudaStream_t s) {
    const int gx = per_instance_grid(max_m, count);
    const int gz = per_instance_grid(max_nnz, count);
    // a single instance splits its initial ranges over blocks
    const int gi = count > 1 ? 1 : (int)std::min<int64_t>((std::max(max_m, max_n) + 4095) / 4096, 152);
    k_init<<<dim3(gi > 0 ? gi : 1, count), 1024, 0, s>>>(st, count, max_rounds);
    k_vertex_degrees<<<dim3(gz, count), 256, 0, s>>>(st, count);
    k_vertex_layout<<<count, 1024, 0, s>>>(st, count);
    k_layout_keys<<<dim3(gx, count), 256, 0, s>>>(st, count);
    k_layout_scan<<<count, 1024, 0, s>>>(st, count);
    k_layout_place<<<dim3(gx, count), 256, 0, s>>>(st, count);
    k_layout_rank<<<dim3(gx, count), 256, 0, s>>>(st, count);
    k_layout_commit<<<dim3(gx, count), 256, 0, s>>>(st, count);
    k_edge_rows<<<dim3(gx, count), 256, 0, s>>>(st, count);
    return cudaGetLastError();
}

// Set (or, phase 1, clear) pass of the operands: dense FP8 (tcgen05 path,
// sector writes) or bit-packed (popcount path).
template <int kPhase>
static void launch_scatter(InstState *st, const Plan *plan, bool set, bool dense, int sms,
                           cudaStream_t s) {
    if (dense) {  // blocks of 4 warps (17 KB of tables each): per SM 8 for the A set
                  // pass (its row-local sector writes lose with more), 12 for the MD
                  // set pass, 16 for the clear (measured)
        if (kPhase == 0) k_set_a_tc<<<grid_for(sms, 8), 32 * kSecWarps, 0, s>>>(st, plan);
        else if (set) k_set_md_tc<<<grid_for(sms, 12), 32 * kSecWarps, 0, s>>>(st, plan);
        else k_clear_at_tc<<<grid_for(sms, 16), 32 * kSecWarps, 0, s>>>(st, plan);
        return;
    }
    const int grid = grid_for(sms, 8);
    if (set) k_scatter<kPhase, true><<<grid, 256, 0, s>>>(st, plan);
    else k_scatter<kPhase, false><<<grid, 256, 0, s>>>(st, plan);
}

cudaError_t launch_phase_prologue(InstState *st, Plan *plan, BatchCounters *ctr, int phase,
                                  int contraction, int sms, cudaStream_t s) {
    const bool tc = contraction == kFp8;
    k_plan<<<1, 1024, 0, s>>>(st, plan, phase, tc ? 1 : 0, ctr);
    if (phase == 0) launch_scatter<0>(st, plan, true, tc, sms, s);
    else launch_scatter<1>(st, plan, true, tc, sms, s);
    return cudaGetLastError();
}

cudaError_t launch_phase_contract(InstState *st, Plan *plan, BatchCounters *ctr, int phase,
                                  int contraction, int sms, int32_t *kerr, cudaStream_t s,
                                  int tile_n, int shard, int nshards) {
    const bool tc = contraction == kFp8;
    if (tc) {
        // each share builds its own list and hands it out from its start
        cudaError_t e = cudaMemsetAsync(&plan->list_count, 0, sizeof(int32_t), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(&plan->list_next, 0, sizeof(int32_t), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(&plan->list_light, 0, 2 * sizeof(int32_t), s);
        if (e == cudaSuccess) e = launch_tc_tile_list(st, plan, phase, sms, s, shard, nshards);
        if (e != cudaSuccess) return e;
        return launch_tc_contract(st, plan, ctr, phase, sms, tile_n, kerr, s);
    }
    k_pop_contract<<<grid_for(sms, 6), 256, 0, s>>>(st, plan, phase, shard, nshards);
    return cudaGetLastError();
}

cudaError_t launch_phase_epilogue(InstState *st, Plan *plan, BatchCounters *ctr, int count,
                                  int phase, int contraction, int sms, cudaStream_t s,
                                  int32_t *done_list, int compact_blocks) {
    const bool tc = contraction == kFp8;
    // (the DP pass's clear of A runs inside the MD set pass, which walks the
    // same incidences)
    if (phase == 1) launch_scatter<1>(st, plan, false, tc, sms, s);
    // compact_blocks > 1: a single instance, one block per chunk of 1024 ids
    const dim3 cgrid(compact_blocks > 1 ? compact_blocks : 1, count);
    if (phase == 0) k_compact_edges<<<cgrid, 1024, 0, s>>>(st, count);
    else k_compact_vertices<<<cgrid, 1024, 0, s>>>(st, count, ctr, done_list);
    return cudaGetLastError();
}

// A sharded pass's partial output over INPUT ids (the replicas' layouts may
// order rows differently): phase 0 the DP/SE deletion flag of every
// hyperedge (0 if not alive), phase 1 the dominator count of every vertex.
// export: out[id] = value at the id's current position; import: the value at
// each alive id's position = in[id].
__global__ void k_pass_exchange(InstState *st, int phase, int import, void *buf) {
    InstState &s = st[0];
    const int32_t ids = phase == 0 ? s.m0 : s.n0;
    const int32_t rows = phase == 0 ? s.m : s.n;  // this pass's rows
    const int32_t *o2c = phase == 0 ? s.e_o2c : s.v_o2c;
    for (int32_t id = blockIdx.x * blockDim.x + threadIdx.x; id < ids;
         id += gridDim.x * blockDim.x) {
        const int32_t pos = o2c[id];
        const bool alive = pos >= 0 && pos < rows;
        if (phase == 0) {
            uint8_t *b = static_cast<uint8_t *>(buf);
            if (!import) b[id] = alive ? s.e_del[pos] : 0;
            else if (alive) s.e_del[pos] = b[id] ? 1 : 0;
        } else {
            int32_t *b = static_cast<int32_t *>(buf);
            if (!import) b[id] = alive ? s.v_cnt[pos] : 0;
            else if (alive) s.v_cnt[pos] = b[id];
        }
    }
}

cudaError_t launch_pass_exchange(InstState *st, int phase, int import, void *buf, int sms,
                                 cudaStream_t s) {
    k_pass_exchange<<<grid_for(sms, 2), 256, 0, s>>>(st, phase, import, buf);
    return cudaGetLastError();
}

cudaError_t launch_round_phase(InstState *st, Plan *plan, BatchCounters *ctr, int count,
                               int phase, int contraction, int sms, int32_t *kerr,
                               cudaStream_t s, cudaEvent_t ev_contract_begin,
                               cudaEvent_t ev_contract_end, int32_t *done_list,
                               int compact_blocks, int tile_n) {
    const bool tc = contraction == kFp8;
    cudaError_t e0 = launch_phase_prologue(st, plan, ctr, phase, contraction, sms, s);
    if (e0 != cudaSuccess) return e0;
    if (tc) {
        cudaError_t e = launch_tc_tile_list(st, plan, phase, sms, s, 0, 1);
        if (e != cudaSuccess) return e;
    }
    // Timing events: external event nodes when the round is being captured
    // into a graph, plain records when it is launched directly.
    auto record = [s](cudaEvent_t ev) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
            cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
        else
            cudaEventRecord(ev, s);
    };
    if (ev_contract_begin) record(ev_contract_begin);
    if (tc) {
        cudaError_t e = launch_tc_contract(st, plan, ctr, phase, sms, tile_n, kerr, s);
        if (e != cudaSuccess) return e;
    } else {
        k_pop_contract<<<grid_for(sms, 6), 256, 0, s>>>(st, plan, phase, 0, 1);
    }
    if (ev_contract_end) record(ev_contract_end);
    return launch_phase_epilogue(st, plan, ctr, count, phase, contraction, sms, s, done_list,
                                 compact_blocks);
}

cudaError_t launch_alive_masks(const InstState *st, uint8_t *alive_v, uint8_t *alive_e,
                               cudaStream_t s) {
    k_alive_masks<<<dim3(152, 1), 256, 0, s>>>(st, 1, false, alive_v, alive_e);
    return cudaGetLastError();
}

cudaError_t launch_alive_masks_batch(const InstState *st, int count, uint8_t *alive_v,
                                     uint8_t *alive_e, cudaStream_t s) {
    k_alive_masks<<<dim3(4, count), 256, 0, s>>>(st, count, true, alive_v, alive_e);
    return cudaGetLastError();
}

}  // namespace mhs

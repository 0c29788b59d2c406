// kernels.cu -- encode, compaction, planning and the bit-packed popcount
// contraction with the fused DP / MD epilogue.
//
// Round structure (Algorithm 3, Section 4.1), all on the device:
//   plan(phase 0) -> encode_edges -> contract(DP) -> compact_edges
//   plan(phase 1) -> encode_vertices -> contract(MD) -> compact_vertices
// The contraction of either kind (this file: popcount; contract_tc.cu:
// tcgen05 FP8) computes the pair counts of Eq. (1) / Eq. (2) tile by tile
// and never writes them out: the epilogue turns each count into the
// deletion flags of Algorithm 1 or the dominator counts of Algorithm 2.
#include <cuda_runtime.h>

#include "kernels.h"
#include "mhs_internal.h"

namespace mhs {

namespace {

constexpr uint8_t kFp8One = 0x38;  // 1.0 in E4M3

__device__ __forceinline__ int32_t warp_sum(int32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int32_t warp_max(int32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

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

__device__ __forceinline__ int64_t kpad_bytes(int32_t K) {
    int32_t k = K > 0 ? K : 1;
    return (int64_t)((k + kTcK - 1) / kTcK) * kTcK;
}
__device__ __forceinline__ int32_t kpad_words(int32_t K) {
    int32_t w = (K + 31) / 32;
    return ((w > 0 ? w : 1) + 3) & ~3;
}

// ---------------------------------------------------------------- setup --

__global__ void k_validate(InstState *st) {
    InstState &s = *st;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (tid == 0) {
        if (s.eptr[0] != 0 || (int64_t)s.eptr[s.m0] != s.nnz0) atomicOr(&s.status, kErrBadPtr);
    }
    for (int64_t e = tid; e < s.m0; e += stride)
        if (s.eptr[e + 1] < s.eptr[e]) atomicOr(&s.status, kErrBadPtr);
    for (int64_t p = tid; p < s.nnz0; p += stride) {
        int32_t v = s.evtx[p];
        if (v < 0 || v >= s.n0) atomicOr(&s.status, kErrBadVertex);
    }
}

// Zero the list heads and the per-vertex cursors (v_cnt) of every instance.
__global__ void k_csc_zero(InstState *st, int count) {
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    int32_t *vptr = const_cast<int32_t *>(s.vptr);
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= s.n0;
         v += (int64_t)gridDim.x * blockDim.x) {
        vptr[v] = 0;
        if (v < s.n0) s.v_cnt[v] = 0;
    }
}

// Degree count for the vertex -> hyperedge lists (blockIdx.y = instance).
__global__ void k_csc_count(InstState *st, int count, int32_t *vcount_base_unused) {
    (void)vcount_base_unused;
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    if (s.status) return;
    int32_t *vptr = const_cast<int32_t *>(s.vptr);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < s.nnz0;
         p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&vptr[s.evtx[p] + 1], 1);
}

// Exclusive scan of vptr (one block per instance); also initialises the
// round state and the identity id maps.
__global__ void k_csc_scan_init(InstState *st, int count, int32_t max_rounds) {
    __shared__ int32_t sh[33];
    const int b = blockIdx.x;
    if (b >= count) return;
    InstState &s = st[b];
    int32_t *vptr = const_cast<int32_t *>(s.vptr);
    int32_t carry = 0;
    for (int32_t base = 0; base < s.n0 + 1; base += blockDim.x) {
        int32_t i = base + threadIdx.x;
        int32_t x = i < s.n0 + 1 ? vptr[i] : 0;
        int32_t tot;
        int32_t ex = block_exclusive_scan<int32_t>(x, &tot, sh);
        if (i < s.n0 + 1) vptr[i] = carry + ex + x;  // inclusive of the shifted counts
        carry += tot;
    }
    for (int32_t v = threadIdx.x; v < s.n0; v += blockDim.x) { s.v_o2c[v] = v; s.v_c2o[v] = v; }
    for (int32_t e = threadIdx.x; e < s.m0; e += blockDim.x) { s.e_o2c[e] = e; s.e_c2o[e] = e; }
    if (threadIdx.x == 0) {
        s.n = s.n0; s.m = s.m0; s.m_dp = s.m0; s.n_next = s.n0;
        s.rounds = 0; s.active = s.status == 0; s.max_rounds = max_rounds; s.changed = 0;
        s.dp_deleted = 0; s.md_deleted = 0;
    }
}

// Fill the lists.  v_cnt (zeroed by the caller, unused until the first MD
// pass) serves as the per-vertex cursor.
__global__ void k_csc_fill(InstState *st, int count) {
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    if (s.status) return;
    int32_t *vedg = const_cast<int32_t *>(s.vedg);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.m0;
         e += (int64_t)gridDim.x * blockDim.x)
        for (int32_t p = s.eptr[e]; p < s.eptr[e + 1]; ++p) {
            const int32_t v = s.evtx[p];
            vedg[s.vptr[v] + atomicAdd(&s.v_cnt[v], 1)] = (int32_t)e;
        }
}

// ------------------------------------------------------------- planning --

// phase 0: rows = current hyperedges (DP); phase 1: rows = current vertices (MD).
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
            if (s.active && s.status == 0) {
                rows = phase == 0 ? s.m : s.n;
                tiles = tc ? tc_tiles(rows) : pop_tiles(rows);
                act_any = 1;
            }
        }
        int32_t tot;
        int32_t ex = block_exclusive_scan<int32_t>(rows, &tot, sh);
        if (b < count) plan->row_off[b] = rcarry + ex;
        rcarry += tot;
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
        plan->total_tiles = tcarry;
        plan->any_active = act_any;
        if (phase == 0 && ctr) {
            ctr->active = 0; ctr->n_alive = 0; ctr->m_alive = 0; ctr->dp_deleted = 0;
            ctr->md_deleted = 0; ctr->max_rounds_seen = 0; ctr->changed_any = 0;
            ctr->status_any = 0;
        }
    }
}

// --------------------------------------------------------------- encode --

// One warp per row: zero the row of the dense / bit operand over the
// current K range, then set the incidences of the row's alive partners.
// Returns the number of distinct incidences set by this lane.
template <bool kDense>
__device__ __forceinline__ int32_t write_row(uint8_t *drow, uint32_t *brow, int64_t kbytes,
                                             int32_t kwords, const int32_t *part, int32_t np,
                                             const int32_t *o2c, const int32_t *fval,
                                             int32_t *maxf, int32_t limit, int32_t *err) {
    const int lane = threadIdx.x & 31;
    if (kDense) {
        uint4 z = make_uint4(0, 0, 0, 0);
        for (int64_t c = lane; c < kbytes / 16; c += 32) reinterpret_cast<uint4 *>(drow)[c] = z;
    } else {
        for (int32_t c = lane; c < kwords / 4; c += 32)
            reinterpret_cast<uint4 *>(brow)[c] = make_uint4(0, 0, 0, 0);
    }
    __syncwarp();
    int32_t cnt = 0, mx = 0;
    for (int32_t p = lane; p < np; p += 32) {
        int32_t item = part[p];
        int32_t c = o2c[item];
        if (c < 0) continue;
        if (c >= limit) { atomicOr(err, kErrCapacity); continue; }
        if (fval) mx = max(mx, fval[item]);
        if (kDense) {
            uint32_t *w = reinterpret_cast<uint32_t *>(drow + (c & ~3));
            uint32_t sh = 8u * (c & 3);
            uint32_t old = atomicOr(w, (uint32_t)kFp8One << sh);
            cnt += ((old >> sh) & 0xffu) == 0;
        } else {
            uint32_t bit = 1u << (c & 31);
            uint32_t old = atomicOr(&brow[c >> 5], bit);
            cnt += (old & bit) == 0;
        }
    }
    if (maxf) *maxf = mx;
    return cnt;
}

// Phase 0 rows: current hyperedges; partners: vertices (K = current n).
template <bool kDense>
__global__ void k_encode_edges(InstState *st, const Plan *plan) {
    const int lane = threadIdx.x & 31;
    const int32_t gw0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int32_t nw = (gridDim.x * blockDim.x) >> 5;
    const int32_t total = plan->total_rows;
    for (int32_t g = gw0; g < total; g += nw) {
        const int b = find_owner(plan->row_off, plan->count, g);
        InstState &s = st[b];
        const int32_t r = g - plan->row_off[b];
        const int32_t e = s.e_c2o[r];
        const int32_t p0 = s.eptr[e], np = s.eptr[e + 1] - p0;
        int32_t cnt;
        if (kDense) {
            cnt = write_row<true>(s.A + (int64_t)r * s.A_pitch, nullptr, kpad_bytes(s.n), 0,
                                  s.evtx + p0, np, s.v_o2c, nullptr, nullptr, s.n, &s.status);
        } else {
            cnt = write_row<false>(nullptr, s.Ab + (int64_t)r * s.Ab_pitch, 0, kpad_words(s.n),
                                   s.evtx + p0, np, s.v_o2c, nullptr, nullptr, s.n, &s.status);
        }
        cnt = warp_sum(cnt);
        if (lane == 0) { s.e_s[r] = cnt; s.e_f[r] = s.f[e]; s.e_del[r] = 0; }
    }
}

// Phase 1 rows: current vertices; partners: hyperedges alive after DP (K = m_dp).
template <bool kDense>
__global__ void k_encode_vertices(InstState *st, const Plan *plan) {
    const int lane = threadIdx.x & 31;
    const int32_t gw0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int32_t nw = (gridDim.x * blockDim.x) >> 5;
    const int32_t total = plan->total_rows;
    for (int32_t g = gw0; g < total; g += nw) {
        const int b = find_owner(plan->row_off, plan->count, g);
        InstState &s = st[b];
        const int32_t r = g - plan->row_off[b];
        const int32_t v = s.v_c2o[r];
        const int32_t q0 = s.vptr[v], nq = s.vptr[v + 1] - q0;
        int32_t cnt, mx = 0;
        if (kDense) {
            cnt = write_row<true>(s.At + (int64_t)r * s.At_pitch, nullptr, kpad_bytes(s.m_dp), 0,
                                  s.vedg + q0, nq, s.e_o2c, s.f, &mx, s.m_dp, &s.status);
        } else {
            cnt = write_row<false>(nullptr, s.Atb + (int64_t)r * s.Atb_pitch, 0,
                                   kpad_words(s.m_dp), s.vedg + q0, nq, s.e_o2c, s.f, &mx,
                                   s.m_dp, &s.status);
        }
        cnt = warp_sum(cnt);
        mx = warp_max(mx);
        if (lane == 0) { s.v_deg[r] = cnt; s.v_maxf[r] = mx; s.v_cnt[r] = 0; s.v_del[r] = 0; }
    }
}

// ----------------------------------------------------------- compaction --

// Order-preserving compaction of the hyperedges that DP kept (Algorithm 1's
// returned rows).  One block per instance; chunked so the in-place update
// of e_c2o never overwrites an entry not yet read.
__global__ void k_compact_edges(InstState *st, int count) {
    __shared__ int32_t sh[33];
    const int b = blockIdx.x;
    if (b >= count) return;
    InstState &s = st[b];
    if (!s.active || s.status) return;
    const int32_t m = s.m;
    int32_t carry = 0;
    for (int32_t base = 0; base < m; base += blockDim.x) {
        int32_t r = base + threadIdx.x;
        int32_t keep = 0, orig = -1;
        if (r < m) { keep = s.e_del[r] == 0; orig = s.e_c2o[r]; }
        int32_t tot;
        int32_t ex = block_exclusive_scan<int32_t>(keep, &tot, sh);  // syncs after reads
        if (r < m) {
            s.e_o2c[orig] = keep ? carry + ex : -1;
            if (keep) s.e_c2o[carry + ex] = orig;
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) { s.m_dp = carry; s.dp_deleted = m - carry; }
}

// MD decision (Algorithm 2: delete v_j iff C_j >= max f over E(v_j)),
// order-preserving compaction of the vertices, and round bookkeeping.
__global__ void k_compact_vertices(InstState *st, int count, BatchCounters *ctr) {
    __shared__ int32_t sh[33];
    const int b = blockIdx.x;
    if (b >= count) return;
    InstState &s = st[b];
    if (s.active && s.status == 0) {
        const int32_t n = s.n;
        int32_t carry = 0;
        for (int32_t base = 0; base < n; base += blockDim.x) {
            int32_t r = base + threadIdx.x;
            int32_t keep = 0, orig = -1;
            if (r < n) { keep = s.v_cnt[r] < s.v_maxf[r]; orig = s.v_c2o[r]; s.v_del[r] = !keep; }
            int32_t tot;
            int32_t ex = block_exclusive_scan<int32_t>(keep, &tot, sh);
            if (r < n) {
                s.v_o2c[orig] = keep ? carry + ex : -1;
                if (keep) s.v_c2o[carry + ex] = orig;
            }
            carry += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            s.n_next = carry;
            s.md_deleted = n - carry;
            s.changed = (s.dp_deleted + s.md_deleted) > 0;
            s.m = s.m_dp;
            s.n = carry;
            s.rounds += 1;
            if (!s.changed || (s.max_rounds > 0 && s.rounds >= s.max_rounds)) s.active = 0;
        }
    }
    if (threadIdx.x == 0 && ctr) {
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
__global__ void __launch_bounds__(256) k_pop_contract(InstState *st, const Plan *plan, int phase) {
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
            // D_ij and (not D_ji or i < j).  For i < j that is D_ij; e_i is
            // deleted through this pair iff D_ji and not D_ij.
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int32_t i = i0 + ty + 16 * a;
                if (i >= R) continue;
                const int32_t fi = s.e_f[i], si = s.e_s[i];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int32_t j = j0 + tx + 16 * c;
                    if (j <= i || j >= R) continue;
                    const int32_t x = acc[a][c];
                    const int32_t fj = s.e_f[j], sj = s.e_s[j];
                    const bool dij = fi - (si - x) >= fj;
                    const bool dji = fj - (sj - x) >= fi;
                    if (dij) s.e_del[j] = 1;            // same-value stores
                    else if (dji) s.e_del[i] = 1;
                }
            }
        } else {
            // Algorithm 2: D_ij = [x = d_j and (x != d_i or i < j)].  For
            // i < j: D_ij = [x = d_j], D_ji = [x = d_i and x != d_j].
            if (threadIdx.x < kPopTile) { rcnt[threadIdx.x] = 0; ccnt[threadIdx.x] = 0; }
            __syncthreads();
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int32_t i = i0 + ty + 16 * a;
                if (i >= R) continue;
                const int32_t di = s.v_deg[i];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int32_t j = j0 + tx + 16 * c;
                    if (j <= i || j >= R) continue;
                    const int32_t x = acc[a][c];
                    const int32_t dj = s.v_deg[j];
                    if (x == dj) atomicAdd(&ccnt[tx + 16 * c], 1);
                    else if (x == di) atomicAdd(&rcnt[ty + 16 * a], 1);
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

__global__ void k_alive_masks(const InstState *st, uint8_t *alive_v, uint8_t *alive_e) {
    const InstState &s = *st;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)s.n0 + s.m0;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < s.n0) alive_v[i] = s.v_o2c[i] >= 0;
        else alive_e[i - s.n0] = s.e_o2c[i - s.n0] >= 0;
    }
}

}  // namespace

// ------------------------------------------------------- host launchers --

static int grid_for(int sms, int per_sm) { return sms * per_sm; }

cudaError_t launch_validate(InstState *st, cudaStream_t s) {
    k_validate<<<256, 256, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_build(InstState *st, int count, int32_t max_rounds, int64_t max_nnz,
                         int64_t max_m, int64_t max_n, cudaStream_t s) {
    int64_t work = max_nnz > max_m ? max_nnz : max_m;
    if (max_n + 1 > work) work = max_n + 1;
    int gx = (int)((work + 255) / 256);
    if (gx > 1024) gx = 1024;
    if (gx < 1) gx = 1;
    dim3 g1(gx, count);
    k_csc_zero<<<g1, 256, 0, s>>>(st, count);
    k_csc_count<<<g1, 256, 0, s>>>(st, count, nullptr);
    k_csc_scan_init<<<count, 1024, 0, s>>>(st, count, max_rounds);
    k_csc_fill<<<g1, 256, 0, s>>>(st, count);
    return cudaGetLastError();
}

cudaError_t launch_round_phase(InstState *st, Plan *plan, BatchCounters *ctr, int count,
                               int phase, int contraction, int sms, int32_t *kerr,
                               cudaStream_t s, cudaEvent_t ev_contract_begin,
                               cudaEvent_t ev_contract_end) {
    const bool tc = contraction == kFp8;
    k_plan<<<1, 1024, 0, s>>>(st, plan, phase, tc ? 1 : 0, ctr);
    const int enc_grid = grid_for(sms, 8);
    if (phase == 0) {
        if (tc) k_encode_edges<true><<<enc_grid, 256, 0, s>>>(st, plan);
        else k_encode_edges<false><<<enc_grid, 256, 0, s>>>(st, plan);
    } else {
        if (tc) k_encode_vertices<true><<<enc_grid, 256, 0, s>>>(st, plan);
        else k_encode_vertices<false><<<enc_grid, 256, 0, s>>>(st, plan);
    }
    if (ev_contract_begin) cudaEventRecordWithFlags(ev_contract_begin, s, cudaEventRecordExternal);
    if (tc) {
        cudaError_t e = launch_tc_contract(st, plan, phase, sms, kerr, s);
        if (e != cudaSuccess) return e;
    } else {
        k_pop_contract<<<grid_for(sms, 6), 256, 0, s>>>(st, plan, phase);
    }
    if (ev_contract_end) cudaEventRecordWithFlags(ev_contract_end, s, cudaEventRecordExternal);
    if (phase == 0) k_compact_edges<<<count, 1024, 0, s>>>(st, count);
    else k_compact_vertices<<<count, 1024, 0, s>>>(st, count, ctr);
    return cudaGetLastError();
}

cudaError_t launch_alive_masks(const InstState *st, uint8_t *alive_v, uint8_t *alive_e,
                               cudaStream_t s) {
    k_alive_masks<<<152, 256, 0, s>>>(st, alive_v, alive_e);
    return cudaGetLastError();
}

}  // namespace mhs

// fe.cu -- the full-edge rule FE (Section 3.1) between fixpoints of the
// DP/SE + MD rounds, as the KernelGPU-FE variant of Section 5.1 alternates
// them.
//
// FE takes a hyperedge with |e| = f(e): all its vertices go into the
// solution (k drops by one per vertex), the hyperedge goes, and every other
// hyperedge holding one of those vertices loses one unit of demand per such
// vertex, going when its demand reaches 0.  Applied one hyperedge at a time
// until none is full, it reaches the same state as applying it to all full
// hyperedges at once, which is what these kernels do: for every surviving
// hyperedge, f - |e| is unchanged by the rule (both drop by the number of
// its vertices taken), so a hyperedge is full afterwards only if it was full
// before, and the vertices taken are exactly the union S of the full
// hyperedges' vertices.  One application is therefore exhaustive.
//
// Per instance that reached its DP/MD fixpoint in this round (fe_stage = 1):
//   k_fe_mark     full hyperedges -> e_del; their alive vertices -> v_del (S)
//   k_fe_apply    other hyperedges: f -= |e & S|; f <= 0 -> e_del
//   k_fe_compact  order-preserving compaction of both, forced[] += S, k -= |S|;
//                 if anything went the instance runs more rounds, otherwise
//                 it is finished.
#include <cuda_runtime.h>

#include "kernels.h"
#include "mhs_internal.h"

namespace mhs {

namespace {

__global__ void k_fe_mark(InstState *st, int count) {
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    if (!s.fe_stage || s.status) return;
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < s.m; r += gridDim.x * blockDim.x) {
        const int32_t e = s.e_c2o[r];
        int32_t size = 0;
        for (int32_t p = s.eptr[e]; p < s.eptr[e + 1]; ++p) size += s.v_o2c[s.evtx[p]] >= 0;
        if (size != s.f[e]) continue;
        s.e_del[r] = 1;
        for (int32_t p = s.eptr[e]; p < s.eptr[e + 1]; ++p) {
            const int32_t cv = s.v_o2c[s.evtx[p]];
            if (cv >= 0) s.v_del[cv] = 1;  // same-value stores from every full hyperedge
        }
    }
}

__global__ void k_fe_apply(InstState *st, int count) {
    const int b = blockIdx.y;
    if (b >= count) return;
    InstState &s = st[b];
    if (!s.fe_stage || s.status) return;
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < s.m; r += gridDim.x * blockDim.x) {
        if (s.e_del[r]) continue;  // full: goes whole
        const int32_t e = s.e_c2o[r];
        int32_t lost = 0;
        for (int32_t p = s.eptr[e]; p < s.eptr[e + 1]; ++p) {
            const int32_t cv = s.v_o2c[s.evtx[p]];
            lost += cv >= 0 && s.v_del[cv];
        }
        if (lost) {
            s.f[e] -= lost;
            if (s.f[e] <= 0) s.e_del[r] = 1;
        }
    }
}

// Exclusive block scan of one int per thread (blockDim.x = 1024).
__device__ int32_t scan1024(int32_t x, int32_t *total, int32_t *sh /*[33]*/) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int32_t w = sh[lane];
        int32_t winc = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, winc, o);
            if (lane >= o) winc += y;
        }
        sh[lane] = winc - w;
        if (lane == 31) sh[32] = winc;
    }
    __syncthreads();
    const int32_t r = inc - x + sh[warp];
    *total = sh[32];
    __syncthreads();
    return r;
}

// Keep the current ids whose flag del[] is 0, in order; update both maps.
// Returns the new count.  With `taken` set, records the input id of every
// dropped item there.  Chunked so the in-place update of c2o never
// overwrites an entry not yet read.
__device__ int32_t compact_ids(int32_t count, const uint8_t *del, int32_t *c2o, int32_t *o2c,
                               uint8_t *taken, int32_t *sh) {
    int32_t carry = 0;
    for (int32_t base = 0; base < count; base += blockDim.x) {
        const int32_t r = base + threadIdx.x;
        int32_t keep = 0, orig = -1;
        if (r < count) {
            keep = del[r] == 0;
            orig = c2o[r];
        }
        int32_t tot;
        const int32_t ex = scan1024(keep, &tot, sh);
        if (r < count) {
            o2c[orig] = keep ? carry + ex : -1;
            if (keep) c2o[carry + ex] = orig;
            else if (taken) taken[orig] = 1;
        }
        carry += tot;
        __syncthreads();
    }
    return carry;
}

__global__ void __launch_bounds__(1024) k_fe_compact(InstState *st, int count, BatchCounters *ctr,
                                                     int32_t *done_list) {
    __shared__ int32_t sh[33];
    const int b = blockIdx.x;
    if (b >= count) return;
    InstState &s = st[b];
    const bool go = s.fe_stage != 0;
    const int32_t m = s.m, n = s.n;
    __syncthreads();  // every thread has read the state before thread 0 rewrites it
    if (!go) return;
    const int32_t m2 = compact_ids(m, s.e_del, s.e_c2o, s.e_o2c, nullptr, sh);
    const int32_t n2 = compact_ids(n, s.v_del, s.v_c2o, s.v_o2c, s.forced, sh);
    const bool changed = m2 != m || n2 != n;
    if (threadIdx.x == 0) {
        s.fe_stage = 0;
        s.fe_passes += 1;
        s.k -= n - n2;
        s.m = s.m_dp = m2;
        s.n = s.n_next = n2;
        if (ctr) {
            atomicSub(&ctr->m_alive, m - m2);
            atomicSub(&ctr->n_alive, n - n2);
        }
        if (changed) s.md_full = 1;  // lowered demands change maxf of untouched vertices too
        if (!changed) {
            s.active = 0;
            if (ctr) {
                atomicSub(&ctr->active, 1);
                if (done_list) done_list[atomicAdd(&ctr->n_done, 1)] = b;
            }
        } else if (ctr) {
            atomicOr(&ctr->changed_any, 1);
        }
    }
    if (changed) {  // hyperedge rows of the next round's DP pass, all candidates
        for (int32_t r = threadIdx.x; r < m2; r += blockDim.x) {
            s.e_f[r] = s.f[s.e_c2o[r]];
            s.e_s[r] = -1;
            s.e_del[r] = 0;
        }
        if (s.e_dirty_rb)
            for (int32_t w = threadIdx.x; w < (m2 + 127) / 128; w += blockDim.x) s.e_dirty_rb[w] = 0;
        if (s.occ[0]) {
            const int64_t words = (int64_t)((m2 + 255) / 256) * 2 * s.occ_words[0];
            for (int64_t w = threadIdx.x; w < words; w += blockDim.x) s.occ[0][w] = 0;
        }
        if (threadIdx.x == 0) s.has_loose = 0;
    }
}

}  // namespace

cudaError_t launch_full_edges(InstState *st, int count, BatchCounters *ctr, int32_t *done_list,
                              int sms, cudaStream_t s) {
    const int gx = count > 1 ? 2 : sms * 4;
    k_fe_mark<<<dim3(gx, count), 256, 0, s>>>(st, count);
    k_fe_apply<<<dim3(gx, count), 256, 0, s>>>(st, count);
    k_fe_compact<<<count, 1024, 0, s>>>(st, count, ctr, done_list);
    return cudaGetLastError();
}

}  // namespace mhs

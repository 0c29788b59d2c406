// mhs_api.cpp -- the C ABI of include/mhs.h: validation, device memory,
// the round driver of Algorithm 3 and result extraction.
#include "mhs.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "host_internal.h"
#include "kernels.h"
#include "mhs_internal.h"

using namespace mhs;

namespace mhs {
thread_local std::string g_err;

mhs_status set_error(mhs_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}
}  // namespace mhs

namespace {

#define fail mhs::set_error

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? MHS_ENOMEM : MHS_ECUDA,        \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline int64_t kpad_bytes(int64_t K) { return round_up(std::max<int64_t>(K, 1), kTcK); }
inline int64_t kpad_words(int64_t K) {
    return round_up(std::max<int64_t>((K + 31) / 32, 1), 4);
}
// occupancy words per row block: one bit per K block of kOccK columns
inline int64_t occ_words(int64_t K) { return (kpad_bytes(K) / kOccK + 31) / 32; }
// chunks of 1024 ids in the larger of an instance's two id ranges
inline int64_t compact_chunks(int64_t n0, int64_t m0) {
    return (std::max<int64_t>(std::max(n0, m0), 1) + 1023) / 1024;
}

}  // namespace

// Library-owned stream-ordered memory pool (keeps freed blocks for reuse).
namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};
}  // namespace

cudaError_t mhs::pool_for(int dev, cudaMemPool_t *out) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_pool[dev]) {
        cudaMemPoolProps p;
        std::memset(&p, 0, sizeof(p));
        p.allocType = cudaMemAllocationTypePinned;
        p.handleTypes = cudaMemHandleTypeNone;
        p.location.type = cudaMemLocationTypeDevice;
        p.location.id = dev;
        cudaError_t e = cudaMemPoolCreate(&g_pool[dev], &p);
        if (e != cudaSuccess) return e;
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

namespace {
std::mutex g_pin_mu;
std::vector<void *> g_pin_free;  // slab blocks not in use (the slab is never returned)
}  // namespace

void *mhs::pinned_block() {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        constexpr size_t kChunk = 128 * kPinnedBlock;
        void *c = nullptr;
        if (cudaMallocHost(&c, kChunk) != cudaSuccess) return nullptr;
        for (size_t o = 0; o < kChunk; o += kPinnedBlock)
            g_pin_free.push_back(static_cast<uint8_t *>(c) + o);
    }
    void *b = g_pin_free.back();
    g_pin_free.pop_back();
    return b;
}

void mhs::pinned_release(void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

namespace {
std::vector<std::pair<size_t, void *>> g_stage_free;  // (class, buffer), under g_pin_mu
}  // namespace

void *mhs::pinned_take(size_t bytes, size_t *cls) {
    size_t c = (size_t)64 << 10;
    while (c < bytes) c <<= 1;
    *cls = c;
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        for (size_t i = 0; i < g_stage_free.size(); ++i)
            if (g_stage_free[i].first == c) {
                void *p = g_stage_free[i].second;
                g_stage_free.erase(g_stage_free.begin() + (long)i);
                return p;
            }
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, c) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void mhs::pinned_give(void *p, size_t cls) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_stage_free.push_back({cls, p});
}

namespace {
// Dense operand regions that are known to be all zero, kept for reuse by
// later loads of similar size.  Every phase clears exactly the incidences it
// set, so an instance that finished without a device error leaves its
// operands all zero; a load that reuses them skips the memset (the largest
// fixed cost of a load: 1.6 GB for the 20,000 x 40,000 power-law instance).
struct ZeroBlock {
    int dev;
    uint8_t *p;
    int64_t bytes;
};
std::mutex g_zero_mu;
std::vector<ZeroBlock> g_zero;
// Budget of the cache (a batch of 4,096 instances of up to 2,000 x 4,000
// holds 16.7 GB of operands).  A load whose allocation fails empties the
// cache and retries.
constexpr int64_t kZeroCacheBytes = 32ll << 30;

uint8_t *zero_take(int dev, int64_t bytes) {
    std::lock_guard<std::mutex> lk(g_zero_mu);
    for (size_t i = 0; i < g_zero.size(); ++i) {
        const ZeroBlock &z = g_zero[i];
        if (z.dev == dev && z.bytes >= bytes && z.bytes <= bytes + bytes / 4) {
            uint8_t *p = z.p;
            g_zero.erase(g_zero.begin() + (long)i);
            return p;
        }
    }
    return nullptr;
}

// Keep an all-zero region (its stream has been synchronised); the oldest go
// back to the pool beyond the cache's budget.
void zero_put(int dev, uint8_t *p, int64_t bytes) {
    std::vector<uint8_t *> drop;
    {
        std::lock_guard<std::mutex> lk(g_zero_mu);
        g_zero.push_back({dev, p, bytes});
        int64_t total = 0;
        for (const ZeroBlock &z : g_zero) total += z.bytes;
        while (total > kZeroCacheBytes && !g_zero.empty()) {
            total -= g_zero.front().bytes;
            drop.push_back(g_zero.front().p);
            g_zero.erase(g_zero.begin());
        }
    }
    for (uint8_t *q : drop) cudaFreeAsync(q, nullptr);
}

// Return every cached region of a device to the pool (before retrying an
// allocation that failed).
void zero_flush(int dev) {
    std::vector<uint8_t *> drop;
    {
        std::lock_guard<std::mutex> lk(g_zero_mu);
        for (size_t i = 0; i < g_zero.size();) {
            if (g_zero[i].dev == dev) {
                drop.push_back(g_zero[i].p);
                g_zero.erase(g_zero.begin() + (long)i);
            } else {
                ++i;
            }
        }
    }
    for (uint8_t *q : drop) cudaFreeAsync(q, nullptr);
    if (!drop.empty()) cudaDeviceSynchronize();
}

// Sub-allocation plan of one arena.
struct Arena {
    int64_t bytes = 0;
    int64_t take(int64_t nbytes) {
        int64_t off = bytes;
        bytes += round_up(std::max<int64_t>(nbytes, 1), 256);
        return off;
    }
};

struct HostInst {  // per-instance host bookkeeping
    int32_t n0, m0;
    int64_t nnz0;
    int64_t k;
};

}  // namespace

struct mhs_instance {
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    mhs_options opt{};
    int contraction = kFp8;
    int32_t count = 0;
    std::vector<HostInst> hinst;
    std::vector<InstState> hstate;  // host mirror: pointers and static fields
    // a batch's page-locked staging: its states, then its tensor maps
    uint8_t *stage = nullptr;
    size_t stage_cls = 0;
    int64_t stage_tmaps = 0;        // offset of the tensor maps in `stage`
    // a single instance's host inputs, staged page-locked for their copies
    uint8_t *in_stage = nullptr;
    size_t in_stage_cls = 0;
    uint8_t *arena = nullptr;       // all device memory of the instance
    InstState *dstate = nullptr;
    Plan *dplan = nullptr;
    BatchCounters *dctr = nullptr;
    int32_t *dkerr = nullptr;
    // one pinned slab block: counters [0, 64), error word [64, 128), plan
    // header staging [128, 256), a single instance's tensor maps [256, 768)
    uint8_t *pin = nullptr;
    BatchCounters *hctr = nullptr;
    int32_t *hkerr = nullptr;
    int64_t max_nnz = 0, max_m = 0, max_n = 0;
    int32_t compact_blocks = 1;  // compaction blocks per instance (> 1: chained scan)
    TileChoice tiles{kTcNDefault, 16, 1, 0};  // tcgen05 tile shape of this load
    // arena offsets of the batch-wide input arrays
    int64_t in_eptr = 0, in_evtx = 0, in_f = 0;
    int64_t sum_m1 = 0, sum_nnz = 0, sum_m = 0;
    // dense operands: a separate allocation, reusable when known all zero
    uint8_t *dense = nullptr;
    int64_t dense_bytes = 0;
    bool dense_zeroed = false;  // taken all-zero from the cache or memset at load
    bool faulted = false;       // a device error was seen: the operands may be dirty
    // round graphs: graph[0] plain, graph[1] with timing events
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    // the whole fixpoint: a conditional WHILE node whose body is one round
    cudaGraphExec_t loop_graph = nullptr;
    int32_t round_cap = 0;
    // timing
    bool timing = false;
    cudaEvent_t ev[6] = {};
    float last_ms[4] = {0, 0, 0, 0};
    int32_t rounds_done = 0;
    // sharded passes (mhs_pass_*): 0 between rounds, 1 DP pass open,
    // 2 DP pass ended, 3 MD pass open
    int32_t pass_state = 0;
};

namespace {

static_assert(sizeof(BatchCounters) <= 64, "counters fit their pinned slot");
static_assert(sizeof(Plan) <= 128, "plan header fits its pinned slot");

void destroy(mhs_instance *h) {
    if (!h) return;
    // no copy may still target the pinned block when it returns to the slab
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto &g : h->graph)
        if (g) cudaGraphExecDestroy(g);
    if (h->loop_graph) cudaGraphExecDestroy(h->loop_graph);
    for (auto &e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->arena) cudaFreeAsync(h->arena, h->stream);  // stream-ordered
    if (h->dense) {
        const bool clean = h->dense_zeroed && !h->faulted && (!h->hkerr || *h->hkerr == 0);
        if (clean) zero_put(h->device, h->dense, h->dense_bytes);
        else cudaFreeAsync(h->dense, h->stream);
    }
    pinned_release(h->pin);
    pinned_give(h->stage, h->stage_cls);
    pinned_give(h->in_stage, h->in_stage_cls);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

mhs_status check_options(const mhs_options *opt, mhs_options *out) {
    mhs_default_options(out);
    if (!opt) return MHS_OK;
    *out = *opt;
    if (out->contraction < 0 || out->contraction > 2)
        return fail(MHS_EINVAL, "options.contraction must be 0 (auto), 1 (fp8) or 2 (popcount)");
    if (out->max_rounds < 0) return fail(MHS_EINVAL, "options.max_rounds must be >= 0");
    if (out->layout < 0 || out->layout > 3)
        return fail(MHS_EINVAL,
                    "options.layout must be 0 (auto), 1 (input), 2 (sorted) or 3 (degree)");
    if (out->sparsity < 0 || out->sparsity > 2)
        return fail(MHS_EINVAL, "options.sparsity must be 0 (auto), 1 (skip) or 2 (dense)");
    if (out->edge_rule < 0 || out->edge_rule > 1)
        return fail(MHS_EINVAL, "options.edge_rule must be 0 (DP) or 1 (SE)");
    if (out->full_edges < 0 || out->full_edges > 1)
        return fail(MHS_EINVAL, "options.full_edges must be 0 or 1");
    if (out->full_edges && out->max_rounds)
        return fail(MHS_EINVAL, "options.full_edges needs max_rounds = 0");
    if (out->tile_m != 0 && out->tile_m != kTcM)
        return fail(MHS_EINVAL, "options.tile_m must be 0 (auto) or 128");
    if (out->tile_n != 0 && out->tile_n != 128 && out->tile_n != 256)
        return fail(MHS_EINVAL, "options.tile_n must be 0 (autotune), 128 or 256");
    if (out->group_rows < 0 || out->group_rows > 4096)
        return fail(MHS_EINVAL, "options.group_rows must be 0 (autotune) or 1..4096");
    if (out->half_stages < 0 || out->half_stages > 2)
        return fail(MHS_EINVAL, "options.half_stages must be 0 (autotune), 1 (on) or 2 (off)");
    if (out->reserved[0] != 0) return fail(MHS_EINVAL, "options.reserved must be zero");
    return MHS_OK;
}

// Host-side structural validation of one instance's CSR.
// Checks of one instance's host CSR.  quiet: report only the status (safe
// on several threads at once: the error text is not touched).
mhs_status validate_host(int32_t n, int32_t m, const int64_t *eptr64, const int32_t *eptr32,
                         const int32_t *evtx, const int32_t *demand, std::vector<int32_t> &mark,
                         int32_t tag_base, const char *what, bool quiet = false) {
    auto bad = [quiet](mhs_status st, const char *fmt, auto... args) {
        return quiet ? st : mhs::set_error(st, fmt, args...);
    };
    if (n < 0 || m < 0) return bad(MHS_EINVAL, "%s: n and m must be >= 0", what);
    if (n >= (1 << 24) || m >= (1 << 24))
        return bad(MHS_EINVAL, "%s: n and m must be < 2^24 (exact FP32 counts)", what);
    auto ptr = [&](int64_t i) -> int64_t { return eptr64 ? eptr64[i] : eptr32[i]; };
    if ((size_t)n > mark.size()) mark.assign((size_t)n, -1);
    for (int32_t e = 0; e < m; ++e) {
        int64_t a = ptr(e), b = ptr(e + 1);
        if (b < a) return bad(MHS_EINVAL, "%s: edge_ptr decreases at hyperedge %d", what, e);
        if (b - a > (1ll << 24)) return bad(MHS_EINVAL, "%s: hyperedge %d too large", what, e);
        if (demand[e] < 1) return bad(MHS_EINVAL, "%s: demand of hyperedge %d is < 1", what, e);
        for (int64_t p = a; p < b; ++p) {
            int32_t v = evtx[p];
            if (v < 0 || v >= n)
                return bad(MHS_EINVAL, "%s: hyperedge %d has vertex id %d outside [0,%d)", what,
                            e, v, n);
            if (mark[v] == tag_base + e)
                return bad(MHS_EINVAL, "%s: hyperedge %d lists vertex %d twice", what, e, v);
            mark[v] = tag_base + e;
        }
    }
    return MHS_OK;
}

// validate_host over hyperedge ranges on several threads for a large
// instance; a failure is validated again on this thread for its message.
// With `stage` (page-locked, the layout of the device copies: edge_ptr,
// edge_vtx, demand), each part also copies its range there once it has
// checked it, while the range is still in cache.  The pointer array must
// already be known monotone with edge_ptr[0] = 0.
mhs_status validate_host_parallel(int32_t n, int32_t m, const int32_t *eptr32,
                                  const int32_t *evtx, const int32_t *demand, int64_t nnz,
                                  const char *what, uint8_t *stage = nullptr) {
    std::vector<int32_t> mark;
    const int nt = nnz >= (1 << 16) ? (int)std::min<int64_t>(8, nnz >> 15) : 1;
    int32_t *s_ptr = reinterpret_cast<int32_t *>(stage);
    int32_t *s_vtx = stage ? s_ptr + (m + 1) : nullptr;
    int32_t *s_f = stage ? s_vtx + nnz : nullptr;
    std::atomic<bool> bad{false};
    auto part = [&](int t) {
        const int32_t e0 = (int32_t)((int64_t)m * t / nt);
        const int32_t e1 = (int32_t)((int64_t)m * (t + 1) / nt);
        std::vector<int32_t> mk;
        if (validate_host(n, e1 - e0, nullptr, eptr32 + e0, evtx, demand + e0, mk, 0, what,
                          /*quiet=*/true)) {
            bad = true;
            return;
        }
        if (stage) {
            const int32_t p0 = eptr32[e0], p1 = eptr32[e1];
            std::memcpy(s_ptr + e0, eptr32 + e0, 4 * (size_t)(e1 - e0 + (t == nt - 1 ? 1 : 0)));
            if (p1 > p0) std::memcpy(s_vtx + p0, evtx + p0, 4 * (size_t)(p1 - p0));
            if (e1 > e0) std::memcpy(s_f + e0, demand + e0, 4 * (size_t)(e1 - e0));
        }
    };
    if (nt <= 1) {
        part(0);
        if (!bad) return MHS_OK;
        return validate_host(n, m, nullptr, eptr32, evtx, demand, mark, 0, what);
    }
    std::vector<std::thread> threads;
    int started = 1;
    try {
        for (; started < nt; ++started) threads.emplace_back(part, started);
    } catch (...) {  // a thread that cannot start: its part runs here
    }
    for (int t = started; t < nt; ++t) part(t);
    part(0);
    for (std::thread &x : threads) x.join();
    if (!bad) return MHS_OK;
    return validate_host(n, m, nullptr, eptr32, evtx, demand, mark, 0, what);
}

struct Layout {  // byte offsets inside the arena for one instance
    int64_t occ0, occ1;
    int64_t eptr, evtx, f;
    int64_t v_o2c, v_c2o, e_o2c, e_c2o, e_f, e_s, v_deg, v_maxf, v_cnt, e_del, v_del, forced;
    int64_t e_dirty_rb, v_dirty, v_dirty_rb, e_prev, e_rec, scan;
    int64_t A, At, Ab, Atb;
};

mhs_status create(int32_t count, const int32_t *n, const int32_t *m, const int64_t *nnz,
                  const int64_t *k, const mhs_options *opt_in, void *cuda_stream,
                  mhs_instance **out, std::vector<Layout> &lay, int64_t &glob_off) {
    mhs_options opt;
    mhs_status st = check_options(opt_in, &opt);
    if (st) return st;
    auto *h = new mhs_instance();
    h->opt = opt;
    h->contraction = opt.contraction == kPopcount ? kPopcount : kFp8;
    h->count = count;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        destroy(h);
        return fail(MHS_ECUDA, "no CUDA device");
    }
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (cuda_stream) {
        h->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            destroy(h);
            return fail(MHS_ECUDA, "cudaStreamCreate failed");
        }
        h->own_stream = true;
    }
    const bool dense = h->contraction == kFp8;
    Arena ar;
    lay.resize(count);
    h->hinst.resize(count);
    // inputs are laid out array by array over the batch, so that a batch is
    // uploaded with one copy per array
    int64_t sum_m1 = 0, sum_z = 0, sum_m = 0;
    for (int b = 0; b < count; ++b) { sum_m1 += m[b] + 1; sum_z += nnz[b]; sum_m += m[b]; }
    const int64_t off_eptr = ar.take(4 * sum_m1);
    const int64_t off_evtx = ar.take(4 * sum_z);
    const int64_t off_f = ar.take(4 * sum_m);
    h->in_eptr = off_eptr;
    h->in_evtx = off_evtx;
    h->in_f = off_f;
    h->sum_m1 = sum_m1;
    h->sum_nnz = sum_z;
    h->sum_m = sum_m;
    int64_t c_m1 = 0, c_z = 0, c_m = 0;
    int64_t tiles_dp = 0, tiles_md = 0;
    if (dense) {  // the tile shape: options, else the autotuner's table for this size class
        int64_t rows = 0;
        for (int b = 0; b < count; ++b) rows += std::max<int64_t>(n[b], m[b]);
        h->tiles = choose_tiles(count, rows / std::max(count, 1), opt);
    }
    for (int b = 0; b < count; ++b) {
        Layout &L = lay[b];
        const int64_t n0 = n[b], m0 = m[b], z = nnz[b];
        h->hinst[b] = {n[b], m[b], z, k[b]};
        h->max_nnz = std::max(h->max_nnz, z);
        h->max_m = std::max(h->max_m, m0);
        h->max_n = std::max(h->max_n, n0);
        // every changing round deletes an item, so n + m + 1 rounds always
        // suffice; with FE, every fixpoint but the last is followed by an FE
        // pass that deletes an item, so 2 (n + m) + 2 do
        h->round_cap = (int32_t)std::min<int64_t>(
            std::max<int64_t>(h->round_cap, 2 * (n0 + m0) + 4), INT32_MAX);
        L.eptr = off_eptr + 4 * c_m1;
        L.evtx = off_evtx + 4 * c_z;
        L.f = off_f + 4 * c_m;
        c_m1 += m0 + 1;
        c_z += z;
        c_m += m0;
        L.v_o2c = ar.take(4 * n0);
        L.v_c2o = ar.take(4 * n0);
        L.e_o2c = ar.take(4 * m0);
        L.e_c2o = ar.take(4 * m0);
        L.e_f = ar.take(4 * m0);
        L.e_s = ar.take(4 * m0);
        L.v_deg = ar.take(4 * (n0 + 1));
        L.v_maxf = ar.take(4 * n0);
        L.v_cnt = ar.take(4 * (n0 + 1));
        L.e_del = ar.take(m0);
        L.v_del = ar.take(n0);
        L.forced = opt.full_edges ? ar.take(n0) : -1;
        L.v_dirty = ar.take(n0);
        L.e_prev = ar.take(4 * m0);
        L.e_rec = dense ? ar.take(16 * m0) : -1;
        // a single instance compacts with one block per chunk of 1024 ids
        L.scan = count == 1 ? ar.take(8 * compact_chunks(n0, m0)) : -1;
        L.e_dirty_rb = ar.take(round_up(std::max<int64_t>(m0, 1), kRowAlign) / kTcM);
        L.v_dirty_rb = ar.take(round_up(std::max<int64_t>(n0, 1), kRowAlign) / kTcM);
        if (dense) {
            const int64_t arows = round_up(std::max<int64_t>(m0, 1), kRowAlign);
            const int64_t atrows = round_up(std::max<int64_t>(n0, 1), kRowAlign);
            L.occ0 = ar.take(4 * (arows / kTcM) * occ_words(n0));
            L.occ1 = ar.take(4 * (atrows / kTcM) * occ_words(m0));
        } else {
            L.occ0 = L.occ1 = -1;
        }
        tiles_dp += tc_tiles((int32_t)m0, h->tiles.tile_n);
        tiles_md += tc_tiles((int32_t)n0, h->tiles.tile_n);
    }
    // the operands of all instances, contiguous in their own allocation,
    // all zero at load: the scatter/clear passes leave them all-zero between
    // phases
    Arena ad;
    for (int b = 0; b < count; ++b) {
        Layout &L = lay[b];
        const int64_t n0 = n[b], m0 = m[b];
        const int64_t arows = round_up(std::max<int64_t>(m0, 1), kRowAlign);
        const int64_t atrows = round_up(std::max<int64_t>(n0, 1), kRowAlign);
        if (dense) {
            L.A = ad.take(arows * kpad_bytes(n0));
            L.At = ad.take(atrows * kpad_bytes(m0));
            L.Ab = L.Atb = -1;
        } else {
            L.Ab = ad.take(arows * kpad_words(n0) * 4);
            L.Atb = ad.take(atrows * kpad_words(m0) * 4);
            L.A = L.At = -1;
        }
    }
    h->dense_bytes = ad.bytes;
    // batch-level objects
    const int64_t off_state = ar.take((int64_t)sizeof(InstState) * count);
    const int64_t off_plan = ar.take(sizeof(Plan));
    const int64_t off_rowoff = ar.take(4 * (int64_t)(count + 1));
    const int64_t off_tileoff = ar.take(8 * (int64_t)(count + 1));
    const int64_t off_ctr = ar.take(sizeof(BatchCounters));
    const int64_t off_kerr = ar.take(4);
    const int64_t off_tmaps = ar.take(dense ? (int64_t)tmap_bytes() * 2 * count : 0);
    const int64_t list_cap = dense ? std::max<int64_t>(std::max(tiles_dp, tiles_md), 1) : 0;
    const int64_t off_list = ar.take(8 * list_cap);
    glob_off = off_tmaps;

    cudaMemPool_t pool;
    cudaError_t ce = pool_for(h->device, &pool);
    h->dense = zero_take(h->device, h->dense_bytes);
    h->dense_zeroed = h->dense != nullptr;
    for (int attempt = 0; attempt < 2 && ce == cudaSuccess; ++attempt) {
        if (!h->arena)
            ce = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&h->arena), (size_t)ar.bytes,
                                         pool, h->stream);
        if (ce == cudaSuccess && !h->dense)
            ce = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&h->dense),
                                         (size_t)h->dense_bytes, pool, h->stream);
        if (ce != cudaErrorMemoryAllocation || attempt == 1) break;
        cudaGetLastError();
        zero_flush(h->device);  // cached zero regions go back to the pool, then retry
        ce = cudaSuccess;
    }
    if (ce != cudaSuccess) {
        destroy(h);
        return fail(ce == cudaErrorMemoryAllocation ? MHS_ENOMEM : MHS_ECUDA,
                    "device allocation of %lld bytes failed: %s",
                    (long long)(ar.bytes + h->dense_bytes), cudaGetErrorString(ce));
    }
    uint8_t *base = h->arena;
    uint8_t *dbase = h->dense;
    h->dstate = reinterpret_cast<InstState *>(base + off_state);
    h->dplan = reinterpret_cast<Plan *>(base + off_plan);
    h->dctr = reinterpret_cast<BatchCounters *>(base + off_ctr);
    h->dkerr = reinterpret_cast<int32_t *>(base + off_kerr);
    h->pin = static_cast<uint8_t *>(pinned_block());
    if (!h->pin) {
        destroy(h);
        return fail(MHS_ENOMEM, "pinned host allocation failed");
    }
    h->hctr = reinterpret_cast<BatchCounters *>(h->pin);
    h->hkerr = reinterpret_cast<int32_t *>(h->pin + 64);
    h->hstate.resize(count);
    if (count > 1) {  // without it the copies stage through pageable memory
        h->stage_tmaps = round_up((int64_t)sizeof(InstState) * count, 128);
        h->stage = static_cast<uint8_t *>(pinned_take(
            (size_t)(h->stage_tmaps + (dense ? (int64_t)tmap_bytes() * 2 * count : 0)),
            &h->stage_cls));
    }
    int64_t vbase = 0, ebase = 0;
    for (int b = 0; b < count; ++b) {
        const Layout &L = lay[b];
        InstState s;
        std::memset(&s, 0, sizeof(s));
        s.v_base = vbase;
        s.e_base = ebase;
        vbase += n[b];
        ebase += m[b];
        s.n0 = n[b];
        s.m0 = m[b];
        s.nnz0 = nnz[b];
        s.k = k[b];
        s.layout_sorted = layout_code(opt.layout);
        s.no_skip = opt.sparsity == MHS_SPARSITY_DENSE;
        s.edge_rule = opt.edge_rule;
        s.full_edges = opt.full_edges;
        s.forced = L.forced >= 0 ? base + L.forced : nullptr;
        s.v_dirty = base + L.v_dirty;
        s.e_prev = reinterpret_cast<int32_t *>(base + L.e_prev);
        s.scan_status =
            L.scan >= 0 ? reinterpret_cast<unsigned long long *>(base + L.scan) : nullptr;
        s.scan_chunks = L.scan >= 0 ? (int32_t)compact_chunks(s.n0, s.m0) : 0;
        if (s.scan_chunks > 1) h->compact_blocks = s.scan_chunks;
        s.scan_ticket = 0;
        s.scan_epoch = 0;
        s.e_rec = L.e_rec >= 0 ? reinterpret_cast<int4 *>(base + L.e_rec) : nullptr;
        s.e_dirty_rb = base + L.e_dirty_rb;
        s.v_dirty_rb = base + L.v_dirty_rb;
        s.eptr = reinterpret_cast<int32_t *>(base + L.eptr);
        s.evtx = reinterpret_cast<int32_t *>(base + L.evtx);
        s.f = reinterpret_cast<int32_t *>(base + L.f);
        s.v_o2c = reinterpret_cast<int32_t *>(base + L.v_o2c);
        s.v_c2o = reinterpret_cast<int32_t *>(base + L.v_c2o);
        s.e_o2c = reinterpret_cast<int32_t *>(base + L.e_o2c);
        s.e_c2o = reinterpret_cast<int32_t *>(base + L.e_c2o);
        s.e_f = reinterpret_cast<int32_t *>(base + L.e_f);
        s.e_s = reinterpret_cast<int32_t *>(base + L.e_s);
        s.v_deg = reinterpret_cast<int32_t *>(base + L.v_deg);
        s.v_maxf = reinterpret_cast<int32_t *>(base + L.v_maxf);
        s.v_cnt = reinterpret_cast<int32_t *>(base + L.v_cnt);
        s.e_del = base + L.e_del;
        s.v_del = base + L.v_del;
        const int64_t arows = round_up(std::max<int64_t>(m[b], 1), kRowAlign);
        const int64_t atrows = round_up(std::max<int64_t>(n[b], 1), kRowAlign);
        s.A_rows = (int32_t)arows;
        s.At_rows = (int32_t)atrows;
        if (dense) {
            s.occ[0] = reinterpret_cast<uint32_t *>(base + L.occ0);
            s.occ[1] = reinterpret_cast<uint32_t *>(base + L.occ1);
            s.occ_words[0] = (int32_t)occ_words(n[b]);
            s.occ_words[1] = (int32_t)occ_words(m[b]);
            s.A = dbase + L.A;
            s.At = dbase + L.At;
            s.A_pitch = kpad_bytes(n[b]);
            s.At_pitch = kpad_bytes(m[b]);
            uint8_t *tm = base + off_tmaps + (int64_t)tmap_bytes() * 2 * b;
            s.tmap_A = tm;
            s.tmap_At = tm + tmap_bytes();
        } else {
            s.Ab = reinterpret_cast<uint32_t *>(dbase + L.Ab);
            s.Atb = reinterpret_cast<uint32_t *>(dbase + L.Atb);
            s.Ab_pitch = (int32_t)kpad_words(n[b]);
            s.Atb_pitch = (int32_t)kpad_words(m[b]);
        }
        h->hstate[b] = s;
    }
    // device plan header
    Plan p;
    std::memset(&p, 0, sizeof(p));
    p.count = count;
    p.row_off = reinterpret_cast<int32_t *>(base + off_rowoff);
    p.tile_off = reinterpret_cast<int64_t *>(base + off_tileoff);
    p.tile_list = reinterpret_cast<int64_t *>(base + off_list);
    p.list_cap = (int32_t)std::min<int64_t>(list_cap, INT32_MAX);
    p.group_rows = h->tiles.group_rows;
    p.tile_n = h->tiles.tile_n;
    p.half_stages = h->tiles.half_stages;
    // heavy / light tile queues: one instance on 128 x 256 tiles only (measured:
    // power-law +2.8 %; with 128 x 128 tiles, whose four accumulators already
    // buffer the MMA and the epilogue, interval -6 %; the batch -1 %)
    p.two_queues = count == 1 && h->tiles.tile_n == 256 ? 1 : 0;
    std::memcpy(h->pin + 128, &p, sizeof(p));  // staged in pinned memory: no synchronisation
    ce = cudaMemcpyAsync(h->dplan, h->pin + 128, sizeof(p), cudaMemcpyHostToDevice, h->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(h->dkerr, 0, 4, h->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(h->dctr, 0, sizeof(BatchCounters), h->stream);
    if (ce != cudaSuccess) {
        destroy(h);
        return fail(MHS_ECUDA, "setup copy failed: %s", cudaGetErrorString(ce));
    }
    *out = h;
    return MHS_OK;
}

// Tensor maps (host encode, one copy to the device), state upload, and the
// device-side build of the vertex -> hyperedge lists and id maps.
// The instance states to the device (through the batch's pinned staging).
cudaError_t upload_states(mhs_instance *h) {
    const size_t sb = sizeof(InstState) * (size_t)h->count;
    const void *src = h->hstate.data();
    if (h->stage) {  // no copy from it is in flight: every load step before synchronised
        std::memcpy(h->stage, src, sb);
        src = h->stage;
    }
    return cudaMemcpyAsync(h->dstate, src, sb, cudaMemcpyHostToDevice, h->stream);
}

mhs_status finish_load(mhs_instance *h, int64_t tmap_off) {
    const bool dense = h->contraction == kFp8;
    if (dense) {
        CUDA_TRY(prepare_tc_contract());
        const size_t mb = tmap_bytes() * 2 * h->count;
        // one instance: its pinned block; a batch: its pinned staging, else a local vector
        const bool pinned = mb <= kPinnedBlock - 256 || h->stage;
        std::vector<uint8_t> local(pinned ? 0 : mb);
        uint8_t *maps = mb <= kPinnedBlock - 256 ? h->pin + 256
                        : h->stage              ? h->stage + h->stage_tmaps
                                                : local.data();
        const int count = h->count;
        auto enc = [&](int b) {
            const InstState &s = h->hstate[b];
            return make_operand_tmap(maps + tmap_bytes() * 2 * b, s.A, s.A_pitch, s.A_rows) &&
                   make_operand_tmap(maps + tmap_bytes() * (2 * b + 1), s.At, s.At_pitch,
                                     s.At_rows);
        };
        // Four maps per instance: a large batch encodes them on several
        // threads.  Instance 0 goes first on this thread, which resolves the
        // driver's encoder before any other thread calls it.
        if (!enc(0)) return fail(MHS_ECUDA, "cuTensorMapEncodeTiled failed for instance 0");
        const int nt = count >= 512 ? 4 : 1;
        std::atomic<int> bad{count};  // lowest instance whose encoding failed
        auto share = [&](int t) {
            for (int b = 1 + t; b < count; b += nt)
                if (!enc(b)) {
                    int cur = bad.load();
                    while (b < cur && !bad.compare_exchange_weak(cur, b)) {
                    }
                }
        };
        // a new thread has no current context, which the encoder needs
        auto worker = [&](int t) {
            if (cudaSetDevice(h->device) != cudaSuccess) {
                int cur = bad.load();
                while (1 + t < cur && !bad.compare_exchange_weak(cur, 1 + t)) {
                }
                return;
            }
            share(t);
        };
        std::vector<std::thread> threads;
        int started = 1;
        try {
            for (; started < nt; ++started) threads.emplace_back(worker, started);
        } catch (...) {  // a thread that cannot start: its share runs here
        }
        for (int t = started; t < nt; ++t) share(t);
        share(0);
        for (std::thread &x : threads) x.join();
        if (bad.load() < count)
            return fail(MHS_ECUDA, "cuTensorMapEncodeTiled failed for instance %d", bad.load());
        CUDA_TRY(cudaMemcpyAsync(h->arena + tmap_off, maps, mb, cudaMemcpyHostToDevice, h->stream));
        if (!pinned) CUDA_TRY(cudaStreamSynchronize(h->stream));  // `local` goes out of scope
    }
    CUDA_TRY(upload_states(h));
    if (!h->dense_zeroed) {
        CUDA_TRY(cudaMemsetAsync(h->dense, 0, (size_t)h->dense_bytes, h->stream));
        h->dense_zeroed = true;
    }
    CUDA_TRY(launch_build(h->dstate, h->count, h->opt.max_rounds, h->max_nnz, h->max_m,
                          h->max_n, h->stream));
    return MHS_OK;
}

const char *status_text(int32_t st) {
    if (st & kErrBadVertex) return "vertex id out of range";
    if (st & kErrBadPtr) return "bad edge_ptr";
    if (st & kErrBadDemand) return "demand < 1";
    if (st & kErrCapacity) return "index beyond capacity";
    if (st & kErrTimeout) return "bounded wait timed out";
    return "unknown";
}

mhs_status check_device_status(mhs_instance *h) {
    if (*h->hkerr) {
        h->faulted = true;
        return fail(MHS_EDEVICE, "kernel reported error status 0x%x", *h->hkerr);
    }
    if (h->hctr->status_any) {
        h->faulted = true;
        return fail(MHS_EDEVICE, "instance reported error status 0x%x", h->hctr->status_any);
    }
    return MHS_OK;
}

// Enqueue one round (DP phase, MD phase, counters to pinned host memory).
cudaError_t enqueue_round(mhs_instance *h, bool with_events) {
    cudaError_t e = launch_round_phase(h->dstate, h->dplan, h->dctr, h->count, 0, h->contraction,
                                       h->sms, h->dkerr, h->stream,
                                       with_events ? h->ev[0] : nullptr,
                                       with_events ? h->ev[1] : nullptr, nullptr,
                                       h->compact_blocks, h->tiles.tile_n);
    if (e != cudaSuccess) return e;
    e = launch_round_phase(h->dstate, h->dplan, h->dctr, h->count, 1, h->contraction, h->sms,
                           h->dkerr, h->stream, with_events ? h->ev[2] : nullptr,
                           with_events ? h->ev[3] : nullptr, nullptr, h->compact_blocks,
                           h->tiles.tile_n);
    if (e == cudaSuccess && h->opt.full_edges)
        e = launch_full_edges(h->dstate, h->count, h->dctr, nullptr, h->sms, h->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(h->hctr, h->dctr, sizeof(BatchCounters), cudaMemcpyDeviceToHost,
                        h->stream);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(h->hkerr, h->dkerr, sizeof(int32_t), cudaMemcpyDeviceToHost,
                           h->stream);
}

mhs_status capture_round(mhs_instance *h, bool with_events, cudaGraphExec_t *out) {
    cudaGraph_t g;
    CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_round(h, with_events);
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(MHS_ECUDA, "graph capture failed: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(MHS_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return MHS_OK;
}

// One graph for Algorithm 3 to its fixpoint: reset the loop counter, then
// WHILE(condition) { DP phase; MD phase; condition kernel }, then copy the
// counters and the error word to pinned host memory.
mhs_status build_loop_graph(mhs_instance *h) {
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaGraphCreate(&g, 0));
    auto bail = [&](cudaError_t e, const char *what) {
        cudaGraphDestroy(g);
        return fail(MHS_ECUDA, "loop graph (%s): %s", what, cudaGetErrorString(e));
    };
    cudaGraphConditionalHandle cond;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return bail(e, "handle");
    cudaGraphNode_t reset;
    cudaMemsetParams mp;
    std::memset(&mp, 0, sizeof(mp));
    mp.dst = &h->dctr->loop_iters;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = 1;
    mp.height = 1;
    e = cudaGraphAddMemsetNode(&reset, g, nullptr, 0, &mp);
    if (e != cudaSuccess) return bail(e, "reset");
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    e = cudaGraphAddNode(&loop, g, &reset, nullptr, 1, &cp);
    if (e != cudaSuccess) return bail(e, "conditional node");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bail(e, "capture");
    cudaError_t e1 = launch_round_phase(h->dstate, h->dplan, h->dctr, h->count, 0, h->contraction,
                                        h->sms, h->dkerr, h->stream, nullptr, nullptr, nullptr,
                                        h->compact_blocks, h->tiles.tile_n);
    if (e1 == cudaSuccess)
        e1 = launch_round_phase(h->dstate, h->dplan, h->dctr, h->count, 1, h->contraction, h->sms,
                                h->dkerr, h->stream, nullptr, nullptr, nullptr,
                                h->compact_blocks, h->tiles.tile_n);
    if (e1 == cudaSuccess && h->opt.full_edges)
        e1 = launch_full_edges(h->dstate, h->count, h->dctr, nullptr, h->sms, h->stream);
    if (e1 == cudaSuccess)
        e1 = launch_loop_cond(cond, h->dctr, h->dkerr, h->round_cap, h->stream);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(h->stream, &captured);
    if (e1 != cudaSuccess) return bail(e1, "round");
    if (e != cudaSuccess) return bail(e, "end capture");
    cudaGraphNode_t c1, c2;
    e = cudaGraphAddMemcpyNode1D(&c1, g, &loop, 1, h->hctr, h->dctr, sizeof(BatchCounters),
                                 cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaGraphAddMemcpyNode1D(&c2, g, &c1, 1, h->hkerr, h->dkerr, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bail(e, "copies");
    e = cudaGraphInstantiate(&h->loop_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(MHS_ECUDA, "loop graph instantiate: %s", cudaGetErrorString(e));
    return MHS_OK;
}

mhs_status run_rounds(mhs_instance *h, int32_t limit, mhs_round_stats *stats) {
    if (h->pass_state != 0)
        return fail(MHS_EINVAL, "a sharded round is in progress (finish it with mhs_pass_end)");
    if (limit <= 0 && h->opt.use_graphs && !h->timing) {
        if (!h->loop_graph) {
            mhs_status st = build_loop_graph(h);
            if (st) return st;
        }
        CUDA_TRY(cudaGraphLaunch(h->loop_graph, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        if (*h->hkerr & kErrRoundCap)
            return fail(MHS_EDEVICE, "device round loop reached its cap of %d rounds", h->round_cap);
        mhs_status st = check_device_status(h);
        if (st) return st;
        if (stats) {
            stats->n_alive = h->hctr->n_alive;
            stats->m_alive = h->hctr->m_alive;
            stats->rounds = h->hctr->max_rounds_seen;
            stats->changed = h->hctr->changed_any;
            stats->dp_deleted = h->hctr->dp_deleted;
            stats->md_deleted = h->hctr->md_deleted;
            stats->active = h->hctr->active;
        }
        return MHS_OK;
    }
    if (h->timing) {
        for (auto &e : h->ev)
            if (!e) CUDA_TRY(cudaEventCreate(&e));
        for (float &x : h->last_ms) x = 0.f;
    }
    const int gi = h->timing ? 1 : 0;
    if (h->opt.use_graphs && !h->graph[gi]) {
        mhs_status st = capture_round(h, h->timing, &h->graph[gi]);
        if (st) return st;
    }
    int32_t done = 0;
    bool any = false;
    while (limit <= 0 || done < limit) {
        if (h->timing) CUDA_TRY(cudaEventRecord(h->ev[4], h->stream));
        if (h->graph[gi]) CUDA_TRY(cudaGraphLaunch(h->graph[gi], h->stream));
        else CUDA_TRY(enqueue_round(h, h->timing));
        if (h->timing) CUDA_TRY(cudaEventRecord(h->ev[5], h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        any = true;
        ++done;
        if (h->timing) {
            float a = 0, b = 0, t = 0;
            cudaEventElapsedTime(&a, h->ev[0], h->ev[1]);
            cudaEventElapsedTime(&b, h->ev[2], h->ev[3]);
            cudaEventElapsedTime(&t, h->ev[4], h->ev[5]);
            h->last_ms[0] += a;
            h->last_ms[1] += b;
            h->last_ms[3] += t;
            h->last_ms[2] += t - a - b;
        }
        mhs_status st = check_device_status(h);
        if (st) return st;
        if (h->hctr->active == 0) break;
    }
    if (stats) {
        if (any) {
            stats->n_alive = h->hctr->n_alive;
            stats->m_alive = h->hctr->m_alive;
            stats->rounds = h->hctr->max_rounds_seen;
            stats->changed = h->hctr->changed_any;
            stats->dp_deleted = h->hctr->dp_deleted;
            stats->md_deleted = h->hctr->md_deleted;
            stats->active = h->hctr->active;
        } else {
            std::memset(stats, 0, sizeof(*stats));
        }
    }
    return MHS_OK;
}

}  // namespace

extern "C" {

mhs_status mhs_default_options(mhs_options *opt) {
    if (!opt) return fail(MHS_EINVAL, "opt is NULL");
    std::memset(opt, 0, sizeof(*opt));
    opt->contraction = MHS_CONTRACT_AUTO;
    opt->max_rounds = 0;
    opt->use_graphs = 1;
    return MHS_OK;
}

mhs_status mhs_load(int32_t n, int32_t m, const int32_t *edge_ptr, const int32_t *edge_vtx,
                    const int32_t *demand, int64_t k, const mhs_options *opt, void *cuda_stream,
                    mhs_instance **out) {
    if (!out) return fail(MHS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!edge_ptr || (m > 0 && !demand)) return fail(MHS_EINVAL, "NULL input array");
    if (n < 0 || m < 0) return fail(MHS_EINVAL, "instance: n and m must be >= 0");
    if (n >= (1 << 24) || m >= (1 << 24))
        return fail(MHS_EINVAL, "instance: n and m must be < 2^24 (exact FP32 counts)");
    if (edge_ptr[0] != 0) return fail(MHS_EINVAL, "edge_ptr[0] must be 0");
    // The pointer array first (O(m)): the copies below read edge_ptr[m]
    // vertex ids, which a monotone array with edge_ptr[0] = 0 bounds.
    for (int32_t e = 0; e < m; ++e)
        if (edge_ptr[e + 1] < edge_ptr[e] || edge_ptr[e + 1] - edge_ptr[e] > (1 << 24)) {
            std::vector<int32_t> mk;  // the standard message
            mhs_status st = validate_host(n, m, nullptr, edge_ptr, edge_vtx, demand, mk, 0,
                                          "instance");
            return st ? st : fail(MHS_EINVAL, "instance: bad edge_ptr");
        }
    if (m > 0 && edge_ptr[m] > 0 && !edge_vtx) return fail(MHS_EINVAL, "edge_vtx is NULL");
    int64_t nnz = edge_ptr[m];
    std::vector<Layout> lay;
    int64_t tmoff = 0;
    mhs_instance *h = nullptr;
    mhs_status st = create(1, &n, &m, &nnz, &k, opt, cuda_stream, &h, lay, tmoff);
    if (st) return st;
    // The host checks the incidences, several threads each taking a range
    // of hyperedges and, once it has checked it, copying the range into
    // page-locked staging (a buffer of its own, nothing else writes it while
    // the copies run); the copies to the device follow.  Without staging the
    // inputs are copied from the caller's arrays while the host checks them.
    // No kernel reads them before the checks have passed.
    const InstState &s = h->hstate[0];
    const size_t b_ptr = 4 * ((size_t)m + 1), b_vtx = 4 * (size_t)nnz, b_f = 4 * (size_t)m;
    h->in_stage = static_cast<uint8_t *>(pinned_take(b_ptr + b_vtx + b_f, &h->in_stage_cls));
    const void *src_ptr = edge_ptr, *src_vtx = edge_vtx, *src_f = demand;
    if (uint8_t *in = h->in_stage) {
        st = validate_host_parallel(n, m, edge_ptr, edge_vtx, demand, nnz, "instance", in);
        if (st) {
            destroy(h);
            return st;
        }
        src_ptr = in;
        src_vtx = in + b_ptr;
        src_f = in + b_ptr + b_vtx;
    }
    cudaError_t e = cudaMemcpyAsync(const_cast<int32_t *>(s.eptr), src_ptr, b_ptr,
                                    cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && b_vtx)
        e = cudaMemcpyAsync(const_cast<int32_t *>(s.evtx), src_vtx, b_vtx, cudaMemcpyHostToDevice,
                            h->stream);
    if (e == cudaSuccess && b_f)
        e = cudaMemcpyAsync(const_cast<int32_t *>(s.f), src_f, b_f, cudaMemcpyHostToDevice,
                            h->stream);
    if (e != cudaSuccess) {
        destroy(h);
        return fail(MHS_ECUDA, "input copy failed: %s", cudaGetErrorString(e));
    }
    if (!h->in_stage) {
        st = validate_host_parallel(n, m, edge_ptr, edge_vtx, demand, nnz, "instance");
        if (st) {
            destroy(h);  // (waits for the copies)
            return st;
        }
    }
    st = finish_load(h, tmoff);
    if (st == MHS_OK && cudaStreamSynchronize(h->stream) != cudaSuccess)
        st = fail(MHS_ECUDA, "load failed: %s", cudaGetErrorString(cudaGetLastError()));
    if (st) {
        destroy(h);
        return st;
    }
    *out = h;
    return MHS_OK;
}

mhs_status mhs_load_device(int32_t n, int32_t m, const int32_t *edge_ptr, const int32_t *edge_vtx,
                           const int32_t *demand, int64_t k, const mhs_options *opt,
                           void *cuda_stream, mhs_instance **out) {
    if (!out) return fail(MHS_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 0 || m < 0) return fail(MHS_EINVAL, "n and m must be >= 0");
    if (n >= (1 << 24) || m >= (1 << 24)) return fail(MHS_EINVAL, "n and m must be < 2^24");
    if (!edge_ptr || (m > 0 && !demand)) return fail(MHS_EINVAL, "NULL input array");
    cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
    int32_t nnz32 = 0;
    CUDA_TRY(cudaMemcpyAsync(&nnz32, edge_ptr + m, 4, cudaMemcpyDeviceToHost, cs));
    CUDA_TRY(cudaStreamSynchronize(cs));
    if (nnz32 < 0) return fail(MHS_EINVAL, "edge_ptr[m] < 0");
    if (nnz32 > 0 && !edge_vtx) return fail(MHS_EINVAL, "edge_vtx is NULL");
    int64_t nnz = nnz32;
    std::vector<Layout> lay;
    int64_t tmoff = 0;
    mhs_instance *h = nullptr;
    mhs_status st = create(1, &n, &m, &nnz, &k, opt, cuda_stream, &h, lay, tmoff);
    if (st) return st;
    InstState &s = h->hstate[0];
    cudaError_t e = cudaMemcpyAsync(const_cast<int32_t *>(s.eptr), edge_ptr, 4 * ((size_t)m + 1),
                                    cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpyAsync(const_cast<int32_t *>(s.evtx), edge_vtx, 4 * (size_t)nnz,
                            cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && m > 0)
        e = cudaMemcpyAsync(const_cast<int32_t *>(s.f), demand, 4 * (size_t)m,
                            cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->dstate, h->hstate.data(), sizeof(InstState), cudaMemcpyHostToDevice,
                            h->stream);
    if (e == cudaSuccess) e = launch_validate(h->dstate, 1, h->stream);
    int32_t status = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&status, &h->dstate->status, 4, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        destroy(h);
        return fail(MHS_ECUDA, "device load failed: %s", cudaGetErrorString(e));
    }
    if (status) {
        destroy(h);
        return fail(MHS_EINVAL, "malformed device instance (status 0x%x: %s)", status,
                    status_text(status));
    }
    st = finish_load(h, tmoff);  // device inputs: nothing to wait for before returning
    if (st) {
        destroy(h);
        return st;
    }
    *out = h;
    return MHS_OK;
}

mhs_status mhs_load_batch(int32_t count, const int32_t *n, const int32_t *m,
                          const int64_t *edge_ptr, const int32_t *edge_vtx, const int32_t *demand,
                          const int64_t *k, const mhs_options *opt, void *cuda_stream,
                          mhs_instance **out) {
    if (!out) return fail(MHS_EINVAL, "out is NULL");
    *out = nullptr;
    // kernels index the instances of a batch by blockIdx.y
    if (count < 1 || count > 65535) return fail(MHS_EINVAL, "count must be in [1, 65535]");
    if (!n || !m || !edge_ptr || !k) return fail(MHS_EINVAL, "NULL input array");
    std::vector<int64_t> eoff(count + 1, 0), nnz(count);
    for (int b = 0; b < count; ++b) {
        if (m[b] < 0) return fail(MHS_EINVAL, "instance %d: m < 0", b);
        eoff[b + 1] = eoff[b] + m[b];
    }
    if (edge_ptr[0] != 0) return fail(MHS_EINVAL, "edge_ptr[0] must be 0");
    if (eoff[count] > 0 && !demand) return fail(MHS_EINVAL, "demand is NULL");
    for (int b = 0; b < count; ++b) {
        const int64_t e0 = eoff[b];
        nnz[b] = edge_ptr[e0 + m[b]] - edge_ptr[e0];
        if (nnz[b] > 0 && !edge_vtx) return fail(MHS_EINVAL, "edge_vtx is NULL");
        if (n[b] < 0) return fail(MHS_EINVAL, "instance %d: n < 0", b);
        if (n[b] >= (1 << 24) || m[b] >= (1 << 24))
            return fail(MHS_EINVAL, "instance %d: n and m must be < 2^24 (exact FP32 counts)", b);
        if (nnz[b] < 0 || nnz[b] >= (1ll << 31))
            return fail(MHS_EINVAL, "instance %d: bad edge_ptr range", b);
    }
    // Every instance is validated against the global pointer array (vertex
    // ids local) on several threads for a large batch, while this thread
    // allocates and copies the inputs; no kernel reads them before the
    // validation has passed.  The lowest failing instance is validated again
    // here for its message.
    auto check = [&](int b, std::vector<int32_t> &mark) {
        char what[64];
        std::snprintf(what, sizeof(what), "instance %d", b);
        if ((size_t)n[b] > mark.size()) mark.resize((size_t)n[b], -1);
        std::fill(mark.begin(), mark.begin() + n[b], -1);
        return validate_host(n[b], m[b], edge_ptr + eoff[b], nullptr, edge_vtx, demand + eoff[b],
                             mark, 0, what, /*quiet=*/true);
    };
    // Page-locked staging in the layout of the arena's input arrays (local
    // int32 offsets, vertex ids, demands, each over the whole batch): every
    // checked instance is converted and copied there by the thread that
    // checked it, and three copies take the batch to the device.  Without it
    // (inputs above 1 GB, or no page-locked memory) this thread converts the
    // offsets and copies from the caller's arrays.
    const int64_t sum_m = eoff[count], sum_m1 = sum_m + count, sum_z = edge_ptr[sum_m];
    const int64_t stage_bytes = 4 * (sum_m1 + sum_z + sum_m);
    size_t stage_cls = 0;
    uint8_t *stage = stage_bytes <= (1ll << 30)
                         ? static_cast<uint8_t *>(pinned_take((size_t)stage_bytes, &stage_cls))
                         : nullptr;
    int32_t *s_ptr = reinterpret_cast<int32_t *>(stage);
    int32_t *s_vtx = stage ? s_ptr + sum_m1 : nullptr;
    int32_t *s_f = stage ? s_vtx + sum_z : nullptr;
    auto to_stage = [&](int b) {
        const int64_t e0 = eoff[b], p0 = edge_ptr[e0];
        int32_t *dp = s_ptr + e0 + b;  // instance b's m[b] + 1 offsets
        for (int32_t i = 0; i <= m[b]; ++i) dp[i] = (int32_t)(edge_ptr[e0 + i] - p0);
        if (nnz[b] > 0) std::memcpy(s_vtx + p0, edge_vtx + p0, 4 * (size_t)nnz[b]);
        if (m[b] > 0) std::memcpy(s_f + e0, demand + e0, 4 * (size_t)m[b]);
    };
    // threads: one per core, up to 16 (none for a small batch)
    const int nt = count >= 64
                       ? (int)std::min<unsigned>(16, std::max(1u, std::thread::hardware_concurrency()))
                       : 1;
    std::atomic<int> first_bad{count};
    auto share = [&](int t) {
        std::vector<int32_t> mark;
        for (int b = t; b < count && b < first_bad.load(); b += nt) {
            if (check(b, mark)) {
                int cur = first_bad.load();
                while (b < cur && !first_bad.compare_exchange_weak(cur, b)) {
                }
            } else if (stage) {
                to_stage(b);
            }
        }
    };
    std::vector<std::thread> threads;
    int started = 1;
    try {
        for (; started < nt; ++started) threads.emplace_back(share, started);
    } catch (...) {  // a thread that cannot start: its share runs here, below
    }
    // joins the checks; the lowest malformed instance's message, else MHS_OK
    auto finish_checks = [&]() {
        for (int t = started; t < nt; ++t) share(t);
        share(0);
        for (std::thread &x : threads) x.join();
        threads.clear();
        const int bad = first_bad.load();
        if (bad >= count) return MHS_OK;
        std::vector<int32_t> mark((size_t)std::max(n[bad], 1), -1);
        char what[64];
        std::snprintf(what, sizeof(what), "instance %d", bad);
        mhs_status st = validate_host(n[bad], m[bad], edge_ptr + eoff[bad], nullptr, edge_vtx,
                                      demand + eoff[bad], mark, 0, what);
        return st ? st : fail(MHS_EINVAL, "%s: malformed", what);
    };
    std::vector<Layout> lay;
    int64_t tmoff = 0;
    mhs_instance *h = nullptr;
    mhs_status st = create(count, n, m, nnz.data(), k, opt, cuda_stream, &h, lay, tmoff);
    if (st) {  // a malformed input is reported first, as a check before the allocation would
        const std::string msg = g_err;
        const mhs_status vst = finish_checks();
        pinned_give(stage, stage_cls);
        if (vst) return vst;
        return fail(st, "%s", msg.c_str());
    }
    if (stage) {  // checked and staged: three copies; the buffer lives as long as the handle
        h->in_stage = stage;
        h->in_stage_cls = stage_cls;
        st = finish_checks();
        if (st) {
            destroy(h);
            return st;
        }
        cudaError_t e = cudaMemcpyAsync(h->arena + h->in_eptr, s_ptr, 4 * (size_t)sum_m1,
                                        cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess && sum_z > 0)
            e = cudaMemcpyAsync(h->arena + h->in_evtx, s_vtx, 4 * (size_t)sum_z,
                                cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess && sum_m > 0)
            e = cudaMemcpyAsync(h->arena + h->in_f, s_f, 4 * (size_t)sum_m,
                                cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) st = finish_load(h, tmoff);
        else st = fail(MHS_ECUDA, "input copy failed: %s", cudaGetErrorString(e));
        if (st == MHS_OK && cudaStreamSynchronize(h->stream) != cudaSuccess)
            st = fail(MHS_ECUDA, "load failed");
        if (st) {
            destroy(h);
            return st;
        }
        *out = h;
        return MHS_OK;
    }
    // one copy per input array: local int32 offsets, vertex ids, demands
    std::vector<int32_t> local_ptr((size_t)h->sum_m1);
    {
        size_t w = 0;
        for (int b = 0; b < count; ++b) {
            const int64_t e0 = eoff[b];
            for (int32_t i = 0; i <= m[b]; ++i)
                local_ptr[w++] = (int32_t)(edge_ptr[e0 + i] - edge_ptr[e0]);
        }
    }
    cudaError_t e = cudaMemcpyAsync(h->arena + h->in_eptr, local_ptr.data(), 4 * local_ptr.size(),
                                    cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && h->sum_nnz > 0)
        e = cudaMemcpyAsync(h->arena + h->in_evtx, edge_vtx, 4 * (size_t)h->sum_nnz,
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && h->sum_m > 0)
        e = cudaMemcpyAsync(h->arena + h->in_f, demand, 4 * (size_t)h->sum_m,
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // local_ptr is pageable
    st = finish_checks();
    if (st) {
        destroy(h);
        return st;
    }
    if (e != cudaSuccess) {
        destroy(h);
        return fail(MHS_ECUDA, "input copy failed: %s", cudaGetErrorString(e));
    }
    st = finish_load(h, tmoff);
    if (st == MHS_OK && cudaStreamSynchronize(h->stream) != cudaSuccess)
        st = fail(MHS_ECUDA, "load failed");
    if (st) {
        destroy(h);
        return st;
    }
    *out = h;
    return MHS_OK;
}

mhs_status mhs_load_batch_device(int32_t count, const int32_t *n, const int32_t *m,
                                 const int64_t *edge_ptr, const int32_t *edge_vtx,
                                 const int32_t *demand, const int64_t *k,
                                 const mhs_options *opt, void *cuda_stream, mhs_instance **out) {
    if (!out) return fail(MHS_EINVAL, "out is NULL");
    *out = nullptr;
    // kernels index the instances of a batch by blockIdx.y
    if (count < 1 || count > 65535) return fail(MHS_EINVAL, "count must be in [1, 65535]");
    if (!n || !m || !edge_ptr || !k) return fail(MHS_EINVAL, "NULL input array");
    std::vector<int64_t> eoff(count + 1, 0);
    for (int b = 0; b < count; ++b) {
        if (n[b] < 0 || m[b] < 0) return fail(MHS_EINVAL, "instance %d: n or m < 0", b);
        if (n[b] >= (1 << 24) || m[b] >= (1 << 24))
            return fail(MHS_EINVAL, "instance %d: n and m must be < 2^24", b);
        eoff[b + 1] = eoff[b] + m[b];
    }
    if (eoff[count] > 0 && !demand) return fail(MHS_EINVAL, "demand is NULL");
    cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
    // instance boundaries in the device CSR: gather edge_ptr[eoff[b]]
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    CUDA_TRY(pool_for(dev, &pool));
    int64_t *tmp = nullptr;
    // [0, count]: hyperedge offsets; [count + 1, 2 count + 1]: their CSR
    // positions; then the OR of the validation statuses
    CUDA_TRY(cudaMallocFromPoolAsync(reinterpret_cast<void **>(&tmp),
                                     sizeof(int64_t) * (2 * ((size_t)count + 1) + 1), pool, cs));
    std::vector<int64_t> bounds(count + 1);
    cudaError_t e = cudaMemcpyAsync(tmp, eoff.data(), sizeof(int64_t) * (count + 1),
                                    cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = launch_gather_bounds(edge_ptr, tmp, tmp + count + 1, count, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bounds.data(), tmp + count + 1, sizeof(int64_t) * (count + 1),
                            cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        cudaFreeAsync(tmp, cs);
        return fail(MHS_ECUDA, "batch bounds: %s", cudaGetErrorString(e));
    }
    std::vector<int64_t> nnz(count);
    for (int b = 0; b < count; ++b) {
        nnz[b] = bounds[b + 1] - bounds[b];
        if (nnz[b] < 0 || nnz[b] >= (1ll << 31)) {
            cudaFreeAsync(tmp, cs);
            return fail(MHS_EINVAL, "instance %d: bad edge_ptr range", b);
        }
    }
    if (bounds[0] != 0) {
        cudaFreeAsync(tmp, cs);
        return fail(MHS_EINVAL, "edge_ptr[0] must be 0");
    }
    const int64_t total_nnz = bounds[count];
    if (total_nnz > 0 && !edge_vtx) {
        cudaFreeAsync(tmp, cs);
        return fail(MHS_EINVAL, "edge_vtx is NULL");
    }
    std::vector<Layout> lay;
    int64_t tmoff = 0;
    mhs_instance *h = nullptr;
    mhs_status st = create(count, n, m, nnz.data(), k, opt, cuda_stream, &h, lay, tmoff);
    if (st) {
        cudaFreeAsync(tmp, cs);
        return st;
    }
    // device-to-device: vertex ids and demands in one copy each, local offsets by a kernel
    e = cudaSuccess;
    if (h->sum_nnz > 0)
        e = cudaMemcpyAsync(h->arena + h->in_evtx, edge_vtx, 4 * (size_t)h->sum_nnz,
                            cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && h->sum_m > 0)
        e = cudaMemcpyAsync(h->arena + h->in_f, demand, 4 * (size_t)h->sum_m,
                            cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = upload_states(h);
    if (e == cudaSuccess) e = launch_localize_ptr(h->dstate, count, edge_ptr, tmp, h->stream);
    if (e == cudaSuccess) e = launch_validate(h->dstate, count, h->stream);
    int32_t *any_status = reinterpret_cast<int32_t *>(tmp + 2 * ((int64_t)count + 1));
    int32_t hany = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(any_status, 0, sizeof(int32_t), h->stream);
    if (e == cudaSuccess) e = launch_status_or(h->dstate, count, any_status, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&hany, any_status, sizeof(int32_t), cudaMemcpyDeviceToHost,
                            h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFreeAsync(tmp, h->stream);
    if (e != cudaSuccess) {
        destroy(h);
        return fail(MHS_ECUDA, "batch device load: %s", cudaGetErrorString(e));
    }
    if (hany) {  // some instance is malformed: read the states to name the first
        std::vector<InstState> chk(count);
        e = cudaMemcpyAsync(chk.data(), h->dstate, sizeof(InstState) * count,
                            cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        for (int b = 0; e == cudaSuccess && b < count; ++b)
            if (chk[b].status) {
                const int32_t sv = chk[b].status;
                destroy(h);
                return fail(MHS_EINVAL, "instance %d malformed (status 0x%x: %s)", b, sv,
                            status_text(sv));
            }
        destroy(h);
        return fail(MHS_ECUDA, "batch device load: %s",
                    e != cudaSuccess ? cudaGetErrorString(e) : "status read back inconsistent");
    }
    st = finish_load(h, tmoff);
    if (st == MHS_OK && cudaStreamSynchronize(h->stream) != cudaSuccess)
        st = fail(MHS_ECUDA, "load failed");
    if (st) {
        destroy(h);
        return st;
    }
    *out = h;
    return MHS_OK;
}

int32_t mhs_count(const mhs_instance *inst) { return inst ? inst->count : 0; }

mhs_status mhs_reduce_round(mhs_instance *inst, mhs_round_stats *stats) {
    if (!inst) return fail(MHS_EINVAL, "instance is NULL");
    const mhs_status st = run_rounds(inst, 1, stats);
    if (st) inst->faulted = true;  // a round may have stopped half way
    return st;
}

mhs_status mhs_kernelize(mhs_instance *inst, mhs_round_stats *stats) {
    if (!inst) return fail(MHS_EINVAL, "instance is NULL");
    const mhs_status st = run_rounds(inst, 0, stats);
    if (st) inst->faulted = true;
    return st;
}

// ---- sharded passes ------------------------------------------------------

namespace {
mhs_status pass_check(const mhs_instance *h, int32_t phase, bool open) {
    if (!h) return fail(MHS_EINVAL, "instance is NULL");
    if (h->count != 1) return fail(MHS_EINVAL, "sharded passes take a single instance");
    if (phase != 0 && phase != 1) return fail(MHS_EINVAL, "phase must be 0 (DP/SE) or 1 (MD)");
    const int32_t want = open ? (phase == 0 ? 1 : 3) : (phase == 0 ? 0 : 2);
    if (h->pass_state != want)
        return fail(MHS_EINVAL,
                    "passes run in order: begin(0), contract(0)..., end(0), begin(1), "
                    "contract(1)..., end(1) (state %d, phase %d)",
                    h->pass_state, phase);
    return MHS_OK;
}
}  // namespace

mhs_status mhs_pass_begin(mhs_instance *inst, int32_t phase) {
    mhs_status st = pass_check(inst, phase, false);
    if (st) return st;
    if (inst->opt.full_edges && inst->opt.max_rounds)
        return fail(MHS_EINVAL, "full_edges needs max_rounds = 0");
    CUDA_TRY(launch_phase_prologue(inst->dstate, inst->dplan, inst->dctr, phase, inst->contraction,
                                   inst->sms, inst->stream));
    inst->pass_state = phase == 0 ? 1 : 3;
    return MHS_OK;
}

mhs_status mhs_pass_contract(mhs_instance *inst, int32_t phase, int32_t shard, int32_t nshards) {
    mhs_status st = pass_check(inst, phase, true);
    if (st) return st;
    if (nshards < 1 || nshards > 4096 || shard < 0 || shard >= nshards)
        return fail(MHS_EINVAL, "need 1 <= nshards <= 4096 and 0 <= shard < nshards");
    CUDA_TRY(launch_phase_contract(inst->dstate, inst->dplan, inst->dctr, phase,
                                   inst->contraction, inst->sms, inst->dkerr, inst->stream,
                                   inst->tiles.tile_n, shard, nshards));
    return MHS_OK;
}

mhs_status mhs_pass_partial(const mhs_instance *inst, int32_t phase, void *dev_out,
                            int64_t *elems_out) {
    mhs_status st = pass_check(inst, phase, true);
    if (st) return st;
    const InstState &s = inst->hstate[0];
    const int64_t elems = phase == 0 ? s.m0 : s.n0;
    if (elems_out) *elems_out = elems;
    if (dev_out && elems > 0) {
        CUDA_TRY(launch_pass_exchange(inst->dstate, phase, 0, dev_out, inst->sms, inst->stream));
        CUDA_TRY(cudaStreamSynchronize(inst->stream));
    }
    return MHS_OK;
}

mhs_status mhs_pass_merge(mhs_instance *inst, int32_t phase, const void *dev_in) {
    mhs_status st = pass_check(inst, phase, true);
    if (st) return st;
    if (!dev_in) return fail(MHS_EINVAL, "dev_in is NULL");
    const InstState &s = inst->hstate[0];
    const int64_t elems = phase == 0 ? s.m0 : s.n0;
    if (elems > 0) {
        CUDA_TRY(launch_pass_exchange(inst->dstate, phase, 1, const_cast<void *>(dev_in),
                                      inst->sms, inst->stream));
        CUDA_TRY(cudaStreamSynchronize(inst->stream));
    }
    return MHS_OK;
}

mhs_status mhs_pass_end(mhs_instance *inst, int32_t phase, mhs_round_stats *stats) {
    mhs_status st = pass_check(inst, phase, true);
    if (st) return st;
    cudaError_t e = launch_phase_epilogue(inst->dstate, inst->dplan, inst->dctr, 1, phase,
                                          inst->contraction, inst->sms, inst->stream, nullptr,
                                          inst->compact_blocks);
    if (e == cudaSuccess && phase == 1 && inst->opt.full_edges)
        e = launch_full_edges(inst->dstate, 1, inst->dctr, nullptr, inst->sms, inst->stream);
    if (e != cudaSuccess) {
        inst->faulted = true;
        return fail(MHS_ECUDA, "pass end: %s", cudaGetErrorString(e));
    }
    inst->pass_state = phase == 0 ? 2 : 0;
    if (phase == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return MHS_OK;
    }
    CUDA_TRY(cudaMemcpyAsync(inst->hctr, inst->dctr, sizeof(BatchCounters), cudaMemcpyDeviceToHost,
                             inst->stream));
    CUDA_TRY(cudaMemcpyAsync(inst->hkerr, inst->dkerr, sizeof(int32_t), cudaMemcpyDeviceToHost,
                             inst->stream));
    CUDA_TRY(cudaStreamSynchronize(inst->stream));
    st = check_device_status(inst);
    if (st) return st;
    if (stats) {
        stats->n_alive = inst->hctr->n_alive;
        stats->m_alive = inst->hctr->m_alive;
        stats->rounds = inst->hctr->max_rounds_seen;
        stats->changed = inst->hctr->changed_any;
        stats->dp_deleted = inst->hctr->dp_deleted;
        stats->md_deleted = inst->hctr->md_deleted;
        stats->active = inst->hctr->active;
    }
    return MHS_OK;
}

mhs_status mhs_result_at(const mhs_instance *inst, int32_t index, int32_t *vtx_out,
                         int32_t vtx_cap, int32_t *n_out, int32_t *edge_out, int32_t *demand_out,
                         int32_t edge_cap, int32_t *m_out, int64_t *k_out, int32_t *rounds_out) {
    if (!inst) return fail(MHS_EINVAL, "instance is NULL");
    if (index < 0 || index >= inst->count) return fail(MHS_EINVAL, "index out of range");
    InstState s;
    cudaStream_t cs = inst->stream;
    CUDA_TRY(cudaMemcpyAsync(&s, inst->dstate + index, sizeof(s), cudaMemcpyDeviceToHost, cs));
    CUDA_TRY(cudaStreamSynchronize(cs));
    if (n_out) *n_out = s.n;
    if (m_out) *m_out = s.m;
    if (k_out) *k_out = s.k;
    if (rounds_out) *rounds_out = s.rounds;
    if (s.status) return fail(MHS_EDEVICE, "instance %d error status 0x%x", index, s.status);
    if ((vtx_out && vtx_cap < s.n) || ((edge_out || demand_out) && edge_cap < s.m))
        return fail(MHS_EINVAL, "output capacity too small (need %d vertices, %d edges)", s.n,
                    s.m);
    if (vtx_out && s.n > 0)
        CUDA_TRY(cudaMemcpyAsync(vtx_out, s.v_c2o, 4 * (size_t)s.n, cudaMemcpyDeviceToHost, cs));
    std::vector<int32_t> eids;
    int32_t *eo = edge_out;
    if (!eo && demand_out) {
        eids.resize(std::max(s.m, 1));
        eo = eids.data();
    }
    if (eo && s.m > 0)
        CUDA_TRY(cudaMemcpyAsync(eo, s.e_c2o, 4 * (size_t)s.m, cudaMemcpyDeviceToHost, cs));
    std::vector<int32_t> f;
    if (demand_out && s.m > 0) {
        f.resize(s.m0);
        CUDA_TRY(cudaMemcpyAsync(f.data(), s.f, 4 * (size_t)s.m0, cudaMemcpyDeviceToHost, cs));
    }
    CUDA_TRY(cudaStreamSynchronize(cs));
    // positions are in layout order: report input ids ascending
    if (vtx_out) std::sort(vtx_out, vtx_out + s.n);
    if (eo) std::sort(eo, eo + s.m);
    if (demand_out)
        for (int32_t i = 0; i < s.m; ++i) demand_out[i] = f[eo[i]];
    return MHS_OK;
}

mhs_status mhs_forced_at(const mhs_instance *inst, int32_t index, int32_t *vtx_out, int32_t cap,
                         int32_t *count_out, int32_t *fe_passes_out) {
    if (!inst) return fail(MHS_EINVAL, "instance is NULL");
    if (index < 0 || index >= inst->count) return fail(MHS_EINVAL, "index out of range");
    InstState s;
    cudaStream_t cs = inst->stream;
    CUDA_TRY(cudaMemcpyAsync(&s, inst->dstate + index, sizeof(s), cudaMemcpyDeviceToHost, cs));
    CUDA_TRY(cudaStreamSynchronize(cs));
    if (fe_passes_out) *fe_passes_out = s.fe_passes;
    std::vector<uint8_t> flags;
    if (s.forced && s.n0 > 0) {
        flags.resize(s.n0);
        CUDA_TRY(cudaMemcpyAsync(flags.data(), s.forced, (size_t)s.n0, cudaMemcpyDeviceToHost, cs));
        CUDA_TRY(cudaStreamSynchronize(cs));
    }
    int32_t c = 0;
    for (uint8_t x : flags) c += x != 0;
    if (count_out) *count_out = c;
    if (!vtx_out) return MHS_OK;
    if (cap < c) return fail(MHS_EINVAL, "output capacity too small (need %d vertices)", c);
    int32_t w = 0;
    for (int32_t v = 0; v < (int32_t)flags.size(); ++v)
        if (flags[v]) vtx_out[w++] = v;
    return MHS_OK;
}

mhs_status mhs_result(const mhs_instance *inst, int32_t *vtx_out, int32_t vtx_cap, int32_t *n_out,
                      int32_t *edge_out, int32_t *demand_out, int32_t edge_cap, int32_t *m_out,
                      int64_t *k_out, int32_t *rounds_out) {
    return mhs_result_at(inst, 0, vtx_out, vtx_cap, n_out, edge_out, demand_out, edge_cap, m_out,
                         k_out, rounds_out);
}

mhs_status mhs_result_device(const mhs_instance *inst, int32_t index, uint8_t *alive_v,
                             uint8_t *alive_e) {
    if (!inst) return fail(MHS_EINVAL, "instance is NULL");
    if (index < 0 || index >= inst->count) return fail(MHS_EINVAL, "index out of range");
    if (!alive_v || !alive_e) return fail(MHS_EINVAL, "NULL output");
    CUDA_TRY(launch_alive_masks(inst->dstate + index, alive_v, alive_e, inst->stream));
    return MHS_OK;
}

mhs_status mhs_result_batch_device(const mhs_instance *inst, uint8_t *alive_v,
                                   uint8_t *alive_e) {
    if (!inst) return fail(MHS_EINVAL, "instance is NULL");
    if (!alive_v || !alive_e) return fail(MHS_EINVAL, "NULL output");
    CUDA_TRY(launch_alive_masks_batch(inst->dstate, inst->count, alive_v, alive_e, inst->stream));
    return MHS_OK;
}

mhs_status mhs_trace_at(const mhs_instance *inst, int32_t index, int32_t *rows_out,
                        int32_t cap_rounds, int32_t *rounds_out) {
    if (!inst) return fail(MHS_EINVAL, "instance is NULL");
    if (index < 0 || index >= inst->count) return fail(MHS_EINVAL, "index out of range");
    InstState s;
    CUDA_TRY(cudaMemcpyAsync(&s, inst->dstate + index, sizeof(s), cudaMemcpyDeviceToHost,
                             inst->stream));
    CUDA_TRY(cudaStreamSynchronize(inst->stream));
    if (rounds_out) *rounds_out = s.rounds;
    const int32_t nr = std::min(std::min(s.rounds, cap_rounds), (int32_t)kTraceRounds);
    if (rows_out)
        for (int32_t r = 0; r < nr; ++r)
            for (int c = 0; c < 3; ++c) rows_out[3 * r + c] = s.trace[r][c];
    return MHS_OK;
}

mhs_status mhs_export(const mhs_instance *inst, int32_t index, int32_t *edge_ptr_out,
                      int32_t edge_cap, int32_t *edge_vtx_out, int64_t nnz_cap,
                      int32_t *demand_out, int32_t *n_out, int32_t *m_out, int64_t *nnz_out) {
    if (!inst) return fail(MHS_EINVAL, "instance is NULL");
    if (index < 0 || index >= inst->count) return fail(MHS_EINVAL, "index out of range");
    InstState s;
    cudaStream_t cs = inst->stream;
    CUDA_TRY(cudaMemcpyAsync(&s, inst->dstate + index, sizeof(s), cudaMemcpyDeviceToHost, cs));
    CUDA_TRY(cudaStreamSynchronize(cs));
    std::vector<int32_t> eptr(s.m0 + 1), evtx(std::max<int64_t>(s.nnz0, 1)), f(std::max(s.m0, 1)),
        vmap(std::max(s.n0, 1)), ec2o(std::max(s.m, 1));
    CUDA_TRY(cudaMemcpyAsync(eptr.data(), s.eptr, 4 * ((size_t)s.m0 + 1), cudaMemcpyDeviceToHost, cs));
    if (s.nnz0 > 0)
        CUDA_TRY(cudaMemcpyAsync(evtx.data(), s.evtx, 4 * (size_t)s.nnz0, cudaMemcpyDeviceToHost, cs));
    if (s.m0 > 0)
        CUDA_TRY(cudaMemcpyAsync(f.data(), s.f, 4 * (size_t)s.m0, cudaMemcpyDeviceToHost, cs));
    if (s.n0 > 0)
        CUDA_TRY(cudaMemcpyAsync(vmap.data(), s.v_o2c, 4 * (size_t)s.n0, cudaMemcpyDeviceToHost, cs));
    if (s.m > 0)
        CUDA_TRY(cudaMemcpyAsync(ec2o.data(), s.e_c2o, 4 * (size_t)s.m, cudaMemcpyDeviceToHost, cs));
    CUDA_TRY(cudaStreamSynchronize(cs));
    // renumber in input order: vertex v -> number of surviving vertices before it
    std::sort(ec2o.begin(), ec2o.begin() + s.m);
    {
        int32_t next = 0;
        for (int32_t v = 0; v < s.n0; ++v) vmap[v] = vmap[v] >= 0 ? next++ : -1;
    }
    int64_t nnz = 0;
    for (int32_t i = 0; i < s.m; ++i) {
        const int32_t e = ec2o[i];
        for (int32_t p = eptr[e]; p < eptr[e + 1]; ++p) nnz += vmap[evtx[p]] >= 0;
    }
    if (n_out) *n_out = s.n;
    if (m_out) *m_out = s.m;
    if (nnz_out) *nnz_out = nnz;
    if (!edge_ptr_out && !edge_vtx_out && !demand_out) return MHS_OK;
    if (edge_cap < s.m || nnz_cap < nnz)
        return fail(MHS_EINVAL, "export capacity too small (need %d edges, %lld incidences)", s.m,
                    (long long)nnz);
    int64_t w = 0;
    if (edge_ptr_out) edge_ptr_out[0] = 0;
    for (int32_t i = 0; i < s.m; ++i) {
        const int32_t e = ec2o[i];
        for (int32_t p = eptr[e]; p < eptr[e + 1]; ++p) {
            const int32_t c = vmap[evtx[p]];
            if (c >= 0) {
                if (edge_vtx_out) edge_vtx_out[w] = c;
                ++w;
            }
        }
        if (edge_ptr_out) edge_ptr_out[i + 1] = (int32_t)w;
        if (demand_out) demand_out[i] = f[e];
    }
    return MHS_OK;
}

mhs_status mhs_work_stats(const mhs_instance *inst, int64_t *mma_kblocks, int64_t *mma_tiles) {
    if (!inst) return fail(MHS_EINVAL, "instance is NULL");
    BatchCounters c;
    CUDA_TRY(cudaMemcpyAsync(&c, inst->dctr, sizeof(c), cudaMemcpyDeviceToHost, inst->stream));
    CUDA_TRY(cudaStreamSynchronize(inst->stream));
    if (mma_kblocks) *mma_kblocks = (int64_t)c.mma_kblocks;
    if (mma_tiles) *mma_tiles = (int64_t)c.mma_tiles;
    return MHS_OK;
}

mhs_status mhs_tile_config(const mhs_instance *inst, int32_t *tile_n, int32_t *group_rows,
                           int32_t *half_stages, int32_t *from_table) {
    if (!inst) return fail(MHS_EINVAL, "instance is NULL");
    if (tile_n) *tile_n = inst->tiles.tile_n;
    if (group_rows) *group_rows = inst->tiles.group_rows;
    if (half_stages) *half_stages = inst->tiles.half_stages;
    if (from_table) *from_table = inst->tiles.from_table;
    return MHS_OK;
}

mhs_status mhs_set_timing(mhs_instance *inst, int32_t enable) {
    if (!inst) return fail(MHS_EINVAL, "instance is NULL");
    inst->timing = enable != 0;
    return MHS_OK;
}

mhs_status mhs_last_timing(const mhs_instance *inst, float *ms4) {
    if (!inst || !ms4) return fail(MHS_EINVAL, "NULL argument");
    std::memcpy(ms4, inst->last_ms, sizeof(inst->last_ms));
    return MHS_OK;
}

void mhs_free(mhs_instance *inst) { destroy(inst); }

const char *mhs_last_error(void) { return g_err.c_str(); }

const char *mhs_version(void) { return "mhs-gb300 0.1 (sm_103a)"; }

}  // extern "C"

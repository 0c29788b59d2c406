// server.cpp -- continuous-batching server: mhs_server_create / mhs_submit /
// mhs_poll / mhs_server_destroy.
//
// The request loop runs on the device.  Each lane's loop is one CUDA graph
// whose conditional WHILE node repeats, with no host step in between:
//   1. admission: every slot whose (host-mapped) ready flag is set enters
//      the live slot table;
//   2. ONE round of Algorithm 3 (DP then MD) for every live slot at once;
//   3. retirement: the slots whose instance reached its fixpoint (or
//      failed) leave the live table, their state is kept for the host and
//      their index is published in a host-mapped ring;
// until the host asks it to stop or no slot is live or ready, when the
// graph ends and the host launches it again once there is work.
// The lane's host thread only moves data: it loads each admitted request
// into a free slot's arena on a stream of its own (inputs, tensor maps, the
// build kernels, the staged state), waits for that to finish and then sets
// the slot's ready flag; it takes the slots published in the ring, copies
// their results out, returns their arenas to the pool and wakes the pollers.
// Admission is by HBM footprint, at the host, before a request is loaded.
// Requests that arrive while others are on the GPU join at the next round
// boundary, so work of different sizes overlaps in the same launches.
// Requests are split by size into two lanes, each with its own slot table,
// device loop, host thread and streams: small instances are
// batched by the hundreds on a high-priority stream, large ones (which fill
// the GPU on their own) run a few at a time on the other, so a small
// request never waits for the rounds of a large one.  The HBM budget, the
// queue limit and the tickets are shared.
// The result of an instance does not depend on what else is in flight:
// instances share no state, and every per-instance quantity lives in the
// instance's own arena.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host_internal.h"
#include "kernels.h"
#include "mhs.h"
#include "mhs_internal.h"

using namespace mhs;

namespace {

inline int64_t up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline int64_t kbytes(int64_t K) { return up(K > 0 ? K : 1, kTcK); }
inline int64_t kwords(int64_t K) { return up(((K + 31) / 32) > 0 ? (K + 31) / 32 : 1, 4); }
inline int64_t occ_words(int64_t K) { return (kbytes(K) / kOccK + 31) / 32; }
constexpr int64_t kServerListCap = 16 << 20;  // tile-list entries shared by the slots
// Iterations of one launch of a lane's loop at most (it also ends when idle);
// the host launches it again while there is work.
constexpr int32_t kLoopIters = 1 << 16;
inline int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    uint64_t ticket = 0;
    int32_t n = 0, m = 0;
    int64_t k = 0;
    std::vector<int32_t> ptr, vtx, dem;
    int64_t footprint = 0;
    int64_t tiles = 0;  // most tile-list entries one of its phases can need
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    bool done = false;
    mhs_status status = MHS_OK;
    std::vector<int32_t> vout, eout, dout, forced;
    int32_t rounds = 0;
};

// Device layout of one admitted instance inside its arena.
struct Layout {
    int64_t eptr, evtx, f, v_o2c, v_c2o, e_o2c, e_c2o, e_f, e_s, v_deg, v_maxf, v_cnt, e_del,
        v_del, forced, v_dirty, e_dirty_rb, v_dirty_rb, e_prev, e_rec, occ0, occ1, tmaps, dense,
        dense_bytes, bytes;
};

Layout plan_layout(int32_t n, int32_t m, int64_t nnz, bool dense, bool fe) {
    Layout L;
    int64_t b = 0;
    auto take = [&b](int64_t x) {
        int64_t o = b;
        b += up(x > 0 ? x : 1, 256);
        return o;
    };
    L.eptr = take(4 * ((int64_t)m + 1));
    L.evtx = take(4 * nnz);
    L.f = take(4 * (int64_t)m);
    L.v_o2c = take(4 * (int64_t)n);
    L.v_c2o = take(4 * (int64_t)n);
    L.e_o2c = take(4 * (int64_t)m);
    L.e_c2o = take(4 * (int64_t)m);
    L.e_f = take(4 * (int64_t)m);
    L.e_s = take(4 * (int64_t)m);
    L.v_deg = take(4 * ((int64_t)n + 1));
    L.v_maxf = take(4 * (int64_t)n);
    L.v_cnt = take(4 * ((int64_t)n + 1));
    L.e_del = take(m);
    L.v_del = take(n);
    L.forced = fe ? take(n) : -1;
    L.v_dirty = take(n);
    L.e_prev = take(4 * (int64_t)m);
    L.e_rec = dense ? take(16 * (int64_t)m) : -1;
    L.e_dirty_rb = take(up(m > 0 ? m : 1, kRowAlign) / kTcM);
    L.v_dirty_rb = take(up(n > 0 ? n : 1, kRowAlign) / kTcM);
    {
        const int64_t arows = up(m > 0 ? m : 1, kRowAlign), atrows = up(n > 0 ? n : 1, kRowAlign);
        L.occ0 = take(dense ? 4 * (arows / kTcM) * occ_words(n) : 0);
        L.occ1 = take(dense ? 4 * (atrows / kTcM) * occ_words(m) : 0);
    }
    L.tmaps = take(dense ? 2 * (int64_t)tmap_bytes() : 0);
    L.dense = b;
    const int64_t arows = up(m > 0 ? m : 1, kRowAlign), atrows = up(n > 0 ? n : 1, kRowAlign);
    if (dense) {
        take(arows * kbytes(n));
        take(atrows * kbytes(m));
    } else {
        take(arows * kwords(n) * 4);
        take(atrows * kwords(m) * 4);
    }
    L.dense_bytes = b - L.dense;
    L.bytes = b;
    return L;
}

struct Slot {
    bool busy = false;
    std::shared_ptr<Request> req;
    uint8_t *arena = nullptr;
    int64_t bytes = 0;
    int64_t tiles = 0;
};

}  // namespace

struct Lane {
    int id = 0;
    mhs_server *S = nullptr;
    cudaStream_t stream = nullptr;  // the loop
    bool own_stream = false;
    cudaStream_t load = nullptr;    // uploads and result copies, beside the loop
    int32_t slots_n = 0;
    // device slot table and loop bookkeeping (one allocation)
    uint8_t *ctl = nullptr;
    InstState *dstate = nullptr;    // the live slot table (written by the loop only)
    InstState *dstage = nullptr;    // states the host has loaded, before they enter
    InstState *dout = nullptr;      // states of retired slots, for the host
    Plan *dplan = nullptr;
    BatchCounters *dctr = nullptr;
    ServerDev *ddev = nullptr;
    int32_t *dkerr = nullptr, *ddone = nullptr;
    // host-mapped page-locked block: flags, ready[slots], ring[slots]
    uint8_t *mapped = nullptr;
    ServerFlags *hflags = nullptr, *dflags = nullptr;
    int32_t *hready = nullptr, *dready = nullptr;
    int32_t *hring = nullptr, *dring = nullptr;
    uint32_t consumed = 0;          // ring entries taken by the host (wraps with the head)
    bool running = false;           // a launch of the loop may still run
    uint8_t *hmaps = nullptr;       // pinned: 2 tensor maps per slot, staged for upload
    InstState *hstates = nullptr;   // pinned: states of the slots retired at once
    cudaGraphExec_t graph = nullptr;
    int64_t list_cap = 0;
    std::vector<Slot> slots;                         // owned by the lane's worker
    std::deque<std::shared_ptr<Request>> pending;    // guarded by S->mu
    int32_t active_count = 0;                        // guarded by S->mu
    int64_t tiles_in_use = 0;                        // guarded by S->mu
    int64_t in_use_release = 0, tiles_release = 0;   // worker-local
    std::condition_variable cv_work;
    std::thread worker;
};

struct mhs_server {
    mhs_server_options opt{};
    int contraction = kFp8;
    int device = 0, sms = 0;
    cudaMemPool_t pool = nullptr;
    int64_t small_items = 0;  // n + m at most for the small-request lane
    Lane lanes[2];
    // shared state
    std::mutex mu;
    std::condition_variable cv_done;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> table;
    uint64_t next_ticket = 1;
    bool stop = false, paused = false;
    mhs_status fatal = MHS_OK;
    int64_t in_use = 0, peak = 0;
    int64_t submitted = 0, admitted = 0, completed = 0;
};

namespace {

// Upload and initialise one request into slot `si` (worker thread only).
mhs_status admit(Lane &Ln, int si, std::shared_ptr<Request> req) {
    mhs_server *S = Ln.S;
    const bool dense = S->contraction == kFp8;
    const int64_t nnz = req->ptr.empty() ? 0 : req->ptr.back();
    const bool fe = S->opt.full_edges != 0;
    Layout L = plan_layout(req->n, req->m, nnz, dense, fe);
    uint8_t *a = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&a), (size_t)L.bytes, S->pool,
                                            Ln.load);
    if (e != cudaSuccess) return set_error(MHS_ENOMEM, "server: arena allocation failed");
    InstState s;
    std::memset(&s, 0, sizeof(s));
    s.n0 = req->n;
    s.m0 = req->m;
    s.nnz0 = nnz;
    s.k = req->k;
    s.layout_sorted = layout_code(S->opt.layout);
    s.no_skip = S->opt.sparsity == MHS_SPARSITY_DENSE;
    s.edge_rule = S->opt.edge_rule;
    s.full_edges = S->opt.full_edges;
    s.forced = fe ? a + L.forced : nullptr;
    s.v_dirty = a + L.v_dirty;
    s.e_prev = reinterpret_cast<int32_t *>(a + L.e_prev);
    s.e_rec = L.e_rec >= 0 ? reinterpret_cast<int4 *>(a + L.e_rec) : nullptr;
    s.e_dirty_rb = a + L.e_dirty_rb;
    s.v_dirty_rb = a + L.v_dirty_rb;
    s.eptr = reinterpret_cast<int32_t *>(a + L.eptr);
    s.evtx = reinterpret_cast<int32_t *>(a + L.evtx);
    s.f = reinterpret_cast<int32_t *>(a + L.f);
    s.v_o2c = reinterpret_cast<int32_t *>(a + L.v_o2c);
    s.v_c2o = reinterpret_cast<int32_t *>(a + L.v_c2o);
    s.e_o2c = reinterpret_cast<int32_t *>(a + L.e_o2c);
    s.e_c2o = reinterpret_cast<int32_t *>(a + L.e_c2o);
    s.e_f = reinterpret_cast<int32_t *>(a + L.e_f);
    s.e_s = reinterpret_cast<int32_t *>(a + L.e_s);
    s.v_deg = reinterpret_cast<int32_t *>(a + L.v_deg);
    s.v_maxf = reinterpret_cast<int32_t *>(a + L.v_maxf);
    s.v_cnt = reinterpret_cast<int32_t *>(a + L.v_cnt);
    s.e_del = a + L.e_del;
    s.v_del = a + L.v_del;
    const int64_t arows = up(req->m > 0 ? req->m : 1, kRowAlign);
    const int64_t atrows = up(req->n > 0 ? req->n : 1, kRowAlign);
    s.A_rows = (int32_t)arows;
    s.At_rows = (int32_t)atrows;
    uint8_t *maps = Ln.hmaps + (size_t)si * 2 * tmap_bytes();
    if (dense) {
        s.occ[0] = reinterpret_cast<uint32_t *>(a + L.occ0);
        s.occ[1] = reinterpret_cast<uint32_t *>(a + L.occ1);
        s.occ_words[0] = (int32_t)occ_words(req->n);
        s.occ_words[1] = (int32_t)occ_words(req->m);
        s.A = a + L.dense;
        s.At = s.A + arows * kbytes(req->n);
        s.A_pitch = kbytes(req->n);
        s.At_pitch = kbytes(req->m);
        s.tmap_A = a + L.tmaps;
        s.tmap_At = a + L.tmaps + tmap_bytes();
        if (!make_operand_tmap(maps, s.A, s.A_pitch, s.A_rows) ||
            !make_operand_tmap(maps + tmap_bytes(), s.At, s.At_pitch, s.At_rows)) {
            cudaFreeAsync(a, Ln.load);
            return set_error(MHS_ECUDA, "server: tensor map encoding failed");
        }
    } else {
        s.Ab = reinterpret_cast<uint32_t *>(a + L.dense);
        s.Atb = s.Ab + arows * kwords(req->n);
        s.Ab_pitch = (int32_t)kwords(req->n);
        s.Atb_pitch = (int32_t)kwords(req->m);
    }
    // On the load stream, into the slot's staged state (the loop takes it
    // once the ready flag is set, after this work has finished).  Pageable
    // sources: each copy has staged its source when it returns.
    e = cudaMemcpyAsync(a + L.eptr, req->ptr.data(), 4 * req->ptr.size(), cudaMemcpyHostToDevice,
                        Ln.load);
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpyAsync(a + L.evtx, req->vtx.data(), 4 * (size_t)nnz, cudaMemcpyHostToDevice,
                            Ln.load);
    if (e == cudaSuccess && req->m > 0)
        e = cudaMemcpyAsync(a + L.f, req->dem.data(), 4 * (size_t)req->m, cudaMemcpyHostToDevice,
                            Ln.load);
    if (e == cudaSuccess && dense)
        e = cudaMemcpyAsync(a + L.tmaps, maps, 2 * tmap_bytes(), cudaMemcpyHostToDevice, Ln.load);
    if (e == cudaSuccess) e = cudaMemsetAsync(a + L.dense, 0, (size_t)L.dense_bytes, Ln.load);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(Ln.dstage + si, &s, sizeof(s), cudaMemcpyHostToDevice, Ln.load);
    if (e == cudaSuccess) e = launch_build(Ln.dstage + si, 1, 0, nnz, req->m, req->n, Ln.load);
    if (e != cudaSuccess) {
        cudaFreeAsync(a, Ln.load);
        return set_error(MHS_ECUDA, "server: admission failed: %s", cudaGetErrorString(e));
    }
    Slot &sl = Ln.slots[si];
    sl.busy = true;
    sl.req = std::move(req);
    sl.arena = a;
    sl.bytes = L.bytes;
    sl.tiles = sl.req->tiles;
    std::lock_guard<std::mutex> lk(S->mu);
    ++Ln.active_count;
    return MHS_OK;
}

// Fail every request that has not finished (device error or shutdown).
void fail_all_locked(mhs_server *S, mhs_status st) {
    const int64_t t = now_ns();
    for (auto &kv : S->table) {
        Request &r = *kv.second;
        if (!r.done) {
            r.status = st;
            r.done = true;
            r.t_done = t;
        }
    }
    for (auto &ln : S->lanes) {
        ln.pending.clear();
        ln.active_count = 0;
    }
}

// Copy the results of the slots the loop retired (their states are in
// dout, the live slots already empty) to their requests and release the
// slots: two synchronisations of the load stream for the whole set, while
// the loop goes on.
void retire(Lane &Ln, const std::vector<int> &fin) {
    if (fin.empty()) return;
    mhs_server *S = Ln.S;
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < fin.size() && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(Ln.hstates + i, Ln.dout + fin[i], sizeof(InstState),
                            cudaMemcpyDeviceToHost, Ln.load);
    if (e == cudaSuccess) e = cudaStreamSynchronize(Ln.load);
    std::vector<std::vector<uint8_t>> taken(S->opt.full_edges ? fin.size() : 0);
    for (size_t i = 0; i < fin.size() && e == cudaSuccess; ++i) {
        const InstState &s = Ln.hstates[i];
        Request &r = *Ln.slots[fin[i]].req;
        r.vout.resize(s.n);
        r.eout.resize(s.m);
        if (s.n > 0)
            e = cudaMemcpyAsync(r.vout.data(), s.v_c2o, 4 * (size_t)s.n, cudaMemcpyDeviceToHost,
                                Ln.load);
        if (e == cudaSuccess && s.m > 0)
            e = cudaMemcpyAsync(r.eout.data(), s.e_c2o, 4 * (size_t)s.m, cudaMemcpyDeviceToHost,
                                Ln.load);
        if (S->opt.full_edges) {  // FE lowered demands and took vertices
            if (e == cudaSuccess && s.m0 > 0)
                e = cudaMemcpyAsync(r.dem.data(), s.f, 4 * (size_t)s.m0, cudaMemcpyDeviceToHost,
                                    Ln.load);
            taken[i].resize(s.n0);
            if (e == cudaSuccess && s.n0 > 0 && s.forced)
                e = cudaMemcpyAsync(taken[i].data(), s.forced, (size_t)s.n0,
                                    cudaMemcpyDeviceToHost, Ln.load);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(Ln.load);
    const int64_t t = now_ns();
    std::vector<std::shared_ptr<Request>> done;
    for (size_t i = 0; i < fin.size(); ++i) {
        Slot &sl = Ln.slots[fin[i]];
        Request &r = *sl.req;
        if (e == cudaSuccess) {
            const InstState &s = Ln.hstates[i];
            std::sort(r.vout.begin(), r.vout.end());  // layout order -> input ids ascending
            std::sort(r.eout.begin(), r.eout.end());
            r.dout.resize(s.m);
            for (int32_t q = 0; q < s.m; ++q) r.dout[q] = r.dem[r.eout[q]];
            r.rounds = s.rounds;
            r.k = s.k;
            if (!taken.empty())
                for (int32_t v = 0; v < (int32_t)taken[i].size(); ++v)
                    if (taken[i][v]) r.forced.push_back(v);
            r.status = s.status ? MHS_EDEVICE : MHS_OK;
        } else {
            r.status = MHS_ECUDA;
        }
        cudaFreeAsync(sl.arena, Ln.load);
        done.push_back(sl.req);
        Ln.in_use_release += sl.bytes;
        Ln.tiles_release += sl.tiles;
        sl = Slot();
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto &rp : done) {
            rp->t_done = t;
            rp->done = true;
            rp->ptr.clear();
            rp->vtx.clear();
            rp->dem.clear();
            ++S->completed;
            --Ln.active_count;
        }
        S->in_use -= Ln.in_use_release;
        Ln.tiles_in_use -= Ln.tiles_release;
        Ln.in_use_release = 0;
        Ln.tiles_release = 0;
    }
    S->cv_done.notify_all();
    // admission may have waited for this memory
    for (auto &ln : S->lanes) ln.cv_work.notify_one();
}

// Fail everything and stop (the loop's launch has ended or faulted).
void fatal_stop(mhs_server *S, mhs_status st) {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->fatal == MHS_OK) S->fatal = st;
    fail_all_locked(S, S->fatal);
    S->stop = true;
    S->cv_done.notify_all();
    for (auto &ln : S->lanes) ln.cv_work.notify_all();
}

void worker_loop(Lane *L) {
    Lane &Ln = *L;
    mhs_server *S = Ln.S;
    cudaSetDevice(S->device);
    for (;;) {
        bool progress = false;
        // ---- admission: load into free slots, then mark them ready ----
        std::vector<std::pair<int, std::shared_ptr<Request>>> to_admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            bool any_busy = false;
            for (auto &sl : Ln.slots) any_busy |= sl.busy;
            if (!any_busy && !Ln.running)
                Ln.cv_work.wait_for(lk, std::chrono::milliseconds(50), [&] {
                    return S->stop || (!S->paused && !Ln.pending.empty());
                });
            if (S->stop) break;
            if (!S->paused) {
                int si = 0;
                while (!Ln.pending.empty()) {
                    auto &front = Ln.pending.front();
                    if (S->in_use + front->footprint > S->opt.hbm_budget_bytes) break;
                    if (Ln.tiles_in_use + front->tiles > Ln.list_cap) break;
                    while (si < Ln.slots_n && (Ln.slots[si].busy ||
                                               std::any_of(to_admit.begin(), to_admit.end(),
                                                           [si](auto &p) { return p.first == si; })))
                        ++si;
                    if (si >= Ln.slots_n) break;
                    S->in_use += front->footprint;
                    Ln.tiles_in_use += front->tiles;
                    S->peak = std::max(S->peak, S->in_use);
                    front->t_admit = now_ns();
                    to_admit.emplace_back(si, front);
                    Ln.pending.pop_front();
                    ++S->admitted;
                    ++si;
                }
            }
        }
        std::vector<int> loaded;
        for (auto &p : to_admit) {
            mhs_status st = admit(Ln, p.first, p.second);
            if (st != MHS_OK) {
                std::lock_guard<std::mutex> lk(S->mu);
                S->in_use -= p.second->footprint;
                Ln.tiles_in_use -= p.second->tiles;
                p.second->status = st;
                p.second->done = true;
                p.second->t_done = now_ns();
                S->cv_done.notify_all();
            } else {
                loaded.push_back(p.first);
            }
        }
        if (!loaded.empty()) {
            // the staged states, arenas and build kernels are complete before
            // the loop can see a ready flag
            if (cudaStreamSynchronize(Ln.load) != cudaSuccess) {
                fatal_stop(S, MHS_ECUDA);
                break;
            }
            std::atomic_thread_fence(std::memory_order_seq_cst);
            for (int si : loaded) reinterpret_cast<volatile int32_t *>(Ln.hready)[si] = 1;
            std::atomic_thread_fence(std::memory_order_seq_cst);
            progress = true;
        }
        // ---- retirement: the slots the loop published ----
        const uint32_t head = reinterpret_cast<volatile ServerFlags *>(Ln.hflags)->head;
        std::atomic_thread_fence(std::memory_order_seq_cst);
        if (head != Ln.consumed) {
            std::vector<int> fin;
            for (uint32_t q = Ln.consumed; q != head; ++q) {
                const int si =
                    reinterpret_cast<volatile int32_t *>(Ln.hring)[q % (uint32_t)Ln.slots_n];
                if (si >= 0 && si < Ln.slots_n && Ln.slots[si].busy) fin.push_back(si);
            }
            Ln.consumed = head;
            retire(Ln, fin);
            progress = true;
        }
        // ---- the loop's launch: ended, faulted, or to be started ----
        if (Ln.running) {
            const cudaError_t q = cudaStreamQuery(Ln.stream);
            if (q == cudaSuccess) {
                Ln.running = false;
                if (reinterpret_cast<volatile ServerFlags *>(Ln.hflags)->kerr) {
                    fatal_stop(S, MHS_EDEVICE);
                    break;
                }
                continue;  // take what it published last before deciding to start it again
            }
            if (q != cudaErrorNotReady) {
                fatal_stop(S, MHS_ECUDA);
                break;
            }
        }
        if (!Ln.running) {
            bool any_busy = false;
            for (auto &sl : Ln.slots) any_busy |= sl.busy;
            if (any_busy) {
                cudaError_t e = cudaGraphLaunch(Ln.graph, Ln.stream);
                if (e != cudaSuccess) {
                    fatal_stop(S, MHS_ECUDA);
                    break;
                }
                Ln.running = true;
                progress = true;
            }
        }
        if (!progress && Ln.running) {  // rounds are running: look again shortly
            std::unique_lock<std::mutex> lk(S->mu);
            Ln.cv_work.wait_for(lk, std::chrono::microseconds(20), [&] {
                return S->stop || (!S->paused && !Ln.pending.empty());
            });
        }
    }
    // stop: end the loop at its next round boundary and wait for it
    reinterpret_cast<volatile ServerFlags *>(Ln.hflags)->stop = 1;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    if (Ln.running) cudaStreamSynchronize(Ln.stream);
    Ln.running = false;
    cudaStreamSynchronize(Ln.load);
}

// The lane's loop: a memset node resets the iteration count, then a WHILE
// node whose body admits ready slots, runs one round (DP, then MD, then FE
// if enabled) over the slot table, retires finished slots and sets the
// condition.
mhs_status capture_graph(Lane &Ln) {
    mhs_server *S = Ln.S;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    auto bail = [&](cudaError_t err, const char *what) {
        if (g) cudaGraphDestroy(g);
        return set_error(MHS_ECUDA, "server loop graph (%s): %s", what, cudaGetErrorString(err));
    };
    if (e != cudaSuccess) return bail(e, "create");
    cudaGraphConditionalHandle cond;
    e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return bail(e, "handle");
    cudaGraphNode_t reset;
    cudaMemsetParams mp;
    std::memset(&mp, 0, sizeof(mp));
    mp.dst = &Ln.ddev->iters;
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
    e = cudaStreamBeginCaptureToGraph(Ln.stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bail(e, "capture");
    cudaError_t e1 = launch_server_admit(Ln.dstate, Ln.dstage, Ln.dready, Ln.slots_n, Ln.stream);
    if (e1 == cudaSuccess)
        e1 = launch_round_phase(Ln.dstate, Ln.dplan, Ln.dctr, Ln.slots_n, 0, S->contraction,
                                S->sms, Ln.dkerr, Ln.stream, nullptr, nullptr, nullptr);
    if (e1 == cudaSuccess)
        e1 = launch_round_phase(Ln.dstate, Ln.dplan, Ln.dctr, Ln.slots_n, 1, S->contraction,
                                S->sms, Ln.dkerr, Ln.stream, nullptr, nullptr, Ln.ddone);
    if (e1 == cudaSuccess && S->opt.full_edges)
        e1 = launch_full_edges(Ln.dstate, Ln.slots_n, Ln.dctr, Ln.ddone, S->sms, Ln.stream);
    if (e1 == cudaSuccess)
        e1 = launch_server_retire(Ln.dstate, Ln.dout, Ln.ddone, Ln.dctr, Ln.dring, Ln.dflags,
                                  Ln.ddev, Ln.slots_n, Ln.stream);
    if (e1 == cudaSuccess)
        e1 = launch_server_cond(cond, Ln.dctr, Ln.dkerr, Ln.dplan, Ln.ddev, Ln.dflags, Ln.dready,
                                Ln.slots_n, kLoopIters, Ln.stream);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(Ln.stream, &captured);
    if (e1 != cudaSuccess) return bail(e1, "round");
    if (e != cudaSuccess) return bail(e, "end capture");
    e = cudaGraphInstantiate(&Ln.graph, g, 0);
    cudaGraphDestroy(g);
    g = nullptr;
    if (e != cudaSuccess) return set_error(MHS_ECUDA, "server graph: %s", cudaGetErrorString(e));
    return MHS_OK;
}

// Device and pinned memory, and the round graph, of one lane.
mhs_status setup_lane(mhs_server *S, Lane &Ln, int id, int32_t slots, int64_t list_cap,
                      cudaStream_t user_stream, int priority) {
    Ln.id = id;
    Ln.S = S;
    Ln.slots_n = slots;
    Ln.slots.resize(slots);
    Ln.list_cap = list_cap;
    if (user_stream) {
        Ln.stream = user_stream;
    } else {
        if (cudaStreamCreateWithPriority(&Ln.stream, cudaStreamNonBlocking, priority) != cudaSuccess)
            return set_error(MHS_ECUDA, "stream creation failed");
        Ln.own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&Ln.load, cudaStreamNonBlocking) != cudaSuccess)
        return set_error(MHS_ECUDA, "stream creation failed");
    const int64_t ns = slots;
    const int64_t o_state = 0;
    const int64_t o_stage = o_state + up(sizeof(InstState) * ns, 256);
    const int64_t o_out = o_stage + up(sizeof(InstState) * ns, 256);
    const int64_t o_plan = o_out + up(sizeof(InstState) * ns, 256);
    const int64_t o_row = o_plan + up(sizeof(Plan), 256);
    const int64_t o_tile = o_row + up(4 * (ns + 1), 256);
    const int64_t o_ctr = o_tile + up(8 * (ns + 1), 256);
    const int64_t o_dev = o_ctr + up(sizeof(BatchCounters), 256);
    const int64_t o_kerr = o_dev + up(sizeof(ServerDev), 256);
    const int64_t o_done = o_kerr + 256;
    const int64_t o_list = o_done + up(4 * ns, 256);
    const int64_t total = o_list + up(8 * std::max<int64_t>(list_cap, 1), 256);
    if (cudaMallocFromPoolAsync(reinterpret_cast<void **>(&Ln.ctl), (size_t)total, S->pool,
                                Ln.stream) != cudaSuccess)
        return set_error(MHS_ENOMEM, "server control allocation failed");
    Ln.dstate = reinterpret_cast<InstState *>(Ln.ctl + o_state);
    Ln.dstage = reinterpret_cast<InstState *>(Ln.ctl + o_stage);
    Ln.dout = reinterpret_cast<InstState *>(Ln.ctl + o_out);
    Ln.dplan = reinterpret_cast<Plan *>(Ln.ctl + o_plan);
    Ln.dctr = reinterpret_cast<BatchCounters *>(Ln.ctl + o_ctr);
    Ln.ddev = reinterpret_cast<ServerDev *>(Ln.ctl + o_dev);
    Ln.dkerr = reinterpret_cast<int32_t *>(Ln.ctl + o_kerr);
    Ln.ddone = reinterpret_cast<int32_t *>(Ln.ctl + o_done);
    // host-mapped: the flags, then ready[ns], then ring[ns]
    const size_t o_ready = up(sizeof(ServerFlags), 64);
    const size_t o_ring = o_ready + up(4 * ns, 64);
    const size_t mapped_bytes = o_ring + up(4 * ns, 64);
    if (cudaHostAlloc(reinterpret_cast<void **>(&Ln.mapped), mapped_bytes,
                      cudaHostAllocMapped) != cudaSuccess)
        return set_error(MHS_ENOMEM, "mapped host allocation failed");
    std::memset(Ln.mapped, 0, mapped_bytes);
    uint8_t *dmapped = nullptr;
    if (cudaHostGetDevicePointer(reinterpret_cast<void **>(&dmapped), Ln.mapped, 0) !=
        cudaSuccess)
        return set_error(MHS_ECUDA, "mapped host memory unavailable on the device");
    Ln.hflags = reinterpret_cast<ServerFlags *>(Ln.mapped);
    Ln.dflags = reinterpret_cast<ServerFlags *>(dmapped);
    Ln.hready = reinterpret_cast<int32_t *>(Ln.mapped + o_ready);
    Ln.dready = reinterpret_cast<int32_t *>(dmapped + o_ready);
    Ln.hring = reinterpret_cast<int32_t *>(Ln.mapped + o_ring);
    Ln.dring = reinterpret_cast<int32_t *>(dmapped + o_ring);
    if (cudaMallocHost(&Ln.hmaps, 2 * tmap_bytes() * (size_t)ns) != cudaSuccess ||
        cudaMallocHost(&Ln.hstates, sizeof(InstState) * (size_t)ns) != cudaSuccess)
        return set_error(MHS_ENOMEM, "pinned allocation failed");
    Plan p;
    std::memset(&p, 0, sizeof(p));
    p.count = slots;
    p.row_off = reinterpret_cast<int32_t *>(Ln.ctl + o_row);
    p.tile_off = reinterpret_cast<int64_t *>(Ln.ctl + o_tile);
    p.tile_list = reinterpret_cast<int64_t *>(Ln.ctl + o_list);
    p.list_cap = (int32_t)std::min<int64_t>(list_cap, INT32_MAX);
    p.group_rows = tile_group_rows();
    p.tile_n = kTcNDefault;  // the server's lanes contract with the default tile shape
    p.half_stages = 1;
    cudaError_t e = cudaMemsetAsync(Ln.ctl, 0, (size_t)o_list, Ln.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(Ln.dplan, &p, sizeof(p), cudaMemcpyHostToDevice, Ln.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(Ln.stream);
    if (e != cudaSuccess) return set_error(MHS_ECUDA, "server setup: %s", cudaGetErrorString(e));
    return capture_graph(Ln);
}

void destroy_server(mhs_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    for (auto &ln : S->lanes) ln.cv_work.notify_all();
    for (auto &ln : S->lanes)
        if (ln.worker.joinable()) ln.worker.join();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        fail_all_locked(S, MHS_ECUDA);
    }
    S->cv_done.notify_all();
    for (auto &ln : S->lanes) {
        if (ln.stream) cudaStreamSynchronize(ln.stream);
        for (auto &sl : ln.slots)
            if (sl.arena) cudaFreeAsync(sl.arena, ln.stream);
        if (ln.load) cudaStreamSynchronize(ln.load);
        if (ln.graph) cudaGraphExecDestroy(ln.graph);
        if (ln.ctl) cudaFreeAsync(ln.ctl, ln.stream);
        if (ln.stream) cudaStreamSynchronize(ln.stream);
        if (ln.mapped) cudaFreeHost(ln.mapped);
        if (ln.hmaps) cudaFreeHost(ln.hmaps);
        if (ln.hstates) cudaFreeHost(ln.hstates);
        if (ln.load) cudaStreamDestroy(ln.load);
        if (ln.own_stream && ln.stream) cudaStreamDestroy(ln.stream);
    }
    delete S;
}

}  // namespace

extern "C" {

mhs_status mhs_server_default_options(mhs_server_options *opt) {
    if (!opt) return set_error(MHS_EINVAL, "opt is NULL");
    std::memset(opt, 0, sizeof(*opt));
    opt->hbm_budget_bytes = 0;
    opt->max_slots = 256;
    opt->queue_capacity = 65536;
    opt->contraction = MHS_CONTRACT_AUTO;
    opt->small_items = 0;
    return MHS_OK;
}

mhs_status mhs_server_create(const mhs_server_options *opt_in, void *cuda_stream,
                             mhs_server **out) {
    if (!out) return set_error(MHS_EINVAL, "out is NULL");
    *out = nullptr;
    mhs_server_options opt;
    mhs_server_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.max_slots < 1 || opt.max_slots > 4096)
        return set_error(MHS_EINVAL, "max_slots must be in [1, 4096]");
    if (opt.queue_capacity < 1) return set_error(MHS_EINVAL, "queue_capacity must be >= 1");
    if (opt.contraction < 0 || opt.contraction > 2)
        return set_error(MHS_EINVAL, "contraction must be 0, 1 or 2");
    if (opt.hbm_budget_bytes < 0) return set_error(MHS_EINVAL, "hbm_budget_bytes must be >= 0");
    if (opt.layout < 0 || opt.layout > 3)
        return set_error(MHS_EINVAL, "layout must be 0, 1, 2 or 3");
    if (opt.sparsity < 0 || opt.sparsity > 2)
        return set_error(MHS_EINVAL, "sparsity must be 0, 1 or 2");
    if (opt.edge_rule < 0 || opt.edge_rule > 1)
        return set_error(MHS_EINVAL, "edge_rule must be 0 (DP) or 1 (SE)");
    if (opt.full_edges < 0 || opt.full_edges > 1)
        return set_error(MHS_EINVAL, "full_edges must be 0 or 1");
    auto *S = new mhs_server();
    S->opt = opt;
    S->contraction = opt.contraction == MHS_CONTRACT_POPCOUNT ? kPopcount : kFp8;
    // < 0: one lane for every request; 0: default split
    S->small_items = opt.small_items < 0 ? INT64_MAX : (opt.small_items == 0 ? 8192 : opt.small_items);
    auto bail = [&](mhs_status st) {
        destroy_server(S);
        return st;
    };
    if (cudaGetDevice(&S->device) != cudaSuccess) return bail(set_error(MHS_ECUDA, "no device"));
    cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device);
    if (S->opt.hbm_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        S->opt.hbm_budget_bytes = (int64_t)(fr / 4 * 3);
    }
    if (pool_for(S->device, &S->pool) != cudaSuccess)
        return bail(set_error(MHS_ECUDA, "memory pool unavailable"));
    if (S->contraction == kFp8 && prepare_tc_contract() != cudaSuccess)
        return bail(set_error(MHS_ECUDA, "tcgen05 kernel setup failed"));
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);  // hi is the most urgent
    const bool dense = S->contraction == kFp8;
    // lane 0: small requests, many slots, high priority; lane 1: large ones, a few at a time
    mhs_status st = setup_lane(S, S->lanes[0], 0, opt.max_slots, dense ? kServerListCap : 1,
                               nullptr, hi);
    if (st) return bail(st);
    st = setup_lane(S, S->lanes[1], 1, std::min(opt.max_slots, 4), dense ? kServerListCap : 1,
                    static_cast<cudaStream_t>(cuda_stream), lo);
    if (st) return bail(st);
    for (auto &ln : S->lanes) ln.worker = std::thread(worker_loop, &ln);
    *out = S;
    return MHS_OK;
}

mhs_status mhs_submit(mhs_server *S, int32_t n, int32_t m, const int32_t *edge_ptr,
                      const int32_t *edge_vtx, const int32_t *demand, int64_t k,
                      uint64_t *ticket) {
    if (!S || !ticket) return set_error(MHS_EINVAL, "NULL argument");
    if (n < 0 || m < 0 || n >= (1 << 24) || m >= (1 << 24))
        return set_error(MHS_EINVAL, "n and m must be in [0, 2^24)");
    if (!edge_ptr || (m > 0 && !demand)) return set_error(MHS_EINVAL, "NULL input array");
    if (edge_ptr[0] != 0) return set_error(MHS_EINVAL, "edge_ptr[0] must be 0");
    const int32_t nnz = edge_ptr[m];
    if (nnz > 0 && !edge_vtx) return set_error(MHS_EINVAL, "edge_vtx is NULL");
    // structural checks on the host, before anything is queued
    std::vector<int32_t> mark((size_t)n, -1);
    for (int32_t e = 0; e < m; ++e) {
        if (edge_ptr[e + 1] < edge_ptr[e])
            return set_error(MHS_EINVAL, "edge_ptr decreases at hyperedge %d", e);
        if (demand[e] < 1) return set_error(MHS_EINVAL, "demand of hyperedge %d is < 1", e);
        for (int32_t p = edge_ptr[e]; p < edge_ptr[e + 1]; ++p) {
            const int32_t v = edge_vtx[p];
            if (v < 0 || v >= n)
                return set_error(MHS_EINVAL, "hyperedge %d has vertex id %d outside [0,%d)", e, v, n);
            if (mark[v] == e) return set_error(MHS_EINVAL, "hyperedge %d lists vertex %d twice", e, v);
            mark[v] = e;
        }
    }
    auto r = std::make_shared<Request>();
    r->n = n;
    r->m = m;
    r->k = k;
    r->ptr.assign(edge_ptr, edge_ptr + m + 1);
    r->vtx.assign(edge_vtx, edge_vtx + nnz);
    r->dem.assign(demand, demand + m);
    r->footprint = plan_layout(n, m, nnz, S->contraction == kFp8, S->opt.full_edges != 0).bytes;
    // tile-list entries only matter for the tcgen05 contraction
    r->tiles = S->contraction == kFp8
                   ? std::max(tc_tiles(m, kTcNDefault), tc_tiles(n, kTcNDefault))
                   : 0;
    if (S->contraction == kFp8 && r->tiles > kServerListCap)
        return set_error(MHS_ENOMEM, "instance needs %lld tiles, over the server's %lld",
                         (long long)r->tiles, (long long)kServerListCap);
    if (r->footprint > S->opt.hbm_budget_bytes)
        return set_error(MHS_ENOMEM, "instance needs %lld bytes, over the server budget %lld",
                         (long long)r->footprint, (long long)S->opt.hbm_budget_bytes);
    Lane &ln = S->lanes[(int64_t)n + m <= S->small_items ? 0 : 1];
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->fatal) return set_error(S->fatal, "server stopped after a device error");
        const int64_t queued = (int64_t)S->lanes[0].pending.size() + S->lanes[1].pending.size();
        if (queued >= S->opt.queue_capacity)
            return set_error(MHS_EBUSY, "request queue full (%d)", S->opt.queue_capacity);
        r->ticket = S->next_ticket++;
        r->t_submit = now_ns();
        ln.pending.push_back(r);
        S->table[r->ticket] = r;
        ++S->submitted;
        *ticket = r->ticket;
    }
    ln.cv_work.notify_one();
    return MHS_OK;
}

mhs_status mhs_poll(mhs_server *S, uint64_t ticket, int64_t timeout_us, int32_t *vtx_out,
                    int32_t vtx_cap, int32_t *n_out, int32_t *edge_out, int32_t *demand_out,
                    int32_t edge_cap, int32_t *m_out, int64_t *k_out, int32_t *rounds_out,
                    int64_t *times_ns) {
    if (!S) return set_error(MHS_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->table.find(ticket);
    if (it == S->table.end()) return set_error(MHS_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    std::shared_ptr<Request> r = it->second;
    if (!r->done) {
        if (timeout_us != 0) {
            auto pred = [&] { return r->done; };
            if (timeout_us < 0) S->cv_done.wait(lk, pred);
            else S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred);
        }
        if (!r->done) return set_error(MHS_EAGAIN, "request %llu not finished", (unsigned long long)ticket);
    }
    if (r->status != MHS_OK) {
        S->table.erase(it);
        return set_error(r->status, "request %llu failed on the device", (unsigned long long)ticket);
    }
    const int32_t nv = (int32_t)r->vout.size(), ne = (int32_t)r->eout.size();
    if (n_out) *n_out = nv;
    if (m_out) *m_out = ne;
    if (k_out) *k_out = r->k;
    if (rounds_out) *rounds_out = r->rounds;
    if (times_ns) {
        times_ns[0] = r->t_admit - r->t_submit;
        times_ns[1] = r->t_done - r->t_admit;
        times_ns[2] = r->t_done - r->t_submit;
    }
    if (!vtx_out && !edge_out && !demand_out) return MHS_OK;  // counts only; kept
    if ((vtx_out && vtx_cap < nv) || ((edge_out || demand_out) && edge_cap < ne))
        return set_error(MHS_EINVAL, "output capacity too small (need %d vertices, %d edges)", nv, ne);
    if (vtx_out) std::copy(r->vout.begin(), r->vout.end(), vtx_out);
    if (edge_out) std::copy(r->eout.begin(), r->eout.end(), edge_out);
    if (demand_out) std::copy(r->dout.begin(), r->dout.end(), demand_out);
    S->table.erase(it);
    return MHS_OK;
}

mhs_status mhs_server_forced(mhs_server *S, uint64_t ticket, int32_t *vtx_out, int32_t cap,
                             int32_t *count_out) {
    if (!S) return set_error(MHS_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->table.find(ticket);
    if (it == S->table.end())
        return set_error(MHS_EINVAL, "unknown or released ticket %llu", (unsigned long long)ticket);
    const Request &r = *it->second;
    if (!r.done) return set_error(MHS_EAGAIN, "request %llu not finished", (unsigned long long)ticket);
    if (r.status != MHS_OK)
        return set_error(r.status, "request %llu failed on the device", (unsigned long long)ticket);
    const int32_t c = (int32_t)r.forced.size();
    if (count_out) *count_out = c;
    if (!vtx_out) return MHS_OK;
    if (cap < c) return set_error(MHS_EINVAL, "output capacity too small (need %d vertices)", c);
    std::copy(r.forced.begin(), r.forced.end(), vtx_out);
    return MHS_OK;
}

mhs_status mhs_server_pause(mhs_server *S, int32_t paused) {
    if (!S) return set_error(MHS_EINVAL, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->paused = paused != 0;
    }
    for (auto &ln : S->lanes) ln.cv_work.notify_all();
    return MHS_OK;
}

mhs_status mhs_server_get_stats(mhs_server *S, mhs_server_stats *out) {
    if (!S || !out) return set_error(MHS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->admitted = S->admitted;
    out->completed = S->completed;
    for (auto &ln : S->lanes)
        if (ln.hflags) out->rounds += reinterpret_cast<volatile ServerFlags *>(ln.hflags)->rounds;
    out->pending = (int32_t)(S->lanes[0].pending.size() + S->lanes[1].pending.size());
    out->active = S->lanes[0].active_count + S->lanes[1].active_count;
    out->bytes_in_use = S->in_use;
    out->peak_bytes = S->peak;
    out->budget_bytes = S->opt.hbm_budget_bytes;
    return MHS_OK;
}

void mhs_server_destroy(mhs_server *S) { destroy_server(S); }

}  // extern "C"

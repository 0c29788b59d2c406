// noalloc.cu -- mhs_kernelize_noalloc: a complete kernelization of one small
// instance whose working memory is a fixed, file-scope device array, so the
// call allocates nothing.
//
// Who needs it: callers that may not allocate device memory while they run
// -- code inside a custom or fixed-budget allocator, real-time loops that
// forbid cudaMalloc/cudaFree (both can synchronise the device), or plug-ins
// embedded in a host that owns all device memory.  They pass device inputs
// and device outputs; everything else (id maps, bit-packed operands, flags,
// counters, the per-instance state) lives in kScratch below.
//
// The array is kScratchBytes (6 MiB) and every GPU that loads this library
// holds it until the process exits.  It fits instances with n <= 4096,
// m <= 4096 and at most 65,536 incidences; larger ones are rejected with
// MHS_EINVAL.  It uses the bit-packed popcount contraction and the same
// encode / compaction kernels as the main path.
//
// All calls share the one array and it keeps the last call's contents, so
// everything that must start from zero is cleared by each call.  Calls whose
// GPU work overlaps (different streams or threads at the same time) race on
// the array and give wrong results: serialise them.
//
// Set-up: every call looks up the array's device address with
// cudaGetSymbolAddress, with the caller's device current.  No address is
// cached, so a context torn down and created again (cudaDeviceReset) cannot
// leave a stale one behind.  The first call on a device may load the
// library's device code into the context; make that first call before any
// stream capture.
//
// Pointers: every device array the caller passes is checked with
// cudaPointerGetAttributes (device or managed memory of the current device)
// before any kernel touches it; anything else is MHS_EINVAL.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "kernels.h"
#include "mhs.h"
#include "mhs_internal.h"

namespace mhs {
namespace {

constexpr int32_t kNoAllocMaxN = 4096;
constexpr int32_t kNoAllocMaxM = 4096;
constexpr int64_t kNoAllocMaxNnz = 65536;
constexpr size_t kScratchBytes = (size_t)6 << 20;  // 6 MiB

static __device__ __align__(256) uint8_t kScratch[kScratchBytes];

inline int64_t up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline int64_t words(int64_t K) { return up(((K + 31) / 32) > 0 ? (K + 31) / 32 : 1, 4); }

struct Take {
    int64_t bytes = 0;
    int64_t operator()(int64_t n) {
        int64_t o = bytes;
        bytes += up(n > 0 ? n : 1, 256);
        return o;
    }
};

mhs_status err(char *buf, size_t cap, mhs_status st, const char *msg) {
    if (buf && cap) {
        std::strncpy(buf, msg, cap - 1);
        buf[cap - 1] = '\0';
    }
    return st;
}

// True if p is device (or managed) memory that device `dev` can use; a
// pointer of no kind CUDA knows (plain host memory) is rejected.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // the failed query's error is not sticky: clear it
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
}  // namespace mhs

using namespace mhs;

extern "C" mhs_status mhs_kernelize_noalloc(int32_t n, int32_t m, const int32_t *edge_ptr,
                                            const int32_t *edge_vtx, const int32_t *demand,
                                            int32_t nnz, uint8_t *alive_v, uint8_t *alive_e,
                                            int32_t *rounds_out, void *cuda_stream,
                                            char *err_buf, size_t err_cap) {
    if (n < 0 || m < 0 || nnz < 0)
        return err(err_buf, err_cap, MHS_EINVAL, "n, m and nnz must be >= 0");
    if (n > kNoAllocMaxN || m > kNoAllocMaxM || nnz > kNoAllocMaxNnz)
        return err(err_buf, err_cap, MHS_EINVAL,
                   "instance too large for the static scratch (n, m <= 4096, nnz <= 65536)");
    if (!edge_ptr || (m > 0 && !demand) || (nnz > 0 && !edge_vtx) ||
        (n > 0 && !alive_v) || (m > 0 && !alive_e))
        return err(err_buf, err_cap, MHS_EINVAL, "NULL array");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0)
        return err(err_buf, err_cap, MHS_ECUDA, "no current CUDA device");
    if (!on_device(edge_ptr, dev) || (m > 0 && !on_device(demand, dev)) ||
        (nnz > 0 && !on_device(edge_vtx, dev)) || (n > 0 && !on_device(alive_v, dev)) ||
        (m > 0 && !on_device(alive_e, dev)))
        return err(err_buf, err_cap, MHS_EINVAL,
                   "an array is not device memory of the current device");
    void *base_v = nullptr;
    if (cudaGetSymbolAddress(&base_v, kScratch) != cudaSuccess || !base_v)
        return err(err_buf, err_cap, MHS_ECUDA, "cudaGetSymbolAddress(scratch) failed");
    uint8_t *base = static_cast<uint8_t *>(base_v);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
        return err(err_buf, err_cap, MHS_ECUDA, "cannot read the SM count");

    // layout inside the scratch (same roles as the main path's arena)
    Take take;
    const int64_t o_state = take(sizeof(InstState));
    const int64_t o_plan = take(sizeof(Plan));
    const int64_t o_rowoff = take(2 * sizeof(int32_t));
    const int64_t o_tileoff = take(2 * sizeof(int64_t));
    const int64_t o_ctr = take(sizeof(BatchCounters));
    const int64_t o_kerr = take(sizeof(int32_t));
    const int64_t o_vo2c = take(4 * (int64_t)n), o_vc2o = take(4 * (int64_t)n);
    const int64_t o_eo2c = take(4 * (int64_t)m), o_ec2o = take(4 * (int64_t)m);
    const int64_t o_eprev = take(4 * (int64_t)m);
    const int64_t o_ef = take(4 * (int64_t)m), o_es = take(4 * (int64_t)m);
    const int64_t o_vdeg = take(4 * ((int64_t)n + 1)), o_vmaxf = take(4 * (int64_t)n);
    const int64_t o_vcnt = take(4 * ((int64_t)n + 1));
    const int64_t o_edel = take(m), o_vdel = take(n);
    const int64_t arows = up(m > 0 ? m : 1, kRowAlign), atrows = up(n > 0 ? n : 1, kRowAlign);
    const int64_t o_ab = take(arows * words(n) * 4);
    const int64_t o_atb = take(atrows * words(m) * 4);
    if (take.bytes > (int64_t)kScratchBytes)
        return err(err_buf, err_cap, MHS_EINVAL, "instance does not fit the static scratch");

    InstState st;
    std::memset(&st, 0, sizeof(st));
    st.n0 = n;
    st.m0 = m;
    st.nnz0 = nnz;
    st.eptr = edge_ptr;  // inputs are read in place
    st.evtx = edge_vtx;
    st.f = const_cast<int32_t *>(demand);  // read only: rule FE is off here
    st.v_o2c = reinterpret_cast<int32_t *>(base + o_vo2c);
    st.v_c2o = reinterpret_cast<int32_t *>(base + o_vc2o);
    st.e_o2c = reinterpret_cast<int32_t *>(base + o_eo2c);
    st.e_c2o = reinterpret_cast<int32_t *>(base + o_ec2o);
    st.e_prev = reinterpret_cast<int32_t *>(base + o_eprev);
    st.e_f = reinterpret_cast<int32_t *>(base + o_ef);
    st.e_s = reinterpret_cast<int32_t *>(base + o_es);
    st.v_deg = reinterpret_cast<int32_t *>(base + o_vdeg);
    st.v_maxf = reinterpret_cast<int32_t *>(base + o_vmaxf);
    st.v_cnt = reinterpret_cast<int32_t *>(base + o_vcnt);
    st.e_del = base + o_edel;
    st.v_del = base + o_vdel;
    st.Ab = reinterpret_cast<uint32_t *>(base + o_ab);
    st.Atb = reinterpret_cast<uint32_t *>(base + o_atb);
    st.Ab_pitch = (int32_t)words(n);
    st.Atb_pitch = (int32_t)words(m);
    st.A_rows = (int32_t)arows;
    st.At_rows = (int32_t)atrows;

    Plan pl;
    std::memset(&pl, 0, sizeof(pl));
    pl.count = 1;
    pl.row_off = reinterpret_cast<int32_t *>(base + o_rowoff);
    pl.tile_off = reinterpret_cast<int64_t *>(base + o_tileoff);

    InstState *dst = reinterpret_cast<InstState *>(base + o_state);
    Plan *dplan = reinterpret_cast<Plan *>(base + o_plan);
    BatchCounters *dctr = reinterpret_cast<BatchCounters *>(base + o_ctr);
    int32_t *dkerr = reinterpret_cast<int32_t *>(base + o_kerr);

    // pageable sources: each copy returns once the source has been staged
    cudaError_t e = cudaMemcpyAsync(dst, &st, sizeof(st), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dplan, &pl, sizeof(pl), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dkerr, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = launch_validate(dst, 1, s);
    int32_t status = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&status, &dst->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return err(err_buf, err_cap, MHS_ECUDA, cudaGetErrorString(e));
    if (status) return err(err_buf, err_cap, MHS_EINVAL, "malformed instance (bad edge_ptr or vertex id)");

    // the bit-packed operands must start all-zero (a call that stopped early
    // may have left incidences set)
    e = cudaMemsetAsync(base + o_ab, 0, (size_t)(o_atb - o_ab + atrows * words(m) * 4), s);
    if (e == cudaSuccess) e = launch_build(dst, 1, 0, nnz, m, n, s);
    if (e != cudaSuccess) return err(err_buf, err_cap, MHS_ECUDA, cudaGetErrorString(e));
    BatchCounters ctr;
    std::memset(&ctr, 0, sizeof(ctr));
    int32_t kerr = 0;
    // every changing round deletes an item, so n + m + 1 rounds always suffice
    for (int32_t r = 0; r <= n + m + 1; ++r) {
        e = launch_round_phase(dst, dplan, dctr, 1, 0, kPopcount, sms, dkerr, s, nullptr, nullptr);
        if (e == cudaSuccess)
            e = launch_round_phase(dst, dplan, dctr, 1, 1, kPopcount, sms, dkerr, s, nullptr,
                                   nullptr);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&ctr, dctr, sizeof(ctr), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&kerr, dkerr, sizeof(kerr), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return err(err_buf, err_cap, MHS_ECUDA, cudaGetErrorString(e));
        if (kerr || ctr.status_any)
            return err(err_buf, err_cap, MHS_EDEVICE, "kernel reported an error status");
        if (ctr.active == 0) break;
    }
    if (ctr.active != 0)  // unreachable with correct kernels: never report a partial result
        return err(err_buf, err_cap, MHS_EDEVICE, "round cap reached before fixpoint");
    if (n > 0 || m > 0) {
        e = launch_alive_masks(dst, n > 0 ? alive_v : nullptr, m > 0 ? alive_e : nullptr, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return err(err_buf, err_cap, MHS_ECUDA, cudaGetErrorString(e));
    }
    if (rounds_out) *rounds_out = ctr.max_rounds_seen;
    return MHS_OK;
}

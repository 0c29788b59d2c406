// selftest.cu -- diagnostics of the bounded-wait machinery.
//
// mhs_selftest_bounded_wait launches one block that waits on an mbarrier
// nothing will ever arrive at, with the same bounded wait the tcgen05
// contraction uses.  The wait must give up after limit_ns, the kernel must
// write the timeout status and return, and the CUDA context must stay
// usable.  This exercises failure detection without faulting or hanging a
// GPU.
#include <cuda_runtime.h>

#include "bounded_wait.cuh"
#include "host_internal.h"
#include "mhs.h"
#include "mhs_internal.h"

namespace mhs {
namespace {

__global__ void k_wait_forever_bounded(uint64_t limit_ns, int32_t *status, int64_t *waited) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t t0 = globaltimer();
        // nobody arrives: phase 0 never completes
        const bool ok = mbar_wait(smem_u32(&bar), 0, &abort_flag, limit_ns);
        *waited = (int64_t)(globaltimer() - t0);
        *status = ok ? 0 : kErrTimeout;
    }
}

}  // namespace
}  // namespace mhs

extern "C" mhs_status mhs_selftest_bounded_wait(int64_t limit_ns, int32_t *status_out,
                                                int64_t *waited_ns_out) {
    using namespace mhs;
    if (limit_ns <= 0 || limit_ns > 2000000000ll)
        return set_error(MHS_EINVAL, "limit_ns must be in (0, 2e9]");
    int32_t *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 16);
    if (e != cudaSuccess) return set_error(MHS_ECUDA, "selftest: %s", cudaGetErrorString(e));
    int32_t h_status = -1;
    int64_t h_waited = 0;
    k_wait_forever_bounded<<<1, 32>>>((uint64_t)limit_ns, d, reinterpret_cast<int64_t *>(d + 2));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(&h_status, d, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&h_waited, d + 2, 8, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return set_error(MHS_ECUDA, "selftest: %s", cudaGetErrorString(e));
    if (status_out) *status_out = h_status;
    if (waited_ns_out) *waited_ns_out = h_waited;
    return MHS_OK;
}

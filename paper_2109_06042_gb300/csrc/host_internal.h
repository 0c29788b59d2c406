// host_internal.h -- host helpers shared by the C ABI (mhs_api.cpp) and the
// serving loop (server.cpp).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "mhs.h"

namespace mhs {

// Record a thread-local message for mhs_last_error() and return st.
mhs_status set_error(mhs_status st, const char *fmt, ...);

// The library's stream-ordered memory pool of a device (freed blocks are
// kept for reuse, so load/free loops do not reach the driver).
cudaError_t pool_for(int dev, cudaMemPool_t *out);

// InstState::layout_sorted for an mhs_layout option.
inline int32_t layout_code(int32_t layout) {
    return layout == MHS_LAYOUT_INPUT ? 0 : layout == MHS_LAYOUT_SORTED ? 1 : 2;
}

// Blocks of kPinnedBlock bytes of page-locked host memory from a
// process-wide slab.  cudaMallocHost / cudaFreeHost cost tens of
// microseconds and cudaFreeHost synchronises the device, which every
// load / free would otherwise pay.  Blocks are 256-byte aligned.
constexpr size_t kPinnedBlock = 1024;
void *pinned_block();  // nullptr if page-locked memory is unavailable
void pinned_release(void *p);

}  // namespace mhs

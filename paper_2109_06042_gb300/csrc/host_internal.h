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

}  // namespace mhs

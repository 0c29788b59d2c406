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

// Tile shape of the tcgen05 contraction for a load: explicit options, else
// the autotuner's table (tiles.cpp), else the defaults.
struct TileChoice {
    int32_t tile_n;       // 128 or 256 columns per tile
    int32_t group_rows;   // row blocks per L2 group of the tile order
    int32_t half_stages;  // 1: a K block shared in one half is loaded as that half
    int32_t from_table;   // 1: the table gave the shape
};
// typical_rows: the larger of n and m (a batch: its mean over the instances).
TileChoice choose_tiles(int32_t count, int64_t typical_rows, const mhs_options &opt);
const char *tile_table_path();

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

// Larger page-locked staging buffers (a batch's instance states and tensor
// maps), from a process-wide pool in size classes of powers of two from
// 64 KB; a buffer goes back to the pool, never to the system.  *cls receives
// the class to give back; nullptr if page-locked memory is unavailable.
void *pinned_take(size_t bytes, size_t *cls);
void pinned_give(void *p, size_t cls);

}  // namespace mhs

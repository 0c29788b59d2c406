// kernels.h -- launchers shared by the host driver (mhs_api.cpp) and the
// CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "mhs_internal.h"

namespace mhs {

// Batch-wide totals of the last round, accumulated on the device and read
// back once per round (the round's only device-to-host transfer).
struct BatchCounters {
    int32_t active;           // instances still short of their fixpoint
    int32_t n_alive, m_alive; // summed over the batch
    int32_t dp_deleted, md_deleted;
    int32_t max_rounds_seen;
    int32_t changed_any;
    int32_t status_any;
    int32_t n_done;           // instances that reached their fixpoint in the last round
    int32_t loop_iters;       // rounds run by the device-side loop in this launch
    unsigned long long mma_kblocks;  // K steps of 64 contracted since load (tcgen05 path)
    unsigned long long mma_tiles;    // tiles contracted since load (tcgen05 path)
};

cudaError_t launch_validate(InstState *st, int count, cudaStream_t s);
// *out |= the OR of the instances' status words (the caller zeroes *out).
cudaError_t launch_status_or(const InstState *st, int count, int32_t *out, cudaStream_t s);
cudaError_t launch_localize_ptr(InstState *st, int count, const int64_t *gptr, const int64_t *e0,
                                cudaStream_t s);
cudaError_t launch_gather_bounds(const int64_t *gptr, const int64_t *e0, int64_t *out, int count,
                                 cudaStream_t s);
cudaError_t launch_build(InstState *st, int count, int32_t max_rounds, int64_t max_nnz,
                         int64_t max_m, int64_t max_n, cudaStream_t s);
// One phase of a round: phase 0 = DP (Algorithm 1), phase 1 = MD (Algorithm 2).
// done_list (may be NULL): receives the index of every instance that stops
// in this round (phase 1); ctr->n_done counts them.
// tile_n: columns per tcgen05 tile (128 or 256; the value in plan->tile_n).
cudaError_t launch_round_phase(InstState *st, Plan *plan, BatchCounters *ctr, int count,
                               int phase, int contraction, int sms, int32_t *kerr,
                               cudaStream_t s, cudaEvent_t ev_contract_begin,
                               cudaEvent_t ev_contract_end, int32_t *done_list = nullptr,
                               int compact_blocks = 1, int tile_n = kTcNDefault);
// The three parts of launch_round_phase, for a pass split into shares
// (mhs_pass_*): plan and set scatter; the contraction of share `shard` of
// `nshards` (the tile rows of 128-row blocks b with b % nshards == shard);
// the clear scatter (MD) and the compaction.
cudaError_t launch_phase_prologue(InstState *st, Plan *plan, BatchCounters *ctr, int phase,
                                  int contraction, int sms, cudaStream_t s);
cudaError_t launch_phase_contract(InstState *st, Plan *plan, BatchCounters *ctr, int phase,
                                  int contraction, int sms, int32_t *kerr, cudaStream_t s,
                                  int tile_n, int shard, int nshards);
cudaError_t launch_phase_epilogue(InstState *st, Plan *plan, BatchCounters *ctr, int count,
                                  int phase, int contraction, int sms, cudaStream_t s,
                                  int32_t *done_list, int compact_blocks);
// Copy a single instance's partial pass output to (import = 0) or from
// (import = 1) a buffer indexed by input id: uint8[m0] deletion flags
// (phase 0) or int32[n0] dominator counts (phase 1).
cudaError_t launch_pass_exchange(InstState *st, int phase, int import, void *buf, int sms,
                                 cudaStream_t s);
// End of one round of the device-side fixpoint loop: keep looping while
// some instance is active, no error was raised and fewer than round_cap
// rounds ran (hitting the cap raises kErrRoundCap).
cudaError_t launch_loop_cond(cudaGraphConditionalHandle h, BatchCounters *ctr, int32_t *kerr,
                             int32_t round_cap, cudaStream_t s);
// Rule FE for every instance that reached its DP/MD fixpoint in this round
// (after phase 1; fe.cu).  An instance FE changed runs more rounds; one it
// did not change is finished and goes to done_list.
cudaError_t launch_full_edges(InstState *st, int count, BatchCounters *ctr, int32_t *done_list,
                              int sms, cudaStream_t s);
cudaError_t launch_alive_masks(const InstState *st, uint8_t *alive_v, uint8_t *alive_e,
                               cudaStream_t s);

// ---- serving: the device-resident request loop (server.cpp) ----
// Host-mapped page-locked words shared by a lane's loop and its host thread.
struct ServerFlags {
    int32_t stop;      // host -> device: end the loop at its next round boundary
    int32_t kerr;      // device -> host: the loop's error bits
    uint32_t head;     // device -> host: slot indices published in `ring` so far (wraps)
    int32_t pad_;
    long long rounds;  // device -> host: rounds run over the lane's slot table
};
// Device-side bookkeeping of a lane's loop.
struct ServerDev {
    uint32_t head;     // slot indices published so far (wraps; the ring index is head % count)
    int32_t iters;     // iterations of the current launch
    long long rounds;
};
// Start of an iteration: every slot whose host-mapped ready flag is set
// enters the live table (its staged state, which the host has loaded and
// built, is copied in whole) and the flag is cleared.
cudaError_t launch_server_admit(InstState *live, const InstState *staged, int32_t *ready,
                                int count, cudaStream_t s);
// End of a round: the slots whose instance finished (done list) or failed
// (status bits) leave the live table: the state goes to `out` for the host,
// the live slot is zeroed, and the slot index is published in the
// host-mapped ring (capacity `count`) before `flags->head` advances.
cudaError_t launch_server_retire(InstState *live, InstState *out, const int32_t *done,
                                 const BatchCounters *ctr, int32_t *ring, ServerFlags *flags,
                                 ServerDev *dev, int count, cudaStream_t s);
// Loop condition: go on while the host has not asked to stop, no error was
// raised, fewer than `cap` iterations ran in this launch, and some slot is
// active or ready to enter.
cudaError_t launch_server_cond(cudaGraphConditionalHandle h, const BatchCounters *ctr,
                               const int32_t *kerr, const Plan *plan, ServerDev *dev,
                               ServerFlags *flags, const int32_t *ready, int count, int32_t cap,
                               cudaStream_t s);
cudaError_t launch_alive_masks_batch(const InstState *st, int count, uint8_t *alive_v,
                                     uint8_t *alive_e, cudaStream_t s);

// tcgen05 contraction (contract_tc.cu)
cudaError_t launch_tc_contract(InstState *st, Plan *plan, BatchCounters *ctr, int phase, int sms,
                               int tile_n, int32_t *kerr, cudaStream_t s);
// The tiles of phase `phase` that hold nonzero counts (or, in a DP pass of
// an instance with a hyperedge f > |e|, all tiles), into plan->tile_list.
// With nshards > 1 only the tiles of row blocks b with b % nshards == shard.
cudaError_t launch_tc_tile_list(InstState *st, Plan *plan, int phase, int sms, cudaStream_t s,
                                int shard = 0, int nshards = 1);
cudaError_t prepare_tc_contract();  // once per process, before any capture
// Row blocks per L2 group of the tile order (environment MHS_TILE_GROUP_ROWS,
// default 16); stored in Plan::group_rows.
int32_t tile_group_rows();
bool make_operand_tmap(void *out, const void *base, int64_t pitch, int64_t rows);
size_t tmap_bytes();

}  // namespace mhs

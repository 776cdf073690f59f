// rewl_kernels.h -- launch wrappers of the device phases (rewl_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "rewl_layout.h"

namespace rewl {

size_t sweep_smem_bytes(const Problem& P, int wpb, int G, int variant);
cudaError_t prepare_sweep(int G, int model);
cudaError_t launch_sweep(int G, const Problem& P, const DevState& S, const SweepLaunch& A, cudaStream_t st);
cudaError_t launch_exchange(const Problem& P, const DevState& S, cudaStream_t st);
cudaError_t launch_precompute(int G, const Problem& P, uint64_t t0, uint32_t n_att, uint32_t stride, PreTrial* out,
                              int max_blocks, cudaStream_t st);
cudaError_t launch_advance_clock(const DevState& S, uint32_t sweeps, cudaStream_t st);
cudaError_t launch_flat_merge(const Problem& P, const DevState& S, cudaStream_t st);
cudaError_t launch_init(const Problem& P, const DevState& S, cudaStream_t st);
cudaError_t launch_descent(const Problem& P, const DevState& S, uint64_t n_att, cudaStream_t st);
cudaError_t launch_entry(const Problem& P, const DevState& S, uint64_t budget, cudaStream_t st);

// served form (rewl_server.cu)
size_t ring_extra_smem();   // shared memory the ring form adds to a walker's CTA
size_t batch_smem_limit();  // dynamic shared memory a batched sweep CTA may use
cudaError_t prepare_sweep_batch();
// the walkers of d_list all belong to requests of one model (a shape group)
cudaError_t launch_round_batch(const BatchSlot* d_slots, int n_slots, const BatchWalker* d_list, int n_list,
                               size_t smem, int max_pairs, int max_m, int max_h, int form, int model,
                               cudaStream_t st);
// forms of the batched sweep: one walker per 32-lane CTA; the same with a producer warp
// (list of walkers); up to 4 walkers of one request per CTA, 8 lanes each (list of quads)
enum BatchForm : int { kBatchOne = 0, kBatchRing = 1, kBatchQuad = 2 };
cudaError_t launch_slot_report(const BatchSlot* d_slots, int n_slots, SlotReport* out, cudaStream_t st);

}  // namespace rewl

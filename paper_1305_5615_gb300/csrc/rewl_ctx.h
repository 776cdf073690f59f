// rewl_ctx.h -- the state of one solve behind a rewl_handle (internal to the
// library; shared by the single-solve runtime and the request server).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "rewl.h"
#include "rewl_layout.h"

using rewl::DevState;
using rewl::Problem;

struct rewl_ctx {
  Problem P{};
  DevState S{};
  rewl_params params{};
  double overlap = 0.0;
  int e_max = 0;
  std::vector<int32_t> win_start, win_width;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<void*> allocations;
  int G = 32, wpb = 1;
  int n_sm = 152;               // streaming multiprocessors of the device
  int n_active = 0;
  int n_done = 0;
  uint64_t sweep_clock = 0, xround = 0;
  uint64_t attempts = 0;        // WL trials of all walkers so far
  int32_t* h_n_done = nullptr;  // pinned
  cudaGraphExec_t graph = nullptr;
  int graph_n_active = -1;
  uint64_t h2d_bytes = 0, d2h_bytes = 0;
  // sweep-launch timing (params.profile): event pairs pending since the last sync
  std::vector<cudaEvent_t> ev_pool;
  int ev_pending = 0;
  int64_t sweep_launches = 0;
  double sweep_ms = 0.0;
  // draws of the next block prepared on a second stream (plain mode, when both buffers fit)
  bool pre_on = false;
  rewl::PreTrial* pre_buf[2] = {nullptr, nullptr};
  uint32_t pre_stride = 0;
  uint64_t pre_t0[2] = {~0ull, ~0ull};
  int pre_cur = 0;
  cudaStream_t pre_stream = nullptr;
  cudaEvent_t ev_pre[2] = {nullptr, nullptr};
  cudaEvent_t ev_used[2] = {nullptr, nullptr};

  ~rewl_ctx();
  void* dalloc(size_t bytes, rewl_status* st);
};

// Lets the other translation units of the library report through rewl_last_error.
void rewl_set_last_error(const char* msg);

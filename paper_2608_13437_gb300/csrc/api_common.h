// Helpers shared by the C-ABI translation units (single domains and batches).
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <string>

#include "lbm.h"
#include "lbm_internal.h"

namespace lbm {

// An NVTX range around an entry point (header-only NVTX v3: without a tool attached a
// push/pop costs a few nanoseconds), so profiler timelines show the library's phases.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

extern thread_local std::string g_last_error;
lbm_status fail(lbm_status s, const char* fmt, ...);
size_t elem_size(int store);
long long tile_count(long long ncell);
lbm_status validate(const lbm_params* p);
void derive(const lbm_params* p, double* dt, double* tau_R, double* tau_q);
void fill_const(const lbm_params* p, double dt, double tau_R, double tau_q, DomainConst* P);
cudaError_t launch_step(const DomainConst& P, int store, int parity, void* pop, const float* ghost,
                        unsigned* flag, int block_x, int variant, cudaStream_t s);
bool finite_pos(double v);

// Device state of a handle, for library code outside api.cu.
struct HandleView {
  const DomainConst* P;
  int store;
  long long step;
  double dt;
  const void* pop;
  const float* ghost;
  unsigned* flag;
  cudaStream_t stream;
  long long ncell;
};
HandleView handle_view(lbm_handle* h);
void latch_nonfinite(lbm_handle* h);
bool nonfinite_latched(const lbm_handle* h);
void latch_step_flag(lbm_handle* h, unsigned flag);  // bit 0 non-finite, bit 1 stalled copy
bool stall_latched(const lbm_handle* h);

}  // namespace lbm

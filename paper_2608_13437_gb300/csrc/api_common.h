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

// Makes `device` the calling thread's current CUDA device for the lifetime of the
// object and restores the caller's current device afterwards, so every entry point
// issues its work in the context of the device its handle was created on, whatever
// device the caller has current. ok() is false if either device query or switch
// failed (the message is then in error()).
class DeviceScope {
 public:
  explicit DeviceScope(int device) {
    err_ = cudaGetDevice(&prev_);
    if (err_ == cudaSuccess && prev_ != device) {
      err_ = cudaSetDevice(device);
      switched_ = err_ == cudaSuccess;
    }
    if (err_ != cudaSuccess) cudaGetLastError();
  }
  ~DeviceScope() {
    if (switched_) cudaSetDevice(prev_);
  }
  bool ok() const { return err_ == cudaSuccess; }
  const char* error() const { return cudaGetErrorString(err_); }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;

 private:
  int prev_ = -1;
  bool switched_ = false;
  cudaError_t err_ = cudaSuccess;
};

// Opens a DeviceScope for `dev` and returns LBM_E_CUDA from the enclosing entry point
// if the device cannot be made current.
#define LBM_ON_DEVICE(dev)                                                                   \
  ::lbm::DeviceScope lbm_device_scope_(dev);                                                 \
  if (!lbm_device_scope_.ok())                                                              \
  return ::lbm::fail(LBM_E_CUDA, "cannot make device %d current: %s", (int)(dev),            \
                     lbm_device_scope_.error())

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
  int device;  // CUDA device the handle was created on
};
HandleView handle_view(lbm_handle* h);
// Fills *out from the reduced diagnostic values r[0..kDiagA + 2) of the state after
// `step` steps, latches the step flag and the non-finite count, and returns the
// handle's sticky status (LBM_E_TIMEOUT, LBM_E_NONFINITE or LBM_OK).
lbm_status finish_diag(lbm_handle* h, const double* r, unsigned flag, long long step,
                       lbm_diag_t* out);

}  // namespace lbm

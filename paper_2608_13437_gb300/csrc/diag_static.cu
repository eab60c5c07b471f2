// lbm_diag_static: the diagnostics of lbm_diag computed without allocating any
// memory, for callers that must not allocate device memory at the time they ask
// for diagnostics.
//
// Who needs this: lbm_diag allocates its scratch (four doubles per cell, plus
// per-block partial sums) the first time it is called on a handle. Some callers
// cannot allow that allocation when they sample diagnostics: an application whose
// memory pool has already reserved all free device memory (cudaMalloc fails with
// out-of-memory), a solver loop that must not pay the device-wide synchronisation
// that cudaMalloc and cudaFree imply, or code that owns a fixed memory budget set
// up front. Those callers create their handles while allocation is still allowed
// and use this entry point afterwards.
//
// How: the scratch is one file-scope device array of fixed size, enough for
// domains of up to kStaticDiagMaxCells cells. It is part of the library image, so
// it exists on every device that loads the library and stays until the process
// exits. Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with the
// handle's device made current) and caches it; that first call should therefore come
// before any stream capture. A cached address does not survive cudaDeviceReset. All calls share the array and the kernels write every element
// they later read within the same call, so no clearing is needed between calls;
// two calls whose kernels overlap on the GPU (for instance from different streams
// or threads) race on the array and must be serialised by the caller.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "api_common.h"

namespace lbm {
namespace {

constexpr long long kStaticDiagMaxCells = 262144;  // 64^3
constexpr long long kStaticU = 2 * kStaticDiagMaxCells;  // u and mu_local: 4 floats per cell
constexpr long long kStaticPartials = (long long)kDiagBlocks * (kDiagA + 2);
constexpr long long kStaticOut = 16;
constexpr long long kStaticDoubles = kStaticU + kStaticPartials + kStaticOut;

// About 4.2 MiB of device memory per device.
static __device__ __align__(256) double g_static_diag_scratch[kStaticDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on device `dev`, which the caller has made
// current (looked up once per device).
lbm_status scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(LBM_E_INVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_diag_scratch);
    if (e != cudaSuccess || !ptr)
      return fail(LBM_E_CUDA, "cudaGetSymbolAddress of the diagnostic scratch failed: %s",
                  cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double*>(ptr);
  }
  *out = g_scratch_addr[dev];
  return LBM_OK;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" lbm_status lbm_diag_static(lbm_handle* h, lbm_diag_t* out) {
  Range range_("lbm_diag_static");
  if (!h || !out) return fail(LBM_E_INVAL, "NULL argument");
  const HandleView v = handle_view(h);
  if (v.ncell > kStaticDiagMaxCells)
    return fail(LBM_E_INVAL,
                "lbm_diag_static handles at most %lld cells (64^3); this domain has %lld cells "
                "(use lbm_diag)", kStaticDiagMaxCells, v.ncell);
  // the array and its address belong to the handle's device, whatever device the
  // caller has current
  LBM_ON_DEVICE(v.device);
  double* base = nullptr;
  lbm_status s = scratch_address(v.device, &base);
  if (s != LBM_OK) return s;
  float* ufield = reinterpret_cast<float*>(base);
  double* partials = base + kStaticU;
  double* dout = partials + kStaticPartials;
  // The scratch is sized for kStaticDiagMaxCells; the kernels index it by this
  // domain's cell count, which was checked above.
  cudaError_t e = launch_diag(*v.P, v.store, (int)(v.step & 1), v.pop, v.ghost, ufield, partials,
                              dout, v.stream);
  double r[16] = {0};
  unsigned flag = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r, dout, sizeof(double) * (kDiagA + 2), cudaMemcpyDeviceToHost, v.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, v.flag, sizeof(flag), cudaMemcpyDeviceToHost, v.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
  if (e != cudaSuccess) return fail(LBM_E_CUDA, "static diagnostics failed: %s", cudaGetErrorString(e));
  return finish_diag(h, r, flag, v.step, out);
}

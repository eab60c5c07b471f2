// C ABI of liblbm.so for single domains: validation, device state, CUDA-graph
// replay of the fused step, initial states, outputs, checkpoints, autotuning.
// The declarations and their documentation are in include/lbm.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "api_common.h"

using namespace lbm;

namespace lbm {

thread_local std::string g_last_error;

lbm_status fail(lbm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

size_t elem_size(int store) { return store == LBM_STORE_F32 ? 4 : 2; }

long long tile_count(long long ncell) { return (ncell + kTile - 1) / kTile; }

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }
bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

lbm_status validate(const lbm_params* p) {
  if (!p) return fail(LBM_E_INVAL, "params is NULL");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1)
    return fail(LBM_E_INVAL, "grid %d x %d x %d: every size must be >= 1", p->nx, p->ny, p->nz);
  const long long n = (long long)p->nx * p->ny * p->nz;
  if (n >= (1LL << 31)) return fail(LBM_E_INVAL, "grid has %lld cells; at most 2^31 - 1", n);
  if (p->ny > 65535 || p->nz > 65535) return fail(LBM_E_INVAL, "ny and nz must be <= 65535");
  if (!finite_pos(p->dx)) return fail(LBM_E_INVAL, "dx must be finite and > 0");
  if (!(p->dt > 0) && !(finite_pos(p->cfl) && finite_pos(p->lambda_ref)))
    return fail(LBM_E_INVAL, "need dt > 0, or cfl > 0 and lambda_ref > 0");
  if (p->dt > 0 && !std::isfinite(p->dt)) return fail(LBM_E_INVAL, "dt must be finite");
  if (!(std::isfinite(p->gamma) && p->gamma > 1.0)) return fail(LBM_E_INVAL, "gamma must be > 1");
  if (!finite_nonneg(p->mu) || !finite_nonneg(p->kappa))
    return fail(LBM_E_INVAL, "mu and kappa must be finite and >= 0");
  if (!(p->tau_R > 0) || !(p->tau_q > 0) || std::isnan(p->tau_R) || std::isnan(p->tau_q))
    return fail(LBM_E_INVAL, "tau_R and tau_q must be > 0");
  if (!finite_pos(p->T_ref)) return fail(LBM_E_INVAL, "T_ref must be finite and > 0");
  if (!finite_nonneg(p->f_mu) || !finite_nonneg(p->C_sigma) || !finite_nonneg(p->J_min))
    return fail(LBM_E_INVAL, "f_mu, C_sigma and J_min must be finite and >= 0");
  if (!(p->omega_min > 0.0 && p->omega_min <= 2.0))
    return fail(LBM_E_INVAL, "omega_min must lie in (0, 2]");
  if (p->store < 0 || p->store > 2) return fail(LBM_E_INVAL, "store must be 0, 1 or 2");
  if (p->stochastic_round < 0 || p->stochastic_round > 1)
    return fail(LBM_E_INVAL, "stochastic_round must be 0 or 1");
  if (p->bc_x < 0 || p->bc_x > 1) return fail(LBM_E_INVAL, "bc_x must be 0 or 1");
  if (p->source_mode < 0 || p->source_mode > 1) return fail(LBM_E_INVAL, "source_mode must be 0 or 1");
  if (p->sensor_mode < 0 || p->sensor_mode > 1) return fail(LBM_E_INVAL, "sensor_mode must be 0 or 1");
  if (p->collide < 0 || p->collide > 1) return fail(LBM_E_INVAL, "collide must be 0 or 1");
  if (p->streaming < 0 || p->streaming > 1) return fail(LBM_E_INVAL, "streaming must be 0 or 1");
  if (p->pop_buffer && (reinterpret_cast<uintptr_t>(p->pop_buffer) & 255u))
    return fail(LBM_E_INVAL, "pop_buffer must be 256-byte aligned");
  return LBM_OK;
}

// Derived time step and relaxation times (Table 1; Sec. 3.1 for relax_in_dt).
void derive(const lbm_params* p, double* dt, double* tau_R, double* tau_q) {
  *dt = p->dt > 0 ? p->dt : p->cfl * 0.5 * p->dx / p->lambda_ref;
  *tau_R = p->relax_in_dt ? p->tau_R * *dt : p->tau_R;
  *tau_q = p->relax_in_dt ? p->tau_q * *dt : p->tau_q;
}

void fill_const(const lbm_params* p, double dt, double tau_R, double tau_q, DomainConst* P) {
  std::memset(P, 0, sizeof(*P));
  P->nx = p->nx;
  P->ny = p->ny;
  P->nz = p->nz;
  P->bc_x = p->bc_x;
  P->ncell = (long long)p->nx * p->ny * p->nz;
  P->ntile = tile_count(P->ncell);
  const double c = p->dx / dt;
  P->c = (float)c;
  P->inv_c = (float)(1.0 / c);
  P->half_inv_c = (float)(0.5 / c);
  P->dt = (float)dt;
  P->gm1 = (float)(p->gamma - 1.0);
  P->gamma = (float)p->gamma;
  P->mu = (float)p->mu;
  P->visc0 = (float)(p->mu / tau_R);
  P->heat0 = (float)(p->kappa / tau_q);
  P->inv_T_ref = (float)(1.0 / p->T_ref);
  P->fmu_coef = (float)(4.0 * p->f_mu * dt / (p->dx * p->dx));
  P->C_sigma = (float)p->C_sigma;
  P->J_min = (float)p->J_min;
  P->omega_min = (float)p->omega_min;
  // Source increment per step (Sec. 2.2): explicit dt S_k or exact relaxation.
  P->src_R = (float)(p->source_mode ? std::expm1(-dt / tau_R) : -dt / tau_R);
  P->src_q = (float)(p->source_mode ? std::expm1(-dt / tau_q) : -dt / tau_q);
  for (int k = 0; k < kF; ++k) P->scale[k] = P->inv_scale[k] = 1.0f;
  P->sutherland = p->sutherland;
  P->sensor_mode = p->sensor_mode;
  P->collide = p->collide;
  P->sround = p->stochastic_round;
  P->eso = p->streaming;
  P->dx64 = p->dx;
}

cudaError_t launch_step(const DomainConst& P, int store, int parity, void* pop, const float* ghost,
                        unsigned* flag, int block_x, int variant, cudaStream_t s) {
  switch (store) {
    case LBM_STORE_F32: return launch_step_f32(P, parity, pop, ghost, flag, block_x, variant, s);
    case LBM_STORE_F16: return launch_step_f16(P, parity, pop, ghost, flag, block_x, variant, s);
    default: return launch_step_bf16(P, parity, pop, ghost, flag, block_x, variant, s);
  }
}

cudaError_t staged_prepare(const DomainConst& P, int store, int variant, int* grid) {
  switch (store) {
    case LBM_STORE_F32: return staged_prepare_f32(P, variant, grid);
    case LBM_STORE_F16: return staged_prepare_f16(P, variant, grid);
    default: return staged_prepare_bf16(P, variant, grid);
  }
}

cudaError_t launch_step_staged(const DomainConst& P, int store, int parity, void* pop, unsigned* flag,
                               int variant, int grid, int skip_first, cudaStream_t s) {
  switch (store) {
    case LBM_STORE_F32: return launch_step_staged_f32(P, parity, pop, flag, variant, grid, skip_first, s);
    case LBM_STORE_F16: return launch_step_staged_f16(P, parity, pop, flag, variant, grid, skip_first, s);
    default: return launch_step_staged_bf16(P, parity, pop, flag, variant, grid, skip_first, s);
  }
}

cudaError_t launch_step_diag(const DomainConst& P, int store, int parity, void* pop,
                             const float* ghost, unsigned* flag, float* ufield, float* rec,
                             int block_x, cudaStream_t s) {
  switch (store) {
    case LBM_STORE_F32:
      return launch_step_diag_f32(P, parity, pop, ghost, flag, ufield, rec, block_x, s);
    case LBM_STORE_F16:
      return launch_step_diag_f16(P, parity, pop, ghost, flag, ufield, rec, block_x, s);
    default: return launch_step_diag_bf16(P, parity, pop, ghost, flag, ufield, rec, block_x, s);
  }
}

}  // namespace lbm

struct lbm_handle {
  lbm_params prm;
  int device = 0;              // CUDA device current at lbm_create; every call runs there
  DomainConst P;
  double dt = 0, tau_R = 0, tau_q = 0;
  double rho_ref = 0, E_ref = 0;
  double scale[kF];
  long long ncell = 0;
  size_t pop_bytes = 0;
  void* pop = nullptr;
  bool own_pop = false;
  float* ghost = nullptr;      // [2][14][ny*nz]
  unsigned* flag = nullptr;    // non-finite flag (device)
  unsigned* maxbits = nullptr; // per-field max |deviation| (device)
  double* sums = nullptr;      // field means (device)
  float* trig = nullptr;       // TGV table: sin, cos, cos 2x of the nodes of each axis (device)
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // capture-only stream
  long long step = 0;
  bool initialized = false;
  bool nonfinite = false;
  int block_x = 64;
  int variant = 0;             // step kernel: register budget (0, 1) or staged form (2-4)
  int staged_grid = 0;         // persistent grid of the staged forms
  bool stalled = false;        // a staged step gave up waiting for a bulk copy
  bool skip_next_copy = false; // test hook: the next direct staged step skips one copy
  cudaGraphExec_t g_pair = nullptr, g_chunk = nullptr;
  bool graphs_valid = false;
  float* ufield = nullptr;     // diagnostics scratch: 4 floats per cell
  double* partials = nullptr;
  double* dout = nullptr;
  float* wrec = nullptr;       // per-warp records of the diagnostic step
  long long wrec_n = 0;
  double* hdiag = nullptr;     // pinned host copy of dout and the flag
  void* stage = nullptr;       // device staging for host-side outputs (kStageBytes)
  cudaEvent_t ev_diag = nullptr;
};

namespace {

constexpr int kChunkPairs = 16;  // a chunk graph holds 32 steps

#define LBM_CUDA(expr)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(LBM_E_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));                \
  } while (0)

void drop_graphs(lbm_handle* h) {
  if (h->g_pair) cudaGraphExecDestroy(h->g_pair);
  if (h->g_chunk) cudaGraphExecDestroy(h->g_chunk);
  h->g_pair = h->g_chunk = nullptr;
  h->graphs_valid = false;
}

int effective_block(const lbm_handle* h) {
  int b = h->block_x;
  const int need = ((h->P.nx + 31) / 32) * 32;
  return b > need ? need : b;
}

cudaError_t step_launch(lbm_handle* h, int parity, cudaStream_t s) {
  if (h->variant >= kFirstStagedVariant)
    return launch_step_staged(h->P, h->prm.store, parity, h->pop, h->flag, h->variant,
                              h->staged_grid, 0, s);
  return launch_step(h->P, h->prm.store, parity, h->pop, h->ghost, h->flag, effective_block(h),
                     h->variant, s);
}

// Flag bits written by the step kernels: 1 = a non-finite moment, 2 = a staged step
// gave up waiting for a bulk copy (its state is then incomplete).
void latch_flag(lbm_handle* h, unsigned flag) {
  if (flag & 1u) h->nonfinite = true;
  if (flag & 2u) h->stalled = true;
}

lbm_status capture(lbm_handle* h, int pairs, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  LBM_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  for (int j = 0; j < 2 * pairs && le == cudaSuccess; ++j)
    le = step_launch(h, j & 1, h->cap);
  cudaError_t ee = cudaStreamEndCapture(h->cap, &g);
  if (le != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(LBM_E_CUDA, "graph capture failed: %s",
                cudaGetErrorString(le != cudaSuccess ? le : ee));
  }
  cudaError_t ie = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return fail(LBM_E_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ie));
  return LBM_OK;
}

lbm_status ensure_graphs(lbm_handle* h) {
  if (h->graphs_valid) return LBM_OK;
  drop_graphs(h);
  lbm_status s = capture(h, 1, &h->g_pair);
  if (s != LBM_OK) return s;
  s = capture(h, kChunkPairs, &h->g_chunk);
  if (s != LBM_OK) return s;
  h->graphs_valid = true;
  return LBM_OK;
}

lbm_status direct_step(lbm_handle* h) {
  if (h->skip_next_copy && h->variant >= kFirstStagedVariant) {
    h->skip_next_copy = false;
    LBM_CUDA(launch_step_staged(h->P, h->prm.store, (int)(h->step & 1), h->pop, h->flag, h->variant,
                                h->staged_grid, 1, h->stream));
  } else {
    LBM_CUDA(step_launch(h, (int)(h->step & 1), h->stream));
  }
  h->step += 1;
  return LBM_OK;
}

void reset_scales(lbm_handle* h) {
  for (int k = 0; k < kF; ++k) {
    h->scale[k] = 1.0;
    h->P.scale[k] = h->P.inv_scale[k] = 1.0f;
  }
}

// The storage reference Q_ref = (rho_ref, 0, 0, 0, E_ref, 0...) as the device uses it
// (FP32); the handle reports the same values.
void set_reference(lbm_handle* h, double rho_ref, double E_ref) {
  h->P.rho_ref = (float)rho_ref;
  h->P.E_ref = (float)E_ref;
  h->rho_ref = (double)h->P.rho_ref;
  h->E_ref = (double)h->P.E_ref;
}

// Runs both init passes for an initial state: Q_ref must be set beforehand.
lbm_status run_init(lbm_handle* h, InitSpec& sp) {
  reset_scales(h);
  if (h->prm.store == LBM_STORE_F16) {
    LBM_CUDA(cudaMemsetAsync(h->maxbits, 0, kF * sizeof(unsigned), h->stream));
    LBM_CUDA(launch_init(h->P, h->prm.store, sp, 0, h->pop, h->ghost, h->maxbits, nullptr, h->stream));
    unsigned bits[kF];
    LBM_CUDA(cudaMemcpyAsync(bits, h->maxbits, sizeof(bits), cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < kF; ++k) {
      float m;
      std::memcpy(&m, &bits[k], sizeof(m));
      // |g| <= 1024 at init: 64x headroom below the largest half, and far above
      // the smallest normal half.
      const float sk = (std::isfinite(m) && m > 0.0f) ? m / 1024.0f : 1.0f;
      h->P.scale[k] = sk;
      h->P.inv_scale[k] = 1.0f / sk;
      h->scale[k] = sk;
    }
  }
  // word 3 of the flag block: set by the kernel if the initial state is not finite
  LBM_CUDA(cudaMemsetAsync(h->flag + 3, 0, sizeof(unsigned), h->stream));
  LBM_CUDA(launch_init(h->P, h->prm.store, sp, 1, h->pop, h->ghost, nullptr, h->flag + 3, h->stream));
  LBM_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(unsigned), h->stream));
  unsigned bad = 0;
  LBM_CUDA(cudaMemcpyAsync(&bad, h->flag + 3, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  if (bad) {
    h->initialized = false;
    h->graphs_valid = false;
    return fail(LBM_E_INVAL, "the initial state has non-finite values");
  }
  h->step = 0;
  h->initialized = true;
  h->nonfinite = false;
  h->stalled = false;
  h->graphs_valid = false;
  return LBM_OK;
}

// Host <-> device staging for outputs: at most this many bytes per temporary.
constexpr size_t kStageBytes = 256u << 20;

}  // namespace

extern "C" {

size_t lbm_population_bytes(const lbm_params* p) {
  if (!p || p->nx < 1 || p->ny < 1 || p->nz < 1 || p->store < 0 || p->store > 2) return 0;
  const long long n = (long long)p->nx * p->ny * p->nz;
  if (n >= (1LL << 31)) return 0;
  return (size_t)tile_count(n) * kP * kTile * elem_size(p->store);
}

const char* lbm_last_error(void) { return g_last_error.c_str(); }

const char* lbm_status_string(lbm_status s) {
  switch (s) {
    case LBM_OK: return "LBM_OK";
    case LBM_E_INVAL: return "LBM_E_INVAL";
    case LBM_E_NOMEM: return "LBM_E_NOMEM";
    case LBM_E_CUDA: return "LBM_E_CUDA";
    case LBM_E_NONFINITE: return "LBM_E_NONFINITE";
    case LBM_E_STATE: return "LBM_E_STATE";
    case LBM_E_IO: return "LBM_E_IO";
    case LBM_E_TIMEOUT: return "LBM_E_TIMEOUT";
  }
  return "unknown status";
}

lbm_status lbm_create(const lbm_params* p, lbm_handle** out) {
  if (!out) return fail(LBM_E_INVAL, "out is NULL");
  *out = nullptr;
  lbm_status s = validate(p);
  if (s != LBM_OK) return s;
  int device = 0;
  {
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(LBM_E_CUDA, "no current CUDA device: %s", cudaGetErrorString(e));
    }
  }
  lbm_handle* h = new (std::nothrow) lbm_handle();
  if (!h) return fail(LBM_E_NOMEM, "host allocation failed");
  h->prm = *p;
  h->device = device;
  derive(p, &h->dt, &h->tau_R, &h->tau_q);
  if (!(h->dt > 0) || !std::isfinite(h->dt)) {
    delete h;
    return fail(LBM_E_INVAL, "derived dt is not a positive finite number");
  }
  fill_const(p, h->dt, h->tau_R, h->tau_q, &h->P);
  h->P.pf_tiles = p->store == LBM_STORE_F32 ? 0 : kDefaultPrefetch16;
  // Measured on GB300 at 512^3: blocks of 64 threads and the 170-register budget for
  // every storage type (with its L2 prefetch the 16-bit step no longer gains from the
  // higher occupancy of the 128-register budget); lbm_autotune re-times.
  h->block_x = 64;
  h->variant = 0;
  h->ncell = h->P.ncell;
  h->pop_bytes = lbm_population_bytes(p);
  for (int k = 0; k < kF; ++k) h->scale[k] = 1.0;
  h->stream = static_cast<cudaStream_t>(p->cuda_stream);
  auto cleanup = [&](lbm_status st) {
    lbm_destroy(h);
    return st;
  };
  if (p->pop_buffer) {
    h->pop = p->pop_buffer;
  } else {
    cudaError_t e = cudaMalloc(&h->pop, h->pop_bytes);
    if (e != cudaSuccess) {
      h->pop = nullptr;
      cudaGetLastError();
      return cleanup(fail(LBM_E_NOMEM, "cudaMalloc of %zu population bytes failed: %s", h->pop_bytes,
                          cudaGetErrorString(e)));
    }
    h->own_pop = true;
  }
  const size_t ghost_bytes = sizeof(float) * 2 * kF * (size_t)p->ny * p->nz;
  if (cudaMalloc(&h->ghost, ghost_bytes) != cudaSuccess || cudaMalloc(&h->flag, 64) != cudaSuccess ||
      cudaMalloc(&h->maxbits, 64 + kF * sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&h->sums, kFieldSumDoubles * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->trig, sizeof(float) * tgv_table_floats(p->nx, p->ny, p->nz)) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(LBM_E_NOMEM, "cudaMalloc of small device buffers failed"));
  }
  if (cudaMemset(h->ghost, 0, ghost_bytes) != cudaSuccess || cudaMemset(h->flag, 0, 64) != cudaSuccess)
    return cleanup(fail(LBM_E_CUDA, "cudaMemset failed"));
  h->P.check = h->flag + 2;  // word 2 of the flag block: the checked build's address count
  if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess)
    return cleanup(fail(LBM_E_CUDA, "cudaStreamCreate failed"));
  *out = h;
  return LBM_OK;
}

lbm_status lbm_destroy(lbm_handle* h) {
  if (!h) return LBM_OK;
  DeviceScope scope(h->device);  // best effort: release what can be released either way
  if (h->stream || h->pop) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  if (h->own_pop && h->pop) cudaFree(h->pop);
  if (h->ghost) cudaFree(h->ghost);
  if (h->flag) cudaFree(h->flag);
  if (h->maxbits) cudaFree(h->maxbits);
  if (h->sums) cudaFree(h->sums);
  if (h->trig) cudaFree(h->trig);
  if (h->ufield) cudaFree(h->ufield);
  if (h->partials) cudaFree(h->partials);
  if (h->dout) cudaFree(h->dout);
  if (h->wrec) cudaFree(h->wrec);
  if (h->stage) cudaFree(h->stage);
  if (h->hdiag) cudaFreeHost(h->hdiag);
  if (h->ev_diag) cudaEventDestroy(h->ev_diag);
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
  return LBM_OK;
}

lbm_status lbm_get_info(const lbm_handle* h, lbm_info_t* out) {
  if (!h || !out) return fail(LBM_E_INVAL, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->dt = h->dt;
  out->c = h->prm.dx / h->dt;
  out->tau_R = h->tau_R;
  out->tau_q = h->tau_q;
  out->rho_ref = h->rho_ref;
  out->E_ref = h->E_ref;
  for (int k = 0; k < kF; ++k) out->scale[k] = h->scale[k];
  out->step = h->step;
  out->ncell = h->ncell;
  out->population_bytes = h->pop_bytes;
  out->store = h->prm.store;
  out->block_x = effective_block(h);
  out->variant = h->variant;
  out->prefetch_tiles = h->P.pf_tiles;
  out->device = h->device;
  return LBM_OK;
}

lbm_status lbm_init_tgv(lbm_handle* h, double U0, double M0, double rho0) {
  Range range_("lbm_init_tgv");
  if (!h) return fail(LBM_E_INVAL, "handle is NULL");
  LBM_ON_DEVICE(h->device);
  if (!(std::isfinite(U0) && finite_pos(M0) && finite_pos(rho0)))
    return fail(LBM_E_INVAL, "TGV needs finite U0 and M0, rho0 > 0");
  const double p0 = rho0 * U0 * U0 / (h->prm.gamma * M0 * M0);
  if (!finite_pos(p0)) return fail(LBM_E_INVAL, "TGV background pressure must be > 0 (U0 != 0)");
  set_reference(h, rho0, p0 / (h->prm.gamma - 1.0));
  InitSpec sp;
  std::vector<float> table;
  tgv_spec(h->P, h->prm.gamma, U0, M0, rho0, h->prm.dx, &sp, &table);
  // pageable source: the call returns once the table is staged, in stream order
  LBM_CUDA(cudaMemcpyAsync(h->trig, table.data(), sizeof(float) * table.size(),
                           cudaMemcpyHostToDevice, h->stream));
  sp.trig = h->trig;
  return run_init(h, sp);
}

lbm_status lbm_init_riemann(lbm_handle* h, int axis, int i_split, const double left[3],
                            const double right[3]) {
  Range range_("lbm_init_riemann");
  if (!h || !left || !right) return fail(LBM_E_INVAL, "NULL argument");
  LBM_ON_DEVICE(h->device);
  if (axis < 0 || axis > 2) return fail(LBM_E_INVAL, "axis must be 0, 1 or 2");
  for (int j = 0; j < 3; ++j)
    if (!std::isfinite(left[j]) || !std::isfinite(right[j])) return fail(LBM_E_INVAL, "non-finite state");
  if (!(left[0] > 0 && right[0] > 0 && left[2] > 0 && right[2] > 0))
    return fail(LBM_E_INVAL, "densities and pressures must be > 0");
  set_reference(h, right[0], right[2] / (h->prm.gamma - 1.0) + 0.5 * right[0] * right[1] * right[1]);
  InitSpec sp;
  riemann_spec(h->P, h->prm.gamma, axis, i_split, left, right, &sp);
  return run_init(h, sp);
}

// Page-locked host memory (cudaHostAlloc, cudaHostRegister) is mapped into the GPU's
// address space, so kernels read and write it directly over the CPU-GPU link
// (NVLink-C2C between Grace and the GPU): host inputs and outputs in such memory need
// no device staging buffer and no separate copy. Returns the device address of a
// page-locked buffer, or nullptr for pageable memory and for a pointer that is not a
// multiple of `align` (those take the staged path).
static void* mapped_host(const void* p, size_t align) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  if (reinterpret_cast<uintptr_t>(a.devicePointer) % align) return nullptr;
  return a.devicePointer;
}

static lbm_status init_from_fields(lbm_handle* h, const void* fields, int src_on_device, int dtype,
                                   int kind, int nfield) {
  Range range_("lbm_init_fields");
  if (!h || !fields) return fail(LBM_E_INVAL, "NULL argument");
  LBM_ON_DEVICE(h->device);
  if (dtype != LBM_DT_F32 && dtype != LBM_DT_F64) return fail(LBM_E_INVAL, "dtype must be F32 or F64");
  const size_t bytes = (size_t)nfield * h->ncell * (dtype == LBM_DT_F64 ? 8 : 4);
  void* dev = const_cast<void*>(fields);
  void* tmp = nullptr;
  void* mapped = src_on_device ? nullptr : mapped_host(fields, dtype == LBM_DT_F64 ? 8 : 4);
  if (mapped) {
    dev = mapped;  // page-locked: the kernels read it directly
  } else if (!src_on_device) {
    if (cudaMalloc(&tmp, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(LBM_E_NOMEM, "cudaMalloc of %zu staging bytes failed", bytes);
    }
    cudaError_t e = cudaMemcpyAsync(tmp, fields, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) {
      cudaFree(tmp);
      return fail(LBM_E_CUDA, "copy of initial fields failed: %s", cudaGetErrorString(e));
    }
    dev = tmp;
  }
  InitSpec sp;
  fields_spec(h->prm.gamma, kind, dev, dtype == LBM_DT_F64, &sp);
  lbm_status st = LBM_OK;
  double sums[2] = {0, 0};
  cudaError_t e = launch_field_means(h->P, sp, h->sums, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sums, h->sums, sizeof(sums), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    st = fail(LBM_E_CUDA, "field means failed: %s", cudaGetErrorString(e));
  } else {
    const double cnt = (double)field_sample(h->ncell).cells;
    const double rho_ref = sums[0] / cnt, E_ref = sums[1] / cnt;
    if (!std::isfinite(rho_ref) || !std::isfinite(E_ref)) {
      st = fail(LBM_E_INVAL, "initial fields contain non-finite values");
    } else {
      set_reference(h, rho_ref, E_ref);
      st = run_init(h, sp);
    }
  }
  if (tmp) cudaFree(tmp);
  return st;
}

lbm_status lbm_init_fields(lbm_handle* h, const void* fields, int src_on_device, int dtype) {
  return init_from_fields(h, fields, src_on_device, dtype, 2, 5);
}

lbm_status lbm_init_state(lbm_handle* h, const void* Q, int src_on_device, int dtype) {
  return init_from_fields(h, Q, src_on_device, dtype, 3, kF);
}

lbm_status lbm_step(lbm_handle* h, int n) {
  Range range_("lbm_step");
  if (!h) return fail(LBM_E_INVAL, "handle is NULL");
  LBM_ON_DEVICE(h->device);
  if (n < 0) return fail(LBM_E_INVAL, "n must be >= 0");
  if (!h->initialized) return fail(LBM_E_STATE, "lbm_step before an init");
  if (h->nonfinite) return fail(LBM_E_NONFINITE, "non-finite moments were detected earlier");
  if (h->stalled) return fail(LBM_E_TIMEOUT, "a staged step gave up waiting for a bulk copy; re-init");
  if (n == 0) return LBM_OK;
  if (!h->prm.use_graphs) {
    for (int j = 0; j < n; ++j) {
      lbm_status s = direct_step(h);
      if (s != LBM_OK) return s;
    }
    return LBM_OK;
  }
  if (h->skip_next_copy) {  // the test hook needs a direct launch
    lbm_status s0 = direct_step(h);
    if (s0 != LBM_OK || --n == 0) return s0;
  }
  lbm_status s = ensure_graphs(h);
  if (s != LBM_OK) return s;
  if (h->step & 1) {
    s = direct_step(h);
    if (s != LBM_OK) return s;
    --n;
  }
  while (n >= 2 * kChunkPairs) {
    LBM_CUDA(cudaGraphLaunch(h->g_chunk, h->stream));
    h->step += 2 * kChunkPairs;
    n -= 2 * kChunkPairs;
  }
  while (n >= 2) {
    LBM_CUDA(cudaGraphLaunch(h->g_pair, h->stream));
    h->step += 2;
    n -= 2;
  }
  if (n) return direct_step(h);
  return LBM_OK;
}

lbm_status lbm_synchronize(lbm_handle* h) {
  if (!h) return fail(LBM_E_INVAL, "handle is NULL");
  LBM_ON_DEVICE(h->device);
  unsigned flag = 0;
  LBM_CUDA(cudaMemcpyAsync(&flag, h->flag, sizeof(flag), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  latch_flag(h, flag);
  if (h->stalled) return fail(LBM_E_TIMEOUT, "a staged step gave up waiting for a bulk copy; re-init");
  if (h->nonfinite) return fail(LBM_E_NONFINITE, "non-finite moments detected");
  return LBM_OK;
}

// The handle's device staging buffer for outputs written to host memory, allocated on
// first use and kept (no allocation or implicit device synchronisation per call).
static lbm_status ensure_stage(lbm_handle* h) {
  if (h->stage) return LBM_OK;
  if (cudaMalloc(&h->stage, kStageBytes) != cudaSuccess) {
    cudaGetLastError();
    h->stage = nullptr;
    return fail(LBM_E_NOMEM, "staging allocation failed");
  }
  return LBM_OK;
}

lbm_status lbm_moments(lbm_handle* h, int which, void* dst, int dst_on_device, int dtype) {
  Range range_("lbm_moments");
  if (!h || !dst) return fail(LBM_E_INVAL, "NULL argument");
  LBM_ON_DEVICE(h->device);
  if (which != LBM_MOM_Q && which != LBM_MOM_PRIM) return fail(LBM_E_INVAL, "bad moment set");
  if (dtype != LBM_DT_F32 && dtype != LBM_DT_F64) return fail(LBM_E_INVAL, "dtype must be F32 or F64");
  const int nf = which == LBM_MOM_Q ? kF : 6;
  const size_t es = dtype == LBM_DT_F64 ? 8 : 4;
  const int parity = (int)(h->step & 1);
  if (dst_on_device) {
    LBM_CUDA(launch_moments(h->P, h->prm.store, parity, h->pop, h->ghost, which, dst,
                            dtype == LBM_DT_F64, 0, h->ncell, h->stream));
    return LBM_OK;
  }
  if (void* m = mapped_host(dst, es)) {  // page-locked: the kernel writes it directly
    cudaError_t e = launch_moments(h->P, h->prm.store, parity, h->pop, h->ghost, which, m,
                                   dtype == LBM_DT_F64, 0, h->ncell, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(LBM_E_CUDA, "moments failed: %s", cudaGetErrorString(e));
    return LBM_OK;
  }
  long long chunk = (long long)(kStageBytes / (es * nf));
  if (chunk > h->ncell) chunk = h->ncell;
  lbm_status st = ensure_stage(h);
  if (st != LBM_OK) return st;
  void* tmp = h->stage;
  cudaError_t e = cudaSuccess;
  for (long long c0 = 0; c0 < h->ncell && e == cudaSuccess; c0 += chunk) {
    const long long cnt = (c0 + chunk <= h->ncell) ? chunk : h->ncell - c0;
    e = launch_moments(h->P, h->prm.store, parity, h->pop, h->ghost, which, tmp,
                       dtype == LBM_DT_F64, c0, cnt, h->stream);
    for (int j = 0; j < nf && e == cudaSuccess; ++j)  // one plain copy per field row
      e = cudaMemcpyAsync(static_cast<char*>(dst) + ((size_t)j * h->ncell + c0) * es,
                          static_cast<char*>(tmp) + (size_t)j * cnt * es, (size_t)cnt * es,
                          cudaMemcpyDeviceToHost, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(LBM_E_CUDA, "moments failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_sensor(lbm_handle* h, void* dst, int dst_on_device, int dtype) {
  if (!h || !dst) return fail(LBM_E_INVAL, "NULL argument");
  LBM_ON_DEVICE(h->device);
  if (dtype != LBM_DT_F32 && dtype != LBM_DT_F64) return fail(LBM_E_INVAL, "dtype must be F32 or F64");
  const size_t es = dtype == LBM_DT_F64 ? 8 : 4;
  const int parity = (int)(h->step & 1);
  if (dst_on_device) {
    LBM_CUDA(launch_sensor(h->P, h->prm.store, parity, h->pop, h->ghost, dst, dtype == LBM_DT_F64, 0,
                           h->ncell, h->stream));
    return LBM_OK;
  }
  if (void* m = mapped_host(dst, es)) {  // page-locked: the kernel writes it directly
    cudaError_t e = launch_sensor(h->P, h->prm.store, parity, h->pop, h->ghost, m,
                                  dtype == LBM_DT_F64, 0, h->ncell, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(LBM_E_CUDA, "sensor failed: %s", cudaGetErrorString(e));
    return LBM_OK;
  }
  long long chunk = (long long)(kStageBytes / (es * 3));
  if (chunk > h->ncell) chunk = h->ncell;
  lbm_status st = ensure_stage(h);
  if (st != LBM_OK) return st;
  void* tmp = h->stage;
  cudaError_t e = cudaSuccess;
  for (long long c0 = 0; c0 < h->ncell && e == cudaSuccess; c0 += chunk) {
    const long long cnt = (c0 + chunk <= h->ncell) ? chunk : h->ncell - c0;
    e = launch_sensor(h->P, h->prm.store, parity, h->pop, h->ghost, tmp, dtype == LBM_DT_F64, c0, cnt,
                      h->stream);
    for (int j = 0; j < 3 && e == cudaSuccess; ++j)
      e = cudaMemcpyAsync(static_cast<char*>(dst) + ((size_t)j * h->ncell + c0) * es,
                          static_cast<char*>(tmp) + (size_t)j * cnt * es, (size_t)cnt * es,
                          cudaMemcpyDeviceToHost, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(LBM_E_CUDA, "sensor failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

static lbm_status ensure_diag_scratch(lbm_handle* h) {
  if (h->ufield) return LBM_OK;
  if (cudaMalloc(&h->ufield, sizeof(float) * 4 * (size_t)h->ncell) != cudaSuccess ||
      cudaMalloc(&h->partials, sizeof(double) * (size_t)kDiagBlocks * (kDiagA + 2)) != cudaSuccess ||
      cudaMalloc(&h->dout, sizeof(double) * 16) != cudaSuccess) {
    cudaGetLastError();
    if (h->ufield) cudaFree(h->ufield);
    if (h->partials) cudaFree(h->partials);
    if (h->dout) cudaFree(h->dout);
    h->ufield = nullptr;
    h->partials = h->dout = nullptr;
    return fail(LBM_E_NOMEM, "diagnostic scratch allocation failed");
  }
  return LBM_OK;
}

}  // extern "C"

namespace lbm {

// Fills *out from the reduced values r[0..kDiagA+2) of the state after `step` steps.
lbm_status finish_diag(lbm_handle* h, const double* r, unsigned flag, long long step,
                              lbm_diag_t* out) {
  const double n = (double)h->ncell;
  out->step = (double)step;
  out->time = (double)step * h->dt;
  out->sum_rho = r[0];
  out->sum_mx = r[1];
  out->sum_my = r[2];
  out->sum_mz = r[3];
  out->sum_E = r[4];
  out->ek_mean = r[5] / n;
  out->nonfinite = r[6];
  out->max_mach = r[9];
  out->max_cfl = r[10];
  out->min_rho = r[11];
  out->min_T = r[12];
  out->eps_s_raw = r[13] / n;
  out->eps_d_raw = 4.0 / 3.0 * r[14] / n;
  latch_flag(h, flag);
  if (r[6] > 0) h->nonfinite = true;
  if (h->stalled) return fail(LBM_E_TIMEOUT, "a staged step gave up waiting for a bulk copy; re-init");
  if (h->nonfinite) return fail(LBM_E_NONFINITE, "non-finite moments detected");
  return LBM_OK;
}

}  // namespace lbm

extern "C" {

lbm_status lbm_diag(lbm_handle* h, lbm_diag_t* out) {
  Range range_("lbm_diag");
  if (!h || !out) return fail(LBM_E_INVAL, "NULL argument");
  LBM_ON_DEVICE(h->device);
  lbm_status st = ensure_diag_scratch(h);
  if (st != LBM_OK) return st;
  double r[16] = {0};
  LBM_CUDA(launch_diag(h->P, h->prm.store, (int)(h->step & 1), h->pop, h->ghost, h->ufield,
                       h->partials, h->dout, h->stream));
  LBM_CUDA(cudaMemcpyAsync(r, h->dout, sizeof(double) * (kDiagA + 2), cudaMemcpyDeviceToHost, h->stream));
  unsigned flag = 0;
  LBM_CUDA(cudaMemcpyAsync(&flag, h->flag, sizeof(flag), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  return finish_diag(h, r, flag, h->step, out);
}

lbm_status lbm_step_diag(lbm_handle* h, int n, lbm_diag_t* out) {
  Range range_("lbm_step_diag");
  if (!h || !out) return fail(LBM_E_INVAL, "NULL argument");
  LBM_ON_DEVICE(h->device);
  if (n < 1) return fail(LBM_E_INVAL, "n must be >= 1");
  if (!h->initialized) return fail(LBM_E_STATE, "lbm_step_diag before an init");
  if (h->nonfinite) return fail(LBM_E_NONFINITE, "non-finite moments were detected earlier");
  if (h->stalled) return fail(LBM_E_TIMEOUT, "a staged step gave up waiting for a bulk copy; re-init");
  lbm_status st = ensure_diag_scratch(h);
  if (st != LBM_OK) return st;
  const int bx = effective_block(h);
  const long long nrec = step_diag_record_count(h->P, bx);
  if (nrec > h->wrec_n) {
    if (h->wrec) cudaFree(h->wrec);
    h->wrec = nullptr;
    h->wrec_n = 0;
    if (cudaMalloc(&h->wrec, sizeof(float) * kDiagRecFloats * (size_t)nrec) != cudaSuccess) {
      cudaGetLastError();
      h->wrec = nullptr;
      return fail(LBM_E_NOMEM, "diagnostic record allocation failed");
    }
    h->wrec_n = nrec;
  }
  if (!h->hdiag) {
    if (cudaMallocHost(&h->hdiag, sizeof(double) * 17) != cudaSuccess) {
      cudaGetLastError();
      h->hdiag = nullptr;
      return fail(LBM_E_NOMEM, "pinned host allocation failed");
    }
  }
  if (!h->ev_diag) LBM_CUDA(cudaEventCreateWithFlags(&h->ev_diag, cudaEventDisableTiming));
  const long long step0 = h->step;
  LBM_CUDA(launch_step_diag(h->P, h->prm.store, (int)(h->step & 1), h->pop, h->ghost, h->flag,
                            h->ufield, h->wrec, bx, h->stream));
  h->step += 1;
  LBM_CUDA(launch_diag_records(h->P, h->wrec, nrec, h->ufield, h->partials, h->dout, h->stream));
  LBM_CUDA(cudaMemcpyAsync(h->hdiag, h->dout, sizeof(double) * (kDiagA + 2), cudaMemcpyDeviceToHost,
                           h->stream));
  LBM_CUDA(cudaMemcpyAsync(h->hdiag + 16, h->flag, sizeof(unsigned), cudaMemcpyDeviceToHost,
                           h->stream));
  LBM_CUDA(cudaEventRecord(h->ev_diag, h->stream));
  if (n > 1) {
    st = lbm_step(h, n - 1);
    if (st != LBM_OK) return st;
  }
  LBM_CUDA(cudaEventSynchronize(h->ev_diag));
  unsigned flag = 0;
  std::memcpy(&flag, h->hdiag + 16, sizeof(flag));
  return finish_diag(h, h->hdiag, flag, step0, out);
}

static lbm_status pop_transfer(lbm_handle* h, void* buf, int on_device, int dtype, bool get) {
  if (!h || !buf) return fail(LBM_E_INVAL, "NULL argument");
  LBM_ON_DEVICE(h->device);
  if (dtype != LBM_DT_F32 && dtype != LBM_DT_F64 && dtype != LBM_DT_NATIVE)
    return fail(LBM_E_INVAL, "bad dtype");
  const size_t es = dtype == LBM_DT_F64 ? 8 : (dtype == LBM_DT_F32 ? 4 : elem_size(h->prm.store));
  const size_t arr = es * (size_t)h->ncell;
  const int parity = (int)(h->step & 1);
  void* tmp = nullptr;
  if (!on_device && cudaMalloc(&tmp, arr) != cudaSuccess) {
    cudaGetLastError();
    return fail(LBM_E_NOMEM, "staging allocation failed");
  }
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < kF && e == cudaSuccess; ++k)
    for (int i = 0; i < kQ && e == cudaSuccess; ++i) {
      char* user = static_cast<char*>(buf) + (size_t)(k * kQ + i) * arr;
      void* dev = on_device ? (void*)user : tmp;
      if (get) {
        e = launch_pop_get(h->P, h->prm.store, parity, h->pop, h->ghost, k, i, dev, dtype, h->stream);
        if (e == cudaSuccess && !on_device)
          e = cudaMemcpyAsync(user, tmp, arr, cudaMemcpyDeviceToHost, h->stream);
      } else {
        if (!on_device) e = cudaMemcpyAsync(tmp, user, arr, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
          e = launch_pop_set(h->P, h->prm.store, parity, h->pop, k, i, dev, dtype, h->stream);
      }
      if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
    }
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return fail(LBM_E_CUDA, "population transfer failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_populations_get(lbm_handle* h, void* dst, int dst_on_device, int dtype) {
  return pop_transfer(h, dst, dst_on_device, dtype, true);
}

lbm_status lbm_populations_set(lbm_handle* h, const void* src, int src_on_device, int dtype) {
  lbm_status s = pop_transfer(h, const_cast<void*>(src), src_on_device, dtype, false);
  if (s != LBM_OK) return s;
  h->initialized = true;
  h->graphs_valid = false;
  return LBM_OK;
}

static lbm_status plane_transfer(lbm_handle* h, int z, int slot, void* buf, int on_device, bool set) {
  Range range_("lbm_plane");
  if (!h || !buf) return fail(LBM_E_INVAL, "NULL argument");
  LBM_ON_DEVICE(h->device);
  if (z < 0 || z >= h->prm.nz) return fail(LBM_E_INVAL, "plane z = %d outside [0, %d)", z, h->prm.nz);
  if (slot < 0 || slot >= kQ) return fail(LBM_E_INVAL, "slot %d outside [0, 7)", slot);
  if (h->P.eso)
    return fail(LBM_E_INVAL, "slot planes follow the AA maps; not available under the esoteric twist");
  const size_t bytes = elem_size(h->prm.store) * kF * (size_t)h->prm.nx * h->prm.ny;
  void* dev = buf;
  if (!on_device) {
    if (cudaMalloc(&dev, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(LBM_E_NOMEM, "staging allocation failed");
    }
  }
  cudaError_t e = cudaSuccess;
  if (set && !on_device) e = cudaMemcpyAsync(dev, buf, bytes, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = launch_plane(h->P, h->prm.store, h->pop, z, slot, dev, set ? 1 : 0, h->stream);
  if (e == cudaSuccess && !set && !on_device)
    e = cudaMemcpyAsync(buf, dev, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (!on_device) {
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dev);
  }
  if (e != cudaSuccess) return fail(LBM_E_CUDA, "plane transfer failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_plane_get(lbm_handle* h, int z, int slot, void* dst, int dst_on_device) {
  return plane_transfer(h, z, slot, dst, dst_on_device, false);
}

lbm_status lbm_plane_set(lbm_handle* h, int z, int slot, const void* src, int src_on_device) {
  return plane_transfer(h, z, slot, const_cast<void*>(src), src_on_device, true);
}

lbm_status lbm_autotune(lbm_handle* h, int pairs_per_trial, lbm_tune_t* out) {
  Range range_("lbm_autotune");
  if (!h) return fail(LBM_E_INVAL, "handle is NULL");
  LBM_ON_DEVICE(h->device);
  if (!h->initialized) return fail(LBM_E_STATE, "autotune needs an initialised state");
  if (h->nonfinite || h->stalled) return fail(LBM_E_STATE, "autotune on a failed state; re-init");
  if (pairs_per_trial < 1) pairs_per_trial = 4;
  struct Cand {
    int variant, block, prefetch;
  };
  std::vector<Cand> cands;
  // The L2 prefetch applies to the plain forms on whole-tile rows only.
  const bool rows = h->P.bc_x == 0 && h->P.nx % 32 == 0;
  for (int v : {0, 1})
    for (int b : {64, 128})
      if (b <= 32 * ((h->P.nx + 31) / 32) || b == 64)
        for (int pf : {0, 512, 1024, 2048})
          if (pf == 0 || rows) cands.push_back({v, b, pf});
  // The staged forms (variants 2-4) are not candidates: measured slower than the plain
  // forms at every size and storage type (their shared-memory pipeline costs more
  // instructions per cell than it saves in latency, and the L2 prefetch hides the
  // same latency for 1-3 instructions per warp). lbm_set_kernel_config still selects
  // them explicitly.
  cudaEvent_t a, b;
  LBM_CUDA(cudaEventCreate(&a));
  LBM_CUDA(cudaEventCreate(&b));
  float best = 1e30f;
  int best_b = h->block_x, best_v = h->variant, best_grid = h->staged_grid, tried = 0;
  int best_pf = h->P.pf_tiles;
  cudaError_t err = cudaSuccess;
  for (const Cand& c : cands) {
    int grid = 0;
    if (c.variant >= kFirstStagedVariant) {
      if (staged_prepare(h->P, h->prm.store, c.variant, &grid) != cudaSuccess) {
        cudaGetLastError();
        continue;  // this form does not fit the device (shared memory); skip it
      }
    }
    h->block_x = c.block;
    h->variant = c.variant;
    h->staged_grid = grid;
    h->P.pf_tiles = c.prefetch;
    for (int j = 0; j < 2 && err == cudaSuccess; ++j)  // warm-up pair
      err = step_launch(h, (int)((h->step + j) & 1), h->stream);
    h->step += 2;
    if (err == cudaSuccess) err = cudaEventRecord(a, h->stream);
    for (int j = 0; j < 2 * pairs_per_trial && err == cudaSuccess; ++j)
      err = step_launch(h, (int)((h->step + j) & 1), h->stream);
    h->step += 2 * pairs_per_trial;
    if (err == cudaSuccess) err = cudaEventRecord(b, h->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(b);
    float ms = 0;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, a, b);
    if (err != cudaSuccess) break;
    ms /= (float)(2 * pairs_per_trial);
    ++tried;
    if (ms < best) {
      best = ms;
      best_b = c.block;
      best_v = c.variant;
      best_grid = grid;
      best_pf = c.prefetch;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  h->block_x = best_b;
  h->variant = best_v;
  h->staged_grid = best_grid;
  h->P.pf_tiles = best_pf;
  h->graphs_valid = false;
  if (err != cudaSuccess) return fail(LBM_E_CUDA, "autotune failed: %s", cudaGetErrorString(err));
  unsigned flag = 0;
  LBM_CUDA(cudaMemcpyAsync(&flag, h->flag, sizeof(flag), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  latch_flag(h, flag);
  if (h->stalled) return fail(LBM_E_TIMEOUT, "a staged step gave up waiting for a bulk copy; re-init");
  if (out) {
    out->block_x = best_v >= kFirstStagedVariant ? 128 : effective_block(h);
    out->variant = best_v;
    out->ms_per_step = best;
    out->candidates = tried;
    out->prefetch_tiles = best_pf;
  }
  return LBM_OK;
}

lbm_status lbm_check_count(const lbm_handle* h, unsigned long long* count) {
  if (!h || !count) return fail(LBM_E_INVAL, "NULL argument");
#ifdef LBM_CHECKED
  LBM_ON_DEVICE(h->device);
  unsigned v = 0;
  LBM_CUDA(cudaMemcpyAsync(&v, h->flag + 2, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  *count = v;
  return LBM_OK;
#else
  *count = 0;
  return fail(LBM_E_STATE, "not a checked build (compiled without LBM_CHECKED)");
#endif
}

lbm_status lbm_test_skip_copy(lbm_handle* h) {
  if (!h) return fail(LBM_E_INVAL, "handle is NULL");
  if (h->variant < kFirstStagedVariant) return fail(LBM_E_INVAL, "the kernel form is not staged");
  h->skip_next_copy = true;
  return LBM_OK;
}

lbm_status lbm_set_kernel_config(lbm_handle* h, int block_x, int variant) {
  if (!h) return fail(LBM_E_INVAL, "handle is NULL");
  LBM_ON_DEVICE(h->device);
  if (variant < 0 || variant > kLastStagedVariant) return fail(LBM_E_INVAL, "variant must be 0 to 4");
  if (variant >= kFirstStagedVariant) {
    if (!staged_eligible(h->P))
      return fail(LBM_E_INVAL,
                  "staged variants need periodic x, nx a multiple of 32, rounding to nearest "
                  "and the AA maps");
    int grid = 0;
    LBM_CUDA(staged_prepare(h->P, h->prm.store, variant, &grid));
    h->variant = variant;
    h->staged_grid = grid;
    h->graphs_valid = false;
    return LBM_OK;
  }
  if (block_x < 32 || block_x > 128 || (block_x & 31))
    return fail(LBM_E_INVAL, "block_x must be 32, 64, 96 or 128");
  h->block_x = block_x;
  h->variant = variant;
  h->graphs_valid = false;
  return LBM_OK;
}

lbm_status lbm_set_prefetch(lbm_handle* h, int tiles) {
  if (!h) return fail(LBM_E_INVAL, "handle is NULL");
  if (tiles < 0 || tiles > kMaxPrefetch)
    return fail(LBM_E_INVAL, "prefetch distance must be 0 to %d tiles", kMaxPrefetch);
  h->P.pf_tiles = tiles;
  h->graphs_valid = false;
  return LBM_OK;
}

// ---------------------------------------------------------------- checkpoints
namespace {

uint32_t crc32_update(uint32_t crc, const void* data, size_t n) {
  static uint32_t table[256];
  static bool ready = false;
  if (!ready) {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int j = 0; j < 8; ++j) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
      table[i] = c;
    }
    ready = true;
  }
  const unsigned char* p = static_cast<const unsigned char*>(data);
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) crc = table[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
  return ~crc;
}

struct CkptHeader {
  char magic[8];
  int32_t version, nx, ny, nz, store, bc_x;
  int64_t step;
  double rho_ref, E_ref;
  double scale[kF];
};

}  // namespace

lbm_status lbm_save(lbm_handle* h, const char* path) {
  if (!h || !path) return fail(LBM_E_INVAL, "NULL argument");
  LBM_ON_DEVICE(h->device);
  if (!h->initialized) return fail(LBM_E_STATE, "nothing to save before an init");
  CkptHeader hd{};
  std::memcpy(hd.magic, "LBMCKPT1", 8);
  hd.version = 1;
  hd.nx = h->prm.nx;
  hd.ny = h->prm.ny;
  hd.nz = h->prm.nz;
  hd.store = h->prm.store;
  hd.bc_x = h->prm.bc_x;
  hd.step = h->step;
  hd.rho_ref = h->rho_ref;
  hd.E_ref = h->E_ref;
  for (int k = 0; k < kF; ++k) hd.scale[k] = h->scale[k];
  const size_t gbytes = sizeof(float) * 2 * kF * (size_t)h->prm.ny * h->prm.nz;
  std::vector<float> ghost(gbytes / sizeof(float));
  LBM_CUDA(cudaMemcpyAsync(ghost.data(), h->ghost, gbytes, cudaMemcpyDeviceToHost, h->stream));
  const size_t es = elem_size(h->prm.store);
  std::vector<char> pops(es * (size_t)h->ncell * kP);
  lbm_status s = lbm_populations_get(h, pops.data(), 0, LBM_DT_NATIVE);
  if (s != LBM_OK) return s;
  uint32_t crc = crc32_update(0, &hd, sizeof(hd));
  crc = crc32_update(crc, ghost.data(), gbytes);
  crc = crc32_update(crc, pops.data(), pops.size());
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(LBM_E_IO, "cannot open %s for writing", path);
  bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 && std::fwrite(ghost.data(), 1, gbytes, f) == gbytes &&
            std::fwrite(pops.data(), 1, pops.size(), f) == pops.size() &&
            std::fwrite(&crc, sizeof(crc), 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(LBM_E_IO, "write to %s failed", path);
  return LBM_OK;
}

lbm_status lbm_load(lbm_handle* h, const char* path) {
  if (!h || !path) return fail(LBM_E_INVAL, "NULL argument");
  LBM_ON_DEVICE(h->device);
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(LBM_E_IO, "cannot open %s", path);
  CkptHeader hd{};
  const size_t gbytes = sizeof(float) * 2 * kF * (size_t)h->prm.ny * h->prm.nz;
  const size_t es = elem_size(h->prm.store);
  std::vector<float> ghost(gbytes / sizeof(float));
  std::vector<char> pops(es * (size_t)h->ncell * kP);
  uint32_t crc_file = 0;
  bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1;
  if (ok && (std::memcmp(hd.magic, "LBMCKPT1", 8) != 0 || hd.version != 1)) {
    std::fclose(f);
    return fail(LBM_E_IO, "%s is not an lbm checkpoint", path);
  }
  if (ok && (hd.nx != h->prm.nx || hd.ny != h->prm.ny || hd.nz != h->prm.nz ||
             hd.store != h->prm.store || hd.bc_x != h->prm.bc_x)) {
    std::fclose(f);
    return fail(LBM_E_INVAL, "checkpoint sizes or storage differ from the handle's");
  }
  ok = ok && std::fread(ghost.data(), 1, gbytes, f) == gbytes &&
       std::fread(pops.data(), 1, pops.size(), f) == pops.size() &&
       std::fread(&crc_file, sizeof(crc_file), 1, f) == 1;
  std::fclose(f);
  if (!ok) return fail(LBM_E_IO, "%s is truncated", path);
  uint32_t crc = crc32_update(0, &hd, sizeof(hd));
  crc = crc32_update(crc, ghost.data(), gbytes);
  crc = crc32_update(crc, pops.data(), pops.size());
  if (crc != crc_file) return fail(LBM_E_IO, "%s: CRC mismatch", path);
  h->rho_ref = hd.rho_ref;
  h->E_ref = hd.E_ref;
  h->P.rho_ref = (float)hd.rho_ref;
  h->P.E_ref = (float)hd.E_ref;
  for (int k = 0; k < kF; ++k) {
    h->scale[k] = hd.scale[k];
    h->P.scale[k] = (float)hd.scale[k];
    h->P.inv_scale[k] = (float)(1.0 / hd.scale[k]);
  }
  LBM_CUDA(cudaMemcpyAsync(h->ghost, ghost.data(), gbytes, cudaMemcpyHostToDevice, h->stream));
  h->step = hd.step;  // parity of the stored canonical order is re-applied by the set
  lbm_status s = lbm_populations_set(h, pops.data(), 0, LBM_DT_NATIVE);
  if (s != LBM_OK) return s;
  LBM_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(unsigned), h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  h->nonfinite = false;
  return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- internal view
// Read access to a handle's device state for other translation units of the
// library (the fixed-scratch diagnostics in diag_static.cu).
namespace lbm {

HandleView handle_view(lbm_handle* h) {
  HandleView v;
  v.P = &h->P;
  v.store = h->prm.store;
  v.step = h->step;
  v.dt = h->dt;
  v.pop = h->pop;
  v.ghost = h->ghost;
  v.flag = h->flag;
  v.stream = h->stream;
  v.ncell = h->ncell;
  v.device = h->device;
  return v;
}

}  // namespace lbm

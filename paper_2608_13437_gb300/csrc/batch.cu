// Batched mode: many independent periodic domains of different sizes and
// parameters, stored in one buffer, advanced by ONE persistent launch per time
// step. The grid holds as many blocks as are resident on the GPU; block b takes
// tiles b, b + grid, b + 2 grid, ... of a table ordered largest domain first. A
// tile is `tile_cells` consecutive cells of one domain; the block stages that
// domain's constants in shared memory and runs the same per-cell update as the
// single-domain kernel. Tile and block sizes come from the autotuner; the step
// pair is replayed from a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "api_common.h"

using namespace lbm;

namespace lbm {
namespace {

struct Tile {
  int domain;
  int first;  // first cell of the tile within its domain
};

template <int PARITY>
__global__ void __launch_bounds__(256) k_batch_step(const DomainConst* __restrict__ consts,
                                                    float* const* __restrict__ pops,
                                                    const Tile* __restrict__ tiles, int ntiles,
                                                    int tile_cells, unsigned* __restrict__ flag) {
  __shared__ DomainConst sP;
  __shared__ float* sPop;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile tile = tiles[t];
    __syncthreads();  // previous tile's readers are done with sP
    if (threadIdx.x == 0) {
      sP = consts[tile.domain];
      sPop = pops[tile.domain];
    }
    __syncthreads();
    const DomainConst& P = sP;
    float* pop = sPop;
    const long long end = min((long long)tile.first + tile_cells, P.ncell);
    for (long long cell = tile.first + threadIdx.x; cell < end; cell += blockDim.x) {
      const int x = (int)(cell % P.nx);
      const long long yz = cell / P.nx;
      const CellIndex c = make_index(P, x, (int)(yz % P.ny), (int)(yz / P.ny));
      float d[kF][kQ];
      load_cell<PARITY, false, float>(P, pop, nullptr, c, d);
      const float probe = collide_cell<false>(P, d, nullptr);
      if (!isfinite(probe)) atomicOr(flag, 1u);
#pragma unroll
      for (int k = 0; k < kF; ++k) store_field<PARITY, float>(P, pop, c, k, d[k]);
    }
  }
}

}  // namespace
}  // namespace lbm

struct lbm_batch {
  int n = 0;
  std::vector<lbm_params> prm;
  std::vector<DomainConst> P;
  std::vector<double> dt, tau_R, tau_q, rho_ref, E_ref;
  std::vector<size_t> offset;   // byte offset of each domain's populations
  long long total_cells = 0;
  void* pool = nullptr;
  DomainConst* d_consts = nullptr;
  float** d_pops = nullptr;
  Tile* d_tiles = nullptr;
  int ntiles = 0;
  int tile_cells = 1024;
  int block = 128;
  int grid = 0;
  unsigned* flag = nullptr;
  float* ghost = nullptr;  // unused by periodic domains; a valid pointer for the plain kernel
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t g_pair = nullptr;
  bool graphs_valid = false;
  long long step = 0;
  bool initialized = false;
  bool nonfinite = false;
};

namespace {

#define LBM_CUDA(expr)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(LBM_E_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));                \
  } while (0)

float* domain_pop(lbm_batch* b, int d) {
  return reinterpret_cast<float*>(static_cast<char*>(b->pool) + b->offset[d]);
}

// Tile table, largest domain first; rebuilt when tile_cells changes.
lbm_status build_tiles(lbm_batch* b) {
  std::vector<int> order(b->n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int c) { return b->P[a].ncell > b->P[c].ncell; });
  std::vector<Tile> tiles;
  for (int d : order)
    for (long long f = 0; f < b->P[d].ncell; f += b->tile_cells) tiles.push_back(Tile{d, (int)f});
  if (b->d_tiles) cudaFree(b->d_tiles);
  b->d_tiles = nullptr;
  LBM_CUDA(cudaMalloc(&b->d_tiles, sizeof(Tile) * tiles.size()));
  LBM_CUDA(cudaMemcpy(b->d_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice));
  b->ntiles = (int)tiles.size();
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_step<0>, b->block, 0);
  if (e != cudaSuccess || per_sm < 1) per_sm = 1;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->grid = std::max(1, std::min(per_sm * sms, b->ntiles));
  b->graphs_valid = false;
  return LBM_OK;
}

cudaError_t launch_batch(lbm_batch* b, int parity, cudaStream_t s) {
  if (parity)
    k_batch_step<1><<<b->grid, b->block, 0, s>>>(b->d_consts, b->d_pops, b->d_tiles, b->ntiles,
                                                   b->tile_cells, b->flag);
  else
    k_batch_step<0><<<b->grid, b->block, 0, s>>>(b->d_consts, b->d_pops, b->d_tiles, b->ntiles,
                                                   b->tile_cells, b->flag);
  return cudaGetLastError();
}

lbm_status ensure_batch_graph(lbm_batch* b) {
  if (b->graphs_valid) return LBM_OK;
  if (b->g_pair) cudaGraphExecDestroy(b->g_pair);
  b->g_pair = nullptr;
  cudaGraph_t g = nullptr;
  LBM_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = launch_batch(b, 0, b->cap);
  if (le == cudaSuccess) le = launch_batch(b, 1, b->cap);
  cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
  if (le != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(LBM_E_CUDA, "batch graph capture failed: %s",
                cudaGetErrorString(le != cudaSuccess ? le : ee));
  }
  cudaError_t ie = cudaGraphInstantiate(&b->g_pair, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return fail(LBM_E_CUDA, "batch graph instantiate failed: %s", cudaGetErrorString(ie));
  b->graphs_valid = true;
  return LBM_OK;
}

lbm_status upload_consts(lbm_batch* b) {
  LBM_CUDA(cudaMemcpy(b->d_consts, b->P.data(), sizeof(DomainConst) * b->n, cudaMemcpyHostToDevice));
  b->graphs_valid = false;
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(int n, const lbm_params* params, lbm_batch** out) {
  if (!out) return fail(LBM_E_INVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !params) return fail(LBM_E_INVAL, "need n >= 1 domains");
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return fail(LBM_E_NOMEM, "host allocation failed");
  b->n = n;
  size_t bytes = 0;
  for (int d = 0; d < n; ++d) {
    lbm_status s = validate(&params[d]);
    if (s != LBM_OK) {
      delete b;
      return fail(s, "domain %d: %s", d, g_last_error.c_str());
    }
    if (params[d].store != LBM_STORE_F32 || params[d].bc_x != 0) {
      delete b;
      return fail(LBM_E_INVAL, "domain %d: the batched mode takes periodic F32 domains", d);
    }
    b->prm.push_back(params[d]);
    double dt, tR, tq;
    derive(&params[d], &dt, &tR, &tq);
    DomainConst P;
    fill_const(&params[d], dt, tR, tq, &P);
    b->P.push_back(P);
    b->dt.push_back(dt);
    b->tau_R.push_back(tR);
    b->tau_q.push_back(tq);
    b->rho_ref.push_back(0.0);
    b->E_ref.push_back(0.0);
    b->offset.push_back(bytes);
    bytes += (size_t)P.stride * sizeof(float) * kP;
    b->total_cells += P.ncell;
  }
  b->stream = static_cast<cudaStream_t>(params[0].cuda_stream);
  auto cleanup = [&](lbm_status st) {
    lbm_batch_destroy(b);
    return st;
  };
  if (cudaMalloc(&b->pool, bytes) != cudaSuccess) {
    cudaGetLastError();
    b->pool = nullptr;
    return cleanup(fail(LBM_E_NOMEM, "cudaMalloc of %zu batch bytes failed", bytes));
  }
  std::vector<float*> ptrs(n);
  for (int d = 0; d < n; ++d) ptrs[d] = domain_pop(b, d);
  if (cudaMalloc(&b->d_consts, sizeof(DomainConst) * n) != cudaSuccess ||
      cudaMalloc(&b->d_pops, sizeof(float*) * n) != cudaSuccess ||
      cudaMalloc(&b->flag, 64) != cudaSuccess || cudaMalloc(&b->ghost, 256) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(LBM_E_NOMEM, "cudaMalloc of batch tables failed"));
  }
  if (cudaMemcpy(b->d_pops, ptrs.data(), sizeof(float*) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->flag, 0, 64) != cudaSuccess)
    return cleanup(fail(LBM_E_CUDA, "batch table upload failed"));
  lbm_status s = upload_consts(b);
  if (s != LBM_OK) return cleanup(s);
  s = build_tiles(b);
  if (s != LBM_OK) return cleanup(s);
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    return cleanup(fail(LBM_E_CUDA, "cudaStreamCreate failed"));
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_OK;
  cudaStreamSynchronize(b->stream);
  if (b->g_pair) cudaGraphExecDestroy(b->g_pair);
  if (b->pool) cudaFree(b->pool);
  if (b->d_consts) cudaFree(b->d_consts);
  if (b->d_pops) cudaFree(b->d_pops);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->flag) cudaFree(b->flag);
  if (b->ghost) cudaFree(b->ghost);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return LBM_OK;
}

lbm_status lbm_batch_init_tgv(lbm_batch* b, const double* U0, const double* M0, const double* rho0) {
  if (!b || !U0 || !M0 || !rho0) return fail(LBM_E_INVAL, "NULL argument");
  for (int d = 0; d < b->n; ++d) {
    const lbm_params& p = b->prm[d];
    if (!(std::isfinite(U0[d]) && finite_pos(M0[d]) && finite_pos(rho0[d])))
      return fail(LBM_E_INVAL, "domain %d: bad TGV parameters", d);
    const double p0 = rho0[d] * U0[d] * U0[d] / (p.gamma * M0[d] * M0[d]);
    if (!finite_pos(p0)) return fail(LBM_E_INVAL, "domain %d: U0 must be nonzero", d);
    b->P[d].rho_ref = (float)rho0[d];
    b->P[d].E_ref = (float)(p0 / (p.gamma - 1.0));
    b->rho_ref[d] = (double)b->P[d].rho_ref;
    b->E_ref[d] = (double)b->P[d].E_ref;
    InitSpec sp{};
    sp.kind = 0;
    sp.U0 = U0[d];
    sp.M0 = M0[d];
    sp.rho0 = rho0[d];
    sp.gamma = p.gamma;
    sp.mu = p.mu;
    sp.kappa = p.kappa;
    sp.tau_R = b->tau_R[d];
    sp.tau_q = b->tau_q[d];
    sp.inv_T_ref = 1.0 / p.T_ref;
    sp.c = p.dx / b->dt[d];
    sp.dx = p.dx;
    sp.sutherland = p.sutherland;
    LBM_CUDA(launch_init(b->P[d], LBM_STORE_F32, sp, 1, domain_pop(b, d), nullptr, nullptr, b->stream));
  }
  lbm_status s = upload_consts(b);
  if (s != LBM_OK) return s;
  LBM_CUDA(cudaMemsetAsync(b->flag, 0, sizeof(unsigned), b->stream));
  LBM_CUDA(cudaStreamSynchronize(b->stream));
  b->step = 0;
  b->initialized = true;
  b->nonfinite = false;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int n) {
  if (!b) return fail(LBM_E_INVAL, "batch is NULL");
  if (n < 0) return fail(LBM_E_INVAL, "n must be >= 0");
  if (!b->initialized) return fail(LBM_E_STATE, "lbm_batch_step before an init");
  if (b->nonfinite) return fail(LBM_E_NONFINITE, "non-finite moments were detected earlier");
  lbm_status s = ensure_batch_graph(b);
  if (s != LBM_OK) return s;
  if (n > 0 && (b->step & 1)) {
    LBM_CUDA(launch_batch(b, 1, b->stream));
    b->step += 1;
    --n;
  }
  while (n >= 2) {
    LBM_CUDA(cudaGraphLaunch(b->g_pair, b->stream));
    b->step += 2;
    n -= 2;
  }
  if (n) {
    LBM_CUDA(launch_batch(b, 0, b->stream));
    b->step += 1;
  }
  return LBM_OK;
}

lbm_status lbm_batch_step_sequential(lbm_batch* b, int n) {
  if (!b) return fail(LBM_E_INVAL, "batch is NULL");
  if (n < 0) return fail(LBM_E_INVAL, "n must be >= 0");
  if (!b->initialized) return fail(LBM_E_STATE, "lbm_batch_step_sequential before an init");
  if (b->nonfinite) return fail(LBM_E_NONFINITE, "non-finite moments were detected earlier");
  for (int j = 0; j < n; ++j) {
    const int parity = (int)(b->step & 1);
    for (int d = 0; d < b->n; ++d) {
      const int bx = std::min(128, ((b->P[d].nx + 31) / 32) * 32);
      LBM_CUDA(launch_step(b->P[d], LBM_STORE_F32, parity, domain_pop(b, d), b->ghost, b->flag, bx,
                           b->stream));
    }
    b->step += 1;
  }
  return LBM_OK;
}

lbm_status lbm_batch_synchronize(lbm_batch* b) {
  if (!b) return fail(LBM_E_INVAL, "batch is NULL");
  unsigned flag = 0;
  LBM_CUDA(cudaMemcpyAsync(&flag, b->flag, sizeof(flag), cudaMemcpyDeviceToHost, b->stream));
  LBM_CUDA(cudaStreamSynchronize(b->stream));
  if (flag) b->nonfinite = true;
  if (b->nonfinite) return fail(LBM_E_NONFINITE, "non-finite moments detected");
  return LBM_OK;
}

lbm_status lbm_batch_moments(lbm_batch* b, int domain, int which, void* dst, int dst_on_device,
                             int dtype) {
  if (!b || !dst) return fail(LBM_E_INVAL, "NULL argument");
  if (domain < 0 || domain >= b->n) return fail(LBM_E_INVAL, "domain index out of range");
  if (which != LBM_MOM_Q && which != LBM_MOM_PRIM) return fail(LBM_E_INVAL, "bad moment set");
  if (dtype != LBM_DT_F32 && dtype != LBM_DT_F64) return fail(LBM_E_INVAL, "dtype must be F32 or F64");
  const DomainConst& P = b->P[domain];
  const int nf = which == LBM_MOM_Q ? kF : 6;
  const size_t es = dtype == LBM_DT_F64 ? 8 : 4;
  const size_t bytes = (size_t)nf * es * P.ncell;
  void* dev = dst;
  if (!dst_on_device) {
    if (cudaMalloc(&dev, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(LBM_E_NOMEM, "staging allocation failed");
    }
  }
  cudaError_t e = launch_moments(P, LBM_STORE_F32, (int)(b->step & 1), domain_pop(b, domain), b->ghost,
                                 which, dev, dtype == LBM_DT_F64, 0, P.ncell, b->stream);
  if (e == cudaSuccess && !dst_on_device)
    e = cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess && !dst_on_device) e = cudaStreamSynchronize(b->stream);
  if (!dst_on_device) cudaFree(dev);
  if (e != cudaSuccess) return fail(LBM_E_CUDA, "batch moments failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_batch_info(const lbm_batch* b, long long* total_cells, int domain, double* dt) {
  if (!b) return fail(LBM_E_INVAL, "batch is NULL");
  if (total_cells) *total_cells = b->total_cells;
  if (dt) {
    if (domain < 0 || domain >= b->n) return fail(LBM_E_INVAL, "domain index out of range");
    *dt = b->dt[domain];
  }
  return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int steps_per_trial, int* tile_cells, int* block_threads,
                              float* ms_per_step) {
  if (!b) return fail(LBM_E_INVAL, "batch is NULL");
  if (!b->initialized) return fail(LBM_E_STATE, "autotune needs an initialised batch");
  if (steps_per_trial < 2) steps_per_trial = 4;
  steps_per_trial += steps_per_trial & 1;  // whole pairs keep the parity
  const int tiles[] = {256, 512, 1024, 2048, 4096};
  const int blocks[] = {128, 256};
  cudaEvent_t a, e;
  LBM_CUDA(cudaEventCreate(&a));
  LBM_CUDA(cudaEventCreate(&e));
  float best = 1e30f;
  int best_t = b->tile_cells, best_b = b->block;
  for (int bl : blocks)
    for (int tc : tiles) {
      b->block = bl;
      b->tile_cells = tc;
      lbm_status s = build_tiles(b);
      if (s != LBM_OK) return s;
      for (int j = 0; j < 2; ++j) LBM_CUDA(launch_batch(b, (int)((b->step + j) & 1), b->stream));
      b->step += 2;
      LBM_CUDA(cudaEventRecord(a, b->stream));
      for (int j = 0; j < steps_per_trial; ++j)
        LBM_CUDA(launch_batch(b, (int)((b->step + j) & 1), b->stream));
      b->step += steps_per_trial;
      LBM_CUDA(cudaEventRecord(e, b->stream));
      LBM_CUDA(cudaEventSynchronize(e));
      float ms = 0;
      LBM_CUDA(cudaEventElapsedTime(&ms, a, e));
      ms /= (float)steps_per_trial;
      if (ms < best) {
        best = ms;
        best_t = tc;
        best_b = bl;
      }
    }
  cudaEventDestroy(a);
  cudaEventDestroy(e);
  b->block = best_b;
  b->tile_cells = best_t;
  lbm_status s = build_tiles(b);
  if (s != LBM_OK) return s;
  if (tile_cells) *tile_cells = best_t;
  if (block_threads) *block_threads = best_b;
  if (ms_per_step) *ms_per_step = best;
  return LBM_OK;
}

}  // extern "C"

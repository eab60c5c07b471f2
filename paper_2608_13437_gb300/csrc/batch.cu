// Batched mode: many independent periodic domains of different sizes and
// parameters, stored in one buffer, advanced by ONE persistent launch per time
// step. The grid holds as many blocks as are resident on the GPU. Each warp claims
// items from a counter, an item being `tiles_per_item` consecutive 32-cell layout
// tiles, until none are left, and keeps the constants of the domain it is working
// on in a slot of shared memory of its own, reloaded when its tile belongs to
// another domain (so the shared memory does not grow with the number of domains).
// A tile's domain and the (x, y, z) of its first cell come from a per-tile table
// (one 8-byte record per tile instead of a search and two divisions); no block-wide
// synchronisation happens, so warps overlap their loads and arithmetic freely. The
// per-cell update is the single-domain one; domains whose rows are whole tiles use its
// warp-uniform tile addressing. Items per warp, block size and register budget
// come from the autotuner; the step pair is replayed from a CUDA graph. 16-bit
// batches may round stochastically (one mode for the whole batch; a separate
// instantiation, as for one domain).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "api_common.h"
#include "step_impl.cuh"

using namespace lbm;

namespace lbm {
namespace batch_kernels {  // named: the host helpers below sit in an anonymous namespace

// L2 prefetch for the tile a record names, in the pattern of the single-domain kernel:
// even steps the tile's 7 slots, odd steps its slots 0-4 and, where a z plane holds
// whole tiles (every size of the batched workloads), slot 6 of the tile a plane before
// and slot 5 of the tile a plane after (periodic wrap). Only a hint; the sizes and the
// buffer of the record's domain come from the constants in global memory.
template <int PARITY, typename S, bool ESO>
__device__ __forceinline__ void prefetch_tile_record(const DomainConst* __restrict__ consts,
                                                     void* const* __restrict__ pops, uint2 r) {
  const int lo = (int)(r.x & 0xFFFFu);
  const DomainConst& P = consts[lo];
  const long long first = (long long)(r.x >> 16) +
                          (long long)P.nx * ((long long)(r.y & 0xFFFFu) + (long long)P.ny * (r.y >> 16));
  const long long w = first / kTile;  // a tile's first cell index is a multiple of 32
  const S* pop = static_cast<const S*>(pops[lo]);
  constexpr unsigned kSlotBytes = kSlotElems * sizeof(S);
  if constexpr (ESO) {  // the single-domain kernel's pattern under the esoteric twist
    l2_prefetch(pop + w * kTileElems, (PARITY ? 5 : 6) * kSlotBytes);
    if (PARITY) l2_prefetch(pop + w * kTileElems + 6 * kSlotElems, kSlotBytes);
    const long long plane = (long long)P.nx * P.ny;
    if (plane % kTile) return;
    const long long tpp = plane / kTile;
    const long long zp = w + tpp < P.ntile ? w + tpp : w + tpp - P.ntile;
    l2_prefetch(pop + zp * kTileElems + (PARITY ? 5 : 6) * kSlotElems, kSlotBytes);
    return;
  }
  if (PARITY == 0) {
    l2_prefetch(pop + w * kTileElems, kQ * kSlotBytes);
    return;
  }
  l2_prefetch(pop + w * kTileElems, 5 * kSlotBytes);
  const long long plane = (long long)P.nx * P.ny;
  if (plane % kTile) return;
  const long long tpp = plane / kTile;
  const long long zm = w >= tpp ? w - tpp : w - tpp + P.ntile;
  const long long zp = w + tpp < P.ntile ? w + tpp : w + tpp - P.ntile;
  l2_prefetch(pop + zm * kTileElems + 6 * kSlotElems, kSlotBytes);
  l2_prefetch(pop + zp * kTileElems + 5 * kSlotElems, kSlotBytes);
}

constexpr int kBatchMaxWarps = 4;  // blocks of at most 128 threads

// ESO: every domain under the esoteric twist (whole-tile rows take it as a compile-time
// form; the other domains from their constants).
template <int PARITY, int MINB, typename S, bool SR, bool ESO>
__global__ void __launch_bounds__(128, MINB) k_batch_step(const DomainConst* __restrict__ consts,
                                                          void* const* __restrict__ pops,
                                                          const uint2* __restrict__ tiles,
                                                          int total_tiles,
                                                          int tiles_per_item, int pf_items,
                                                          unsigned* __restrict__ next_item,
                                                          unsigned* __restrict__ flag) {
  // the constants and buffer of the domain each warp is on (blocks of at most 4 warps)
  __shared__ __align__(16) DomainConst sW[kBatchMaxWarps];
  __shared__ S* sPopW[kBatchMaxWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int cur = -1;  // domain whose constants the warp's slot holds
  const int n_items = (total_tiles + tiles_per_item - 1) / tiles_per_item;
  // Items are claimed in order from one counter (zeroed before the launch), so the
  // tiles in flight stay a compact window of the buffer, as with hardware block
  // scheduling. An item's tile records are loaded at once, one per lane (items hold at
  // most 32 tiles), and handed to the tiles by shuffles, so only an item's first tile
  // waits for a record load; the next item is claimed when the current one starts.
  auto records = [&](int it) {
    const int t = it * tiles_per_item + lane;
    return (it < n_items && lane < tiles_per_item && t < total_tiles) ? __ldg(&tiles[t])
                                                                      : make_uint2(0u, 0u);
  };
  unsigned claim = 0;
  if (lane == 0) claim = atomicAdd(next_item, 1u);
  int item = (int)__shfl_sync(0xffffffffu, claim, 0);
  while (item < n_items) {
    if (lane == 0) claim = atomicAdd(next_item, 1u);
    const uint2 rec = records(item);
    if (pf_items > 0) {  // the tiles of the item pf_items ahead, one per lane
      const int fi = item + pf_items, ft = fi * tiles_per_item + lane;
      if (fi < n_items && lane < tiles_per_item && ft < total_tiles)
        prefetch_tile_record<PARITY, S, ESO>(consts, pops, __ldg(&tiles[ft]));
    }
    const int count = min(tiles_per_item, total_tiles - item * tiles_per_item);
    for (int j = 0; j < count; ++j) {
      // the tile's record: domain | x0 << 16, y0 | z0 << 16 (its first cell)
      const unsigned r0 = __shfl_sync(0xffffffffu, rec.x, j);
      const unsigned r1 = __shfl_sync(0xffffffffu, rec.y, j);
      const int4 ti = make_int4((int)(r0 & 0xFFFFu), (int)(r0 >> 16), (int)(r1 & 0xFFFFu),
                                (int)(r1 >> 16));
      const int lo = ti.x;
      if (lo != cur) {  // warp-uniform: reload the warp's slot
        __syncwarp();   // every lane is done with the previous domain's constants
        const int* src = reinterpret_cast<const int*>(consts + lo);
        int* dst = reinterpret_cast<int*>(&sW[warp]);
        for (int w = lane; w < (int)(sizeof(DomainConst) / 4); w += 32) dst[w] = __ldg(src + w);
        if (lane == 0) sPopW[warp] = static_cast<S*>(pops[lo]);
        __syncwarp();
        cur = lo;
      }
      const DomainConst& P = sW[warp];
      S* pop = sPopW[warp];
      float d[kF][kQ];
      if ((P.nx & (kTile - 1)) == 0) {
        // whole-tile rows: the tile and its neighbour tiles are warp-uniform
        const WarpTiles T = warp_tiles(P, ti.y, ti.z, ti.w);
        load_cell_rows<PARITY, S, ESO>(P, pop, T, lane, d);
        const float probe = collide_cell<false>(P, d, nullptr);
        if (!isfinite(probe)) atomicOr(flag, 1u);
        store_cell_rows<PARITY, S, SR, ESO>(P, pop, T, lane, d);
      } else {
        const int first = ti.y + P.nx * (ti.z + P.ny * ti.w);
        if (first + lane < P.ncell) {
          // this lane's (x, y, z): carry x past the row end (several rows when nx < 32)
          int x = ti.y + lane, y = ti.z, z = ti.w;
          while (x >= P.nx) {
            x -= P.nx;
            if (++y == P.ny) {
              y = 0;
              ++z;
            }
          }
          const CellIndex c = make_index(P, x, y, z);
          load_cell<PARITY, false, S>(P, pop, nullptr, c, d);
          const float probe = collide_cell<false>(P, d, nullptr);
          if (!isfinite(probe)) atomicOr(flag, 1u);
          store_cell<PARITY, S, SR>(P, pop, c, d);
        }
      }
    }
    item = (int)__shfl_sync(0xffffffffu, claim, 0);
  }
}

}  // namespace batch_kernels
}  // namespace lbm

using lbm::batch_kernels::k_batch_step;

struct lbm_batch {
  int n = 0;
  int device = 0;              // CUDA device current at lbm_batch_create; every call runs there
  std::vector<lbm_params> prm;
  std::vector<DomainConst> P;
  std::vector<double> dt, tau_R, tau_q, rho_ref, E_ref;
  std::vector<size_t> offset;   // byte offset of each domain's populations
  long long total_cells = 0;
  void* pool = nullptr;
  int store = LBM_STORE_F32;
  bool sround = false;         // 16-bit storage rounded stochastically (all domains)
  bool eso = false;            // esoteric-twist streaming (all domains)
  DomainConst* d_consts = nullptr;
  void** d_pops = nullptr;
  unsigned* d_maxbits = nullptr;  // per-field maxima for the FP16 scales at init
  uint2* d_tiles = nullptr;    // per tile: domain | x << 16, y | z << 16 of its first cell
  unsigned* d_counter = nullptr;  // work-item counter of the persistent kernel
  int total_tiles = 0;
  int tiles_per_item = 4;      // layout tiles a warp takes at a time
  int prefetch_tiles = 0;      // L2 prefetch distance in tiles (0: off)
  int block = 64;
  int variant = 0;             // register budget: 0 -> 3, 1 -> 4 blocks of 128 per SM
  int grid = 0;
  unsigned* flag = nullptr;
  float* ghost = nullptr;  // unused by periodic domains; a valid pointer for the plain kernel
  float* trig = nullptr;   // TGV table of the domain being initialised (largest domain's size)
  float* dufield = nullptr;  // diagnostics scratch, sized for the largest domain (first use)
  double* dpartials = nullptr;
  double* dout = nullptr;
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

void* domain_pop(lbm_batch* b, int d) { return static_cast<char*>(b->pool) + b->offset[d]; }

template <int P, int M, typename S, bool SR, bool ESO>
void* kernel_ptr() {
  return reinterpret_cast<void*>(k_batch_step<P, M, S, SR, ESO>);
}

template <typename S_, bool SR_, bool ESO_>
struct Form {
  using S = S_;
  static constexpr bool SR = SR_;
  static constexpr bool ESO = ESO_;
};

template <bool ESO, typename F>
auto with_form_map(const lbm_batch* b, F&& f) {
  if (b->store == LBM_STORE_F32) return f(Form<float, false, ESO>{});
  if (b->store == LBM_STORE_F16)
    return b->sround ? f(Form<__half, true, ESO>{}) : f(Form<__half, false, ESO>{});
  return b->sround ? f(Form<__nv_bfloat16, true, ESO>{}) : f(Form<__nv_bfloat16, false, ESO>{});
}

// Calls f with the Form (storage type, rounding, streaming map) of the batch's kernels.
template <typename F>
auto with_form(const lbm_batch* b, F&& f) {
  return b->eso ? with_form_map<true>(b, f) : with_form_map<false>(b, f);
}

// Grid size for the current block size and register budget: every block resident.
lbm_status size_grid(lbm_batch* b) {
  int per_sm = 0;
  void* fn = with_form(b, [&](auto f) {
    using F = decltype(f);
    return b->variant ? kernel_ptr<0, 4, typename F::S, F::SR, F::ESO>()
                      : kernel_ptr<0, 3, typename F::S, F::SR, F::ESO>();
  });
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, b->block, 0);
  if (e != cudaSuccess || per_sm < 1) return fail(LBM_E_CUDA, "batched kernel does not fit on an SM");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int warps_needed = (b->total_tiles + b->tiles_per_item - 1) / b->tiles_per_item;
  const int blocks_needed = (warps_needed * 32 + b->block - 1) / b->block;
  b->grid = std::max(1, std::min(per_sm * sms, blocks_needed));
  b->graphs_valid = false;
  return LBM_OK;
}

template <typename S, bool SR, bool ESO>
void launch_typed(lbm_batch* b, int parity, cudaStream_t s) {
  const dim3 g(b->grid), bl(b->block);
  const int pf_items = b->prefetch_tiles > 0 ? std::max(1, b->prefetch_tiles / b->tiles_per_item) : 0;
#define LBM_BATCH_LAUNCH(PAR, MB)                                                           \
  k_batch_step<PAR, MB, S, SR, ESO><<<g, bl, 0, s>>>(b->d_consts, b->d_pops, b->d_tiles,  \
                                                     b->total_tiles, b->tiles_per_item,     \
                                                     pf_items, b->d_counter, b->flag)
  if (b->variant) {
    if (parity) LBM_BATCH_LAUNCH(1, 4);
    else LBM_BATCH_LAUNCH(0, 4);
  } else {
    if (parity) LBM_BATCH_LAUNCH(1, 3);
    else LBM_BATCH_LAUNCH(0, 3);
  }
#undef LBM_BATCH_LAUNCH
}

// One persistent launch: zero the work-item counter, then the kernel.
cudaError_t launch_batch(lbm_batch* b, int parity, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  with_form(b, [&](auto f) {
    using F = decltype(f);
    launch_typed<typename F::S, F::SR, F::ESO>(b, parity, s);
  });
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
  if (n > 65535) return fail(LBM_E_INVAL, "at most 65535 domains in one batch");
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return fail(LBM_E_NOMEM, "host allocation failed");
  b->n = n;
  b->store = params[0].store;
  b->sround = params[0].stochastic_round != 0 && params[0].store != LBM_STORE_F32;
  b->eso = params[0].streaming == 1;
  b->prefetch_tiles = b->store == LBM_STORE_F32 ? 0 : kDefaultPrefetch16;
  size_t bytes = 0;
  for (int d = 0; d < n; ++d) {
    lbm_status s = validate(&params[d]);
    if (s != LBM_OK) {
      delete b;
      return fail(s, "domain %d: %s", d, g_last_error.c_str());
    }
    if (params[d].bc_x != 0 || params[d].store != params[0].store) {
      delete b;
      return fail(LBM_E_INVAL, "domain %d: the batched mode takes periodic domains of one storage type", d);
    }
    if (params[d].streaming != params[0].streaming) {
      delete b;
      return fail(LBM_E_INVAL, "domain %d: the batched mode takes one streaming map (streaming)", d);
    }
    if (params[d].nx > 65535) {  // tile records hold 16-bit coordinates
      delete b;
      return fail(LBM_E_INVAL, "domain %d: the batched mode takes nx <= 65535", d);
    }
    if (params[d].stochastic_round != params[0].stochastic_round) {
      delete b;
      return fail(LBM_E_INVAL, "domain %d: the batched mode takes one rounding mode (stochastic_round)", d);
    }
    b->prm.push_back(params[d]);
    double dt, tR, tq;
    derive(&params[d], &dt, &tR, &tq);
    DomainConst P;
    fill_const(&params[d], dt, tR, tq, &P);
    P.pf_tiles = b->store == LBM_STORE_F32 ? 0 : kDefaultPrefetch16;  // the sequential launches
    b->P.push_back(P);
    b->dt.push_back(dt);
    b->tau_R.push_back(tR);
    b->tau_q.push_back(tq);
    b->rho_ref.push_back(0.0);
    b->E_ref.push_back(0.0);
    b->offset.push_back(bytes);
    bytes += (size_t)P.ntile * kP * kTile * elem_size(params[0].store);
    b->total_cells += P.ncell;
  }
  b->stream = static_cast<cudaStream_t>(params[0].cuda_stream);
  {  // the first CUDA call: everything above is validated on the host
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return fail(LBM_E_CUDA, "no current CUDA device: %s", cudaGetErrorString(e));
    }
  }
  auto cleanup = [&](lbm_status st) {
    lbm_batch_destroy(b);
    return st;
  };
  if (cudaMalloc(&b->pool, bytes) != cudaSuccess) {
    cudaGetLastError();
    b->pool = nullptr;
    return cleanup(fail(LBM_E_NOMEM, "cudaMalloc of %zu batch bytes failed", bytes));
  }
  std::vector<void*> ptrs(n);
  for (int d = 0; d < n; ++d) ptrs[d] = domain_pop(b, d);
  std::vector<int> prefix(n + 1, 0);
  for (int d = 0; d < n; ++d) prefix[d + 1] = prefix[d] + (int)b->P[d].ntile;
  b->total_tiles = prefix[n];
  std::vector<uint2> tiles((size_t)b->total_tiles);
  for (int d = 0; d < n; ++d) {
    const DomainConst& P = b->P[d];
    for (long long j = 0; j < P.ntile; ++j) {
      const long long first = j * kTile;
      const unsigned x0 = (unsigned)(first % P.nx), y0 = (unsigned)((first / P.nx) % P.ny);
      const unsigned z0 = (unsigned)(first / ((long long)P.nx * P.ny));
      tiles[(size_t)prefix[d] + j] = make_uint2((unsigned)d | (x0 << 16), y0 | (z0 << 16));
    }
  }
  size_t max_table = 0;
  for (int d = 0; d < n; ++d)
    max_table = std::max(max_table, tgv_table_floats(b->P[d].nx, b->P[d].ny, b->P[d].nz));
  if (cudaMalloc(&b->d_consts, sizeof(DomainConst) * n) != cudaSuccess ||
      cudaMalloc(&b->d_pops, sizeof(void*) * n) != cudaSuccess ||
      cudaMalloc(&b->d_maxbits, 64 + kF * sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&b->d_tiles, sizeof(uint2) * tiles.size()) != cudaSuccess ||
      cudaMalloc(&b->d_counter, 64) != cudaSuccess ||
      cudaMalloc(&b->flag, 64) != cudaSuccess || cudaMalloc(&b->ghost, 256) != cudaSuccess ||
      cudaMalloc(&b->trig, sizeof(float) * max_table) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(LBM_E_NOMEM, "cudaMalloc of batch tables failed"));
  }
  if (cudaMemcpy(b->d_pops, ptrs.data(), sizeof(void*) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_tiles, tiles.data(), sizeof(uint2) * tiles.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->flag, 0, 64) != cudaSuccess)
    return cleanup(fail(LBM_E_CUDA, "batch table upload failed"));
  for (int d = 0; d < n; ++d) b->P[d].check = b->flag + 2;  // the checked build's address count
  lbm_status s = upload_consts(b);
  if (s != LBM_OK) return cleanup(s);
  s = size_grid(b);
  if (s != LBM_OK) return cleanup(s);
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    return cleanup(fail(LBM_E_CUDA, "cudaStreamCreate failed"));
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_OK;
  DeviceScope scope(b->device);  // best effort: release what can be released either way
  cudaStreamSynchronize(b->stream);
  if (b->g_pair) cudaGraphExecDestroy(b->g_pair);
  if (b->pool) cudaFree(b->pool);
  if (b->d_consts) cudaFree(b->d_consts);
  if (b->d_pops) cudaFree(b->d_pops);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->d_maxbits) cudaFree(b->d_maxbits);
  if (b->flag) cudaFree(b->flag);
  if (b->ghost) cudaFree(b->ghost);
  if (b->trig) cudaFree(b->trig);
  if (b->dufield) cudaFree(b->dufield);
  if (b->dpartials) cudaFree(b->dpartials);
  if (b->dout) cudaFree(b->dout);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return LBM_OK;
}

lbm_status lbm_batch_init_tgv(lbm_batch* b, const double* U0, const double* M0, const double* rho0) {
  if (!b || !U0 || !M0 || !rho0) return fail(LBM_E_INVAL, "NULL argument");
  LBM_ON_DEVICE(b->device);
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
    InitSpec sp;
    std::vector<float> table;
    tgv_spec(b->P[d], p.gamma, U0[d], M0[d], rho0[d], p.dx, &sp, &table);
    // pageable source: returns once staged, after the previous domain's kernels
    LBM_CUDA(cudaMemcpyAsync(b->trig, table.data(), sizeof(float) * table.size(),
                             cudaMemcpyHostToDevice, b->stream));
    sp.trig = b->trig;
    for (int k = 0; k < kF; ++k) b->P[d].scale[k] = b->P[d].inv_scale[k] = 1.0f;
    if (b->store == LBM_STORE_F16) {  // per-field scale max|f - w Q_ref| / 1024, as for one domain
      LBM_CUDA(cudaMemsetAsync(b->d_maxbits, 0, kF * sizeof(unsigned), b->stream));
      LBM_CUDA(launch_init(b->P[d], b->store, sp, 0, domain_pop(b, d), nullptr, b->d_maxbits, nullptr,
                           b->stream));
      unsigned bits[kF];
      LBM_CUDA(cudaMemcpyAsync(bits, b->d_maxbits, sizeof(bits), cudaMemcpyDeviceToHost, b->stream));
      LBM_CUDA(cudaStreamSynchronize(b->stream));
      for (int k = 0; k < kF; ++k) {
        float m;
        std::memcpy(&m, &bits[k], sizeof(m));
        const float sk = (std::isfinite(m) && m > 0.0f) ? m / 1024.0f : 1.0f;
        b->P[d].scale[k] = sk;
        b->P[d].inv_scale[k] = 1.0f / sk;
      }
    }
    LBM_CUDA(launch_init(b->P[d], b->store, sp, 1, domain_pop(b, d), nullptr, nullptr, nullptr,
                         b->stream));
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
  Range range_("lbm_batch_step");
  if (!b) return fail(LBM_E_INVAL, "batch is NULL");
  LBM_ON_DEVICE(b->device);
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
  Range range_("lbm_batch_step_sequential");
  if (!b) return fail(LBM_E_INVAL, "batch is NULL");
  LBM_ON_DEVICE(b->device);
  if (n < 0) return fail(LBM_E_INVAL, "n must be >= 0");
  if (!b->initialized) return fail(LBM_E_STATE, "lbm_batch_step_sequential before an init");
  if (b->nonfinite) return fail(LBM_E_NONFINITE, "non-finite moments were detected earlier");
  for (int j = 0; j < n; ++j) {
    const int parity = (int)(b->step & 1);
    for (int d = 0; d < b->n; ++d) {
      const int bx = std::min(128, ((b->P[d].nx + 31) / 32) * 32);
      LBM_CUDA(launch_step(b->P[d], b->store, parity, domain_pop(b, d), b->ghost, b->flag, bx, 1,
                           b->stream));
    }
    b->step += 1;
  }
  return LBM_OK;
}

lbm_status lbm_batch_synchronize(lbm_batch* b) {
  if (!b) return fail(LBM_E_INVAL, "batch is NULL");
  LBM_ON_DEVICE(b->device);
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
  LBM_ON_DEVICE(b->device);
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
  cudaError_t e = launch_moments(P, b->store, (int)(b->step & 1), domain_pop(b, domain), b->ghost,
                                 which, dev, dtype == LBM_DT_F64, 0, P.ncell, b->stream);
  if (e == cudaSuccess && !dst_on_device)
    e = cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess && !dst_on_device) e = cudaStreamSynchronize(b->stream);
  if (!dst_on_device) cudaFree(dev);
  if (e != cudaSuccess) return fail(LBM_E_CUDA, "batch moments failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_batch_diag(lbm_batch* b, int domain, lbm_diag_t* out) {
  Range range_("lbm_batch_diag");
  if (!b || !out) return fail(LBM_E_INVAL, "NULL argument");
  LBM_ON_DEVICE(b->device);
  if (domain < 0 || domain >= b->n) return fail(LBM_E_INVAL, "domain index out of range");
  if (!b->initialized) return fail(LBM_E_STATE, "lbm_batch_diag before an init");
  if (!b->dufield) {
    long long most = 0;
    for (int d = 0; d < b->n; ++d) most = std::max(most, b->P[d].ncell);
    if (cudaMalloc(&b->dufield, sizeof(float) * 4 * (size_t)most) != cudaSuccess ||
        cudaMalloc(&b->dpartials, sizeof(double) * (size_t)kDiagBlocks * (kDiagA + 2)) != cudaSuccess ||
        cudaMalloc(&b->dout, sizeof(double) * 16) != cudaSuccess) {
      cudaGetLastError();
      if (b->dufield) cudaFree(b->dufield);
      if (b->dpartials) cudaFree(b->dpartials);
      if (b->dout) cudaFree(b->dout);
      b->dufield = nullptr;
      b->dpartials = b->dout = nullptr;
      return fail(LBM_E_NOMEM, "diagnostic scratch allocation failed");
    }
  }
  const DomainConst& P = b->P[domain];
  double r[16] = {0};
  unsigned flag = 0;
  LBM_CUDA(launch_diag(P, b->store, (int)(b->step & 1), domain_pop(b, domain), b->ghost, b->dufield,
                       b->dpartials, b->dout, b->stream));
  LBM_CUDA(cudaMemcpyAsync(r, b->dout, sizeof(double) * (kDiagA + 2), cudaMemcpyDeviceToHost,
                           b->stream));
  LBM_CUDA(cudaMemcpyAsync(&flag, b->flag, sizeof(flag), cudaMemcpyDeviceToHost, b->stream));
  LBM_CUDA(cudaStreamSynchronize(b->stream));
  const double n = (double)P.ncell;
  out->step = (double)b->step;
  out->time = (double)b->step * b->dt[domain];
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
  if ((flag & 1u) || r[6] > 0) {
    b->nonfinite = true;
    return fail(LBM_E_NONFINITE, "non-finite moments detected");
  }
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
                              float* ms_per_step, int* prefetch_tiles) {
  if (!b) return fail(LBM_E_INVAL, "batch is NULL");
  LBM_ON_DEVICE(b->device);
  if (!b->initialized) return fail(LBM_E_STATE, "autotune needs an initialised batch");
  if (steps_per_trial < 2) steps_per_trial = 8;
  steps_per_trial += steps_per_trial & 1;  // whole pairs keep the parity
  const int items[] = {1, 2, 4, 8, 16, 32};  // at most 32: one tile record per lane
  const int blocks[] = {64, 128};
  const int variants[] = {0, 1};
  cudaEvent_t a, e;
  LBM_CUDA(cudaEventCreate(&a));
  LBM_CUDA(cudaEventCreate(&e));
  // Mean time of one step of the current configuration over steps_per_trial steps
  // (after a warm-up pair).
  auto trial = [&](float* ms) -> lbm_status {
    lbm_status s = size_grid(b);
    if (s != LBM_OK) return s;
    for (int j = 0; j < 2; ++j) LBM_CUDA(launch_batch(b, (int)((b->step + j) & 1), b->stream));
    b->step += 2;
    LBM_CUDA(cudaEventRecord(a, b->stream));
    for (int j = 0; j < steps_per_trial; ++j)
      LBM_CUDA(launch_batch(b, (int)((b->step + j) & 1), b->stream));
    b->step += steps_per_trial;
    LBM_CUDA(cudaEventRecord(e, b->stream));
    LBM_CUDA(cudaEventSynchronize(e));
    LBM_CUDA(cudaEventElapsedTime(ms, a, e));
    *ms /= (float)steps_per_trial;
    return LBM_OK;
  };
  float best = 1e30f;
  int best_i = b->tiles_per_item, best_b = b->block, best_v = b->variant;
  lbm_status st = LBM_OK;
  // First items x blocks x budgets at the current prefetch distance, then the
  // distance for the fastest of them.
  for (int v : variants)
    for (int bl : blocks)
      for (int it : items) {
        if (st != LBM_OK) break;
        b->variant = v;
        b->block = bl;
        b->tiles_per_item = it;
        float ms = 0;
        st = trial(&ms);
        if (st == LBM_OK && ms < best) {
          best = ms;
          best_i = it;
          best_b = bl;
          best_v = v;
        }
      }
  b->tiles_per_item = best_i;
  b->block = best_b;
  b->variant = best_v;
  int best_pf = b->prefetch_tiles;
  for (int pf : {0, 512, 1024, 2048}) {
    if (st != LBM_OK || pf == best_pf) continue;
    b->prefetch_tiles = pf;
    float ms = 0;
    st = trial(&ms);
    if (st == LBM_OK && ms < best) {
      best = ms;
      best_pf = pf;
    }
  }
  b->prefetch_tiles = best_pf;
  cudaEventDestroy(a);
  cudaEventDestroy(e);
  if (st != LBM_OK) return st;
  lbm_status s = size_grid(b);
  if (s != LBM_OK) return s;
  if (tile_cells) *tile_cells = best_i * kTile;
  if (block_threads) *block_threads = best_b;
  if (ms_per_step) *ms_per_step = best;
  if (prefetch_tiles) *prefetch_tiles = best_pf;
  return LBM_OK;
}

lbm_status lbm_batch_check_count(const lbm_batch* b, unsigned long long* count) {
  if (!b || !count) return fail(LBM_E_INVAL, "NULL argument");
#ifdef LBM_CHECKED
  LBM_ON_DEVICE(b->device);
  unsigned v = 0;
  LBM_CUDA(cudaMemcpyAsync(&v, b->flag + 2, sizeof(v), cudaMemcpyDeviceToHost, b->stream));
  LBM_CUDA(cudaStreamSynchronize(b->stream));
  *count = v;
  return LBM_OK;
#else
  *count = 0;
  return fail(LBM_E_STATE, "not a checked build (compiled without LBM_CHECKED)");
#endif
}

lbm_status lbm_batch_set_prefetch(lbm_batch* b, int tiles) {
  if (!b) return fail(LBM_E_INVAL, "batch is NULL");
  if (tiles < 0 || tiles > kMaxPrefetch)
    return fail(LBM_E_INVAL, "prefetch distance must be 0 to %d tiles", kMaxPrefetch);
  b->prefetch_tiles = tiles;
  b->graphs_valid = false;
  return LBM_OK;
}

}  // extern "C"

// Host-side declarations shared by the translation units of liblbm.so.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "lbm_device.cuh"

namespace lbm {

// (x, y, z) of a linear cell index; cell counts are below 2^31, so 32-bit unsigned
// division suffices (much cheaper than 64-bit).
__device__ __forceinline__ void cell_xyz(const DomainConst& P, long long cell, int& x, int& y,
                                         int& z) {
  const unsigned c = (unsigned)cell;
  const unsigned yz = c / (unsigned)P.nx;
  x = (int)(c - yz * (unsigned)P.nx);
  const unsigned zz = yz / (unsigned)P.ny;
  y = (int)(yz - zz * (unsigned)P.ny);
  z = (int)zz;
}

// Fused step: one launch per time step, grid (ceil(nx/block_x), ny, nz), block_x in
// {32, 64, 96, 128}; variant selects the register budget (0: 170, 1: 128 registers).
cudaError_t launch_step_f32(const DomainConst& P, int parity, void* pop, const float* ghost,
                            unsigned* flag, int block_x, int variant, cudaStream_t s);
cudaError_t launch_step_f16(const DomainConst& P, int parity, void* pop, const float* ghost,
                            unsigned* flag, int block_x, int variant, cudaStream_t s);
cudaError_t launch_step_bf16(const DomainConst& P, int parity, void* pop, const float* ghost,
                             unsigned* flag, int block_x, int variant, cudaStream_t s);

// The same step with its reads staged through shared memory by bulk asynchronous copies
// (step_staged_*.cu; variants 2, 3, 4). Only for periodic domains whose rows are whole
// 32-cell tiles, rounding to nearest. prepare sets the kernels' shared-memory limit and returns the
// persistent grid size (SMs x resident blocks, at most one warp per tile). skip_first
// is a failure-detection test hook (one warp's first copy is not issued, so its
// bounded wait runs out and the step reports a stalled copy).
constexpr int kFirstStagedVariant = 2, kLastStagedVariant = 4;
// L2 prefetch distance (tiles ahead) of the plain and batched step kernels for 16-bit
// storage when not tuned: about half the warps resident on the GPU at once, the
// fastest distance measured at 512^3 (FP32 storage gains nothing from it and starts
// with 0); the largest distance accepted.
constexpr int kDefaultPrefetch16 = 1024;
constexpr int kMaxPrefetch = 1 << 20;
inline bool staged_eligible(const DomainConst& P) {
  // no stochastic rounding and no esoteric twist there
  return P.bc_x == 0 && P.nx % 32 == 0 && P.sround == 0 && P.eso == 0;
}
cudaError_t staged_prepare_f32(const DomainConst& P, int variant, int* grid);
cudaError_t staged_prepare_f16(const DomainConst& P, int variant, int* grid);
cudaError_t staged_prepare_bf16(const DomainConst& P, int variant, int* grid);
cudaError_t launch_step_staged_f32(const DomainConst& P, int parity, void* pop, unsigned* flag,
                                   int variant, int grid, int skip_first, cudaStream_t s);
cudaError_t launch_step_staged_f16(const DomainConst& P, int parity, void* pop, unsigned* flag,
                                   int variant, int grid, int skip_first, cudaStream_t s);
cudaError_t launch_step_staged_bf16(const DomainConst& P, int parity, void* pop, unsigned* flag,
                                    int variant, int grid, int skip_first, cudaStream_t s);

// The same step that also computes the diagnostics of the state it reads (step_diag_*.cu):
// writes u and mu_local to ufield (4 floats per cell) and one record of 17 floats per
// warp to rec (step_diag_record_count of them; block_x as for launch_step_*).
cudaError_t launch_step_diag_f32(const DomainConst& P, int parity, void* pop, const float* ghost,
                                 unsigned* flag, float* ufield, float* rec, int block_x,
                                 cudaStream_t s);
cudaError_t launch_step_diag_f16(const DomainConst& P, int parity, void* pop, const float* ghost,
                                 unsigned* flag, float* ufield, float* rec, int block_x,
                                 cudaStream_t s);
cudaError_t launch_step_diag_bf16(const DomainConst& P, int parity, void* pop, const float* ghost,
                                  unsigned* flag, float* ufield, float* rec, int block_x,
                                  cudaStream_t s);
constexpr int kDiagRecFloats = 17;  // words of one warp record
inline long long step_diag_record_count(const DomainConst& P, int block_x) {
  return (long long)((P.nx + block_x - 1) / block_x) * P.ny * P.nz * (block_x / 32);
}

// Initial states (init.cu). kind: 0 TGV, 1 Riemann, 2 caller fields (rho, u, p),
// 3 caller zeroth moments (14 fields). Host-computed FP32 constants; the device works
// in FP32 only (the deviations from Q_ref are formed without cancellation).
struct InitSpec {
  int kind;
  // TGV (kind 0): U0, rho0 U0^2/16, 1/T0, p0, T0 and the differences between the FP64
  // reference (rho0, p0/(gamma-1)) and its FP32 copy in DomainConst
  const float* trig;                   // per axis: sin, cos, cos 2x of the nodes i dx
  float U0, c_dp, inv_T0, p0, T0, drho_ref, dE_ref;
  // Riemann (kind 1): deviations of (rho, rho u, E) and (rho, u, p), T of the two states
  int axis, split;
  float sD[2][5], sprim[2][5], sT[2];
  // caller fields (kinds 2, 3): device (or mapped host) array, FP64 or FP32
  const void* fields;
  int fields_f64;
  float inv_gm1_hi, inv_gm1_lo;        // 1/(gamma - 1) as a float-float pair
};
// Floats of the TGV table of a domain (3 per node of each axis).
size_t tgv_table_floats(int nx, int ny, int nz);
// Host set-up of the three kinds of initial state; P must hold the FP32 Q_ref already.
void tgv_spec(const DomainConst& P, double gamma, double U0, double M0, double rho0, double dx,
              InitSpec* sp, std::vector<float>* table);
void riemann_spec(const DomainConst& P, double gamma, int axis, int split, const double left[3],
                  const double right[3], InitSpec* sp);
void fields_spec(double gamma, int kind, const void* fields, int f64, InitSpec* sp);
// mode 0: per-field max |f - w Q_ref| into maxbits[14] (float bits); mode 1: write
// the encoded populations (canonical slots) and the held-x ghost layers, and set *bad
// (when not null) if some cell's state is not finite.
cudaError_t launch_init(const DomainConst& P, int store, const InitSpec& spec, int mode, void* pop,
                        float* ghost, unsigned* maxbits, unsigned* bad, cudaStream_t s);
// The cells whose fields fix Q_ref: every cell of domains up to kSampleRuns runs of 32
// cells (2^20 cells); beyond that every run_stride-th run of 32 consecutive cells, about
// 2^20 cells in all (a reference near the data is all the shifted storage needs).
constexpr long long kSampleRuns = 1LL << 15;
struct FieldSample {
  long long run_stride;  // sampled runs: 0, run_stride, 2 run_stride, ...
  long long cells;       // cells in the sample
};
FieldSample field_sample(long long ncell);
// Sums of rho and E over the sample of the caller fields (kind 2 or 3) into sums[0..2),
// in a fixed order; sums must hold kFieldSumDoubles doubles (the rest is block scratch).
constexpr int kFieldSumDoubles = 2 + 2 * 1216;
cudaError_t launch_field_means(const DomainConst& P, const InitSpec& spec, double* sums,
                               cudaStream_t s);

// Outputs (io.cu); parity and held-x are runtime values here.
// Cells [c0, c0 + cnt) into out[field][cnt].
cudaError_t launch_moments(const DomainConst& P, int store, int parity, const void* pop,
                           const float* ghost, int which, void* out, int out_f64, long long c0,
                           long long cnt, cudaStream_t s);
cudaError_t launch_sensor(const DomainConst& P, int store, int parity, const void* pop,
                          const float* ghost, void* out, int out_f64, long long c0, long long cnt,
                          cudaStream_t s);
// One population array (k, i) in canonical order, decoded (dtype F32/F64) or native.
cudaError_t launch_pop_get(const DomainConst& P, int store, int parity, const void* pop,
                           const float* ghost, int k, int i, void* out, int dtype, cudaStream_t s);
cudaError_t launch_pop_set(const DomainConst& P, int store, int parity, void* pop, int k, int i,
                           const void* in, int dtype, cudaStream_t s);
// Raw stored values of storage slot `slot` on plane z, all fields, [k][y][x] in the
// storage's element size: copied into buf (set = 0) or from buf (set = 1).
cudaError_t launch_plane(const DomainConst& P, int store, void* pop, int z, int slot, void* buf,
                         int set, cudaStream_t s);

// Diagnostics (diag.cu).
constexpr int kDiagA = 13;  // sums: rho mx my mz E ke nonfinite | max: mach cfl | min: rho T
constexpr int kDiagBlocks = 1216;
// ufield: 4 floats per cell of scratch; partials: kDiagBlocks * (kDiagA + 2) doubles.
cudaError_t launch_diag(const DomainConst& P, int store, int parity, const void* pop,
                        const float* ghost, float* ufield, double* partials, double* out16,
                        cudaStream_t s);
// Finishes the diagnostics from the records of launch_step_diag_* (nrec of them) and
// the u field it wrote; same partials and output as launch_diag.
cudaError_t launch_diag_records(const DomainConst& P, const float* rec, long long nrec,
                                const float* ufield, double* partials, double* out16,
                                cudaStream_t s);

}  // namespace lbm

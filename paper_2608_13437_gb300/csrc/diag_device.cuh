// Per-cell contributions to the diagnostics (Sec. 3.2, Eq. 7) and their reductions,
// shared by the separate diagnostic pass (diag.cu) and the step kernel's diagnostic
// variant (step_diag.cuh). Per-cell values are FP32, computed with explicitly rounded
// operations from the step's own moments and closure, so both kernels produce
// identical values for a cell. Sums are carried as float-float pairs (Knuth's
// two-sum: hi + lo holds about 48 significant bits) and become FP64 only once per
// block, because FP64 throughput on this part is a small fraction of FP32's; extrema
// stay FP32 (exact in any order).
#pragma once

#include "lbm_device.cuh"

namespace lbm {

struct FF {
  float hi, lo;
};

// s + e == a + b exactly (round to nearest, no overflow).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

__device__ __forceinline__ void ff_add(FF& a, float x) {
  float s, e;
  two_sum(a.hi, x, s, e);
  a.hi = s;
  a.lo = __fadd_rn(a.lo, e);
}

__device__ __forceinline__ void ff_merge(FF& a, const FF& b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  a.hi = __fadd_rn(s, e);  // renormalise (fast two-sum)
  a.lo = __fsub_rn(e, __fsub_rn(a.hi, s));
}

__device__ __forceinline__ double ff_value(const FF& a) { return (double)a.hi + (double)a.lo; }

// Sums: 0 rho deviations, 1-3 momentum, 4 E deviations, 5 rho |u|^2 / 2.
constexpr int kDiagSums = 6;
// One warp record of the diagnostic step: the sums' (hi, lo) pairs, the non-finite
// count, max Mach, max (max_a |u_a| + a) dt/dx, min rho, min T.
constexpr int kDiagRecWords = 2 * kDiagSums + 5;

struct DiagAcc {
  FF s[kDiagSums];
  float nonfinite;
  float max_mach, max_cfl, min_rho, min_T;
};

__device__ __forceinline__ void diag_zero(DiagAcc& a) {
#pragma unroll
  for (int j = 0; j < kDiagSums; ++j) a.s[j].hi = a.s[j].lo = 0.0f;
  a.nonfinite = 0.0f;
  a.max_mach = a.max_cfl = 0.0f;
  a.min_rho = a.min_T = INFINITY;
}

__device__ __forceinline__ void diag_add_cell(const DomainConst& P, const CellDiag& c, DiagAcc& a) {
#pragma unroll
  for (int j = 0; j < 5; ++j) ff_add(a.s[j], c.D[j]);
  ff_add(a.s[5], mul(0.5f, fma_(c.m[2], c.u[2], fma_(c.m[1], c.u[1], mul(c.m[0], c.u[0])))));
  if (!c.finite) {
    a.nonfinite = __fadd_rn(a.nonfinite, 1.0f);
    return;
  }
  const float snd = sqrtf(mul(P.gamma, c.T));
  const float umag = sqrtf(fma_(c.u[2], c.u[2], fma_(c.u[1], c.u[1], mul(c.u[0], c.u[0]))));
  const float umax = fmaxf(fabsf(c.u[0]), fmaxf(fabsf(c.u[1]), fabsf(c.u[2])));
  a.max_mach = fmaxf(a.max_mach, __fdiv_rn(umag, snd));
  a.max_cfl = fmaxf(a.max_cfl, __fdiv_rn(add(umax, snd), P.c));
  a.min_rho = fminf(a.min_rho, c.rho);
  a.min_T = fminf(a.min_T, c.T);
}

__device__ __forceinline__ void diag_merge(DiagAcc& a, const DiagAcc& b) {
#pragma unroll
  for (int j = 0; j < kDiagSums; ++j) ff_merge(a.s[j], b.s[j]);
  a.nonfinite = __fadd_rn(a.nonfinite, b.nonfinite);
  a.max_mach = fmaxf(a.max_mach, b.max_mach);
  a.max_cfl = fmaxf(a.max_cfl, b.max_cfl);
  a.min_rho = fminf(a.min_rho, b.min_rho);
  a.min_T = fminf(a.min_T, b.min_T);
}

// Tree reduction over the 32 lanes of a (full) warp; lane 0 holds the result.
__device__ __forceinline__ void diag_warp_reduce(DiagAcc& a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DiagAcc b;
#pragma unroll
    for (int j = 0; j < kDiagSums; ++j) {
      b.s[j].hi = __shfl_down_sync(0xffffffffu, a.s[j].hi, o);
      b.s[j].lo = __shfl_down_sync(0xffffffffu, a.s[j].lo, o);
    }
    b.nonfinite = __shfl_down_sync(0xffffffffu, a.nonfinite, o);
    b.max_mach = __shfl_down_sync(0xffffffffu, a.max_mach, o);
    b.max_cfl = __shfl_down_sync(0xffffffffu, a.max_cfl, o);
    b.min_rho = __shfl_down_sync(0xffffffffu, a.min_rho, o);
    b.min_T = __shfl_down_sync(0xffffffffu, a.min_T, o);
    diag_merge(a, b);
  }
}

__device__ __forceinline__ void diag_store_words(const DiagAcc& a, float* __restrict__ w) {
#pragma unroll
  for (int j = 0; j < kDiagSums; ++j) {
    w[2 * j] = a.s[j].hi;
    w[2 * j + 1] = a.s[j].lo;
  }
  w[12] = a.nonfinite;
  w[13] = a.max_mach;
  w[14] = a.max_cfl;
  w[15] = a.min_rho;
  w[16] = a.min_T;
}

__device__ __forceinline__ void diag_load_words(const float* __restrict__ w, DiagAcc& a) {
#pragma unroll
  for (int j = 0; j < kDiagSums; ++j) {
    a.s[j].hi = w[2 * j];
    a.s[j].lo = w[2 * j + 1];
  }
  a.nonfinite = w[12];
  a.max_mach = w[13];
  a.max_cfl = w[14];
  a.min_rho = w[15];
  a.min_T = w[16];
}

// A block's record in FP64 (kDiagA doubles): 0-5 the sums, 6 non-finite count,
// 7-8 zero, 9 max Mach, 10 max CFL, 11 min rho, 12 min T.
__device__ __forceinline__ void diag_store_partial(const DiagAcc& a, double* __restrict__ rec) {
#pragma unroll
  for (int j = 0; j < kDiagSums; ++j) rec[j] = ff_value(a.s[j]);
  rec[6] = a.nonfinite;
  rec[7] = rec[8] = 0.0;
  rec[9] = a.max_mach;
  rec[10] = a.max_cfl;
  rec[11] = a.min_rho;
  rec[12] = a.min_T;
}

}  // namespace lbm

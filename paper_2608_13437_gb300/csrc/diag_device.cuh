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
// count, max Mach^2, max (max_a |u_a| + a), min rho, min T. The square root of the
// Mach maximum and the division of the speed maximum by c = dx/dt (max CFL) are taken
// once, on the final totals: both maps are monotonic and correctly rounded, so the
// maximum commutes with them.
constexpr int kDiagRecWords = 2 * kDiagSums + 5;

struct DiagAcc {
  FF s[kDiagSums];
  float nonfinite;
  float max_mach2, max_speed, min_rho, min_T;
};

__device__ __forceinline__ void diag_zero(DiagAcc& a) {
#pragma unroll
  for (int j = 0; j < kDiagSums; ++j) a.s[j].hi = a.s[j].lo = 0.0f;
  a.nonfinite = 0.0f;
  a.max_mach2 = a.max_speed = 0.0f;
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
  const float gT = mul(P.gamma, c.T);  // a^2
  const float u2 = fma_(c.u[2], c.u[2], fma_(c.u[1], c.u[1], mul(c.u[0], c.u[0])));
  const float umax = fmaxf(fabsf(c.u[0]), fmaxf(fabsf(c.u[1]), fabsf(c.u[2])));
  // fmaxf drops NaN (a negative T), so the maxima stay non-negative and finite
  a.max_mach2 = fmaxf(a.max_mach2, __fdiv_rn(u2, gT));
  a.max_speed = fmaxf(a.max_speed, add(umax, sqrtf(gT)));
  a.min_rho = fminf(a.min_rho, c.rho);
  a.min_T = fminf(a.min_T, c.T);
}

__device__ __forceinline__ void diag_merge(DiagAcc& a, const DiagAcc& b) {
#pragma unroll
  for (int j = 0; j < kDiagSums; ++j) ff_merge(a.s[j], b.s[j]);
  a.nonfinite = __fadd_rn(a.nonfinite, b.nonfinite);
  a.max_mach2 = fmaxf(a.max_mach2, b.max_mach2);
  a.max_speed = fmaxf(a.max_speed, b.max_speed);
  a.min_rho = fminf(a.min_rho, b.min_rho);
  a.min_T = fminf(a.min_T, b.min_T);
}

__device__ __forceinline__ FF ff_select(bool p, const FF& a, const FF& b) {
  return FF{p ? a.hi : b.hi, p ? a.lo : b.lo};
}

__device__ __forceinline__ FF ff_shfl_xor(const FF& a, int o) {
  return FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// Order-preserving map of a float (not NaN) to a signed integer and back.
__device__ __forceinline__ int float_order(float v) {
  const int i = __float_as_int(v);
  return i < 0 ? i ^ 0x7FFFFFFF : i;
}
__device__ __forceinline__ float order_float(int i) { return __int_as_float(i < 0 ? i ^ 0x7FFFFFFF : i); }

// Reduces the accumulators of a full warp (every lane calls it) and writes the warp's
// record of kDiagRecWords words at w. The sums (padded to 8) go through a
// reduce-scatter butterfly: at lane distances 16, 8 and 4 a lane keeps half of the
// sums it holds, merged with its partner's, and hands the other half over, so lane l
// is left with sum l >> 2, which lanes 4q ... 4q + 3 then complete at distances 2 and
// 1; every sum meets the same partners in the same order as in a plain shuffle tree,
// and the float-float merge is commutative, so the sums equal that tree's bit for
// bit at about a quarter of its shuffles and merges. The extrema (non-negative maxima,
// minima in an order-preserving integer form) and the non-finite count take one
// warp-wide integer reduction each.
__device__ __forceinline__ void diag_warp_reduce_store(const DiagAcc& a, float* __restrict__ w) {
  const int lane = threadIdx.x & 31;
  FF v[8];
#pragma unroll
  for (int j = 0; j < kDiagSums; ++j) v[j] = a.s[j];
  v[6] = v[7] = FF{0.0f, 0.0f};
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  FF h4[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {  // keep sums 4 * b4 + k
    FF keep = ff_select(b4, v[k + 4], v[k]);
    ff_merge(keep, ff_shfl_xor(ff_select(b4, v[k], v[k + 4]), 16));
    h4[k] = keep;
  }
  FF h2[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {  // keep sums 4 * b4 + 2 * b3 + k
    FF keep = ff_select(b3, h4[k + 2], h4[k]);
    ff_merge(keep, ff_shfl_xor(ff_select(b3, h4[k], h4[k + 2]), 8));
    h2[k] = keep;
  }
  FF h = ff_select(b2, h2[1], h2[0]);  // keep sum lane >> 2
  ff_merge(h, ff_shfl_xor(ff_select(b2, h2[0], h2[1]), 4));
  ff_merge(h, ff_shfl_xor(h, 2));
  ff_merge(h, ff_shfl_xor(h, 1));
  const unsigned nonfinite = __reduce_add_sync(0xffffffffu, (unsigned)a.nonfinite);
  const unsigned mach2 = __reduce_max_sync(0xffffffffu, __float_as_uint(a.max_mach2));
  const unsigned speed = __reduce_max_sync(0xffffffffu, __float_as_uint(a.max_speed));
  const int min_rho = __reduce_min_sync(0xffffffffu, float_order(a.min_rho));
  const int min_T = __reduce_min_sync(0xffffffffu, float_order(a.min_T));
  const int q = lane >> 2;
  if ((lane & 3) == 0 && q < kDiagSums) {
    w[2 * q] = h.hi;
    w[2 * q + 1] = h.lo;
  }
  if (lane == 0) {
    w[12] = (float)nonfinite;
    w[13] = __uint_as_float(mach2);
    w[14] = __uint_as_float(speed);
    w[15] = order_float(min_rho);
    w[16] = order_float(min_T);
  }
}

__device__ __forceinline__ void diag_load_words(const float* __restrict__ w, DiagAcc& a) {
#pragma unroll
  for (int j = 0; j < kDiagSums; ++j) {
    a.s[j].hi = w[2 * j];
    a.s[j].lo = w[2 * j + 1];
  }
  a.nonfinite = w[12];
  a.max_mach2 = w[13];
  a.max_speed = w[14];
  a.min_rho = w[15];
  a.min_T = w[16];
}

// A block's record in FP64 (kDiagA doubles): 0-5 the sums, 6 non-finite count,
// 7-8 zero, 9 max Mach^2, 10 max speed |u|_max + a, 11 min rho, 12 min T.
__device__ __forceinline__ void diag_store_partial(const DiagAcc& a, double* __restrict__ rec) {
#pragma unroll
  for (int j = 0; j < kDiagSums; ++j) rec[j] = ff_value(a.s[j]);
  rec[6] = a.nonfinite;
  rec[7] = rec[8] = 0.0;
  rec[9] = a.max_mach2;
  rec[10] = a.max_speed;
  rec[11] = a.min_rho;
  rec[12] = a.min_T;
}

}  // namespace lbm

// Device-side building blocks of the fused compressible-NSF D3Q7 step:
// domain constants, storage codecs, the AA-pattern index maps and the per-cell
// moments -> closure -> sensor -> collision arithmetic.
//
// Scheme (Bukreev, Kummerlaender, Krause): 14 fields Q = (rho, rho u, E, tau, q),
// one D3Q7 population set each (Eq. 2, Sec. 2.2); linear equilibrium
// feq_{k,i} = w_i (Q_k + c_i . Phi_k / c_s^2) with w_0 = 1/4, w_{+-a} = 1/8,
// c_s^2 = c^2/4; BGK collision with the source on the weights (Sec. 2.2); the
// cell-local sensor and blended rate of Sec. 2.3 (Eqs. 3-6).
//
// Populations are held as deviations d = f - w_i Q_ref,k from a reference state
// Q_ref = (rho_ref, 0, 0, 0, E_ref, 0...) (the reference-shifted form the paper
// runs in single precision), so every sum below works on small numbers.
#pragma once

#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int kF = 14;   // fields
constexpr int kQ = 7;    // D3Q7 directions: 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z
constexpr int kP = kF * kQ;
constexpr float kSutherlandT = 0.4042f;

__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// Constants of one domain, passed by value to every kernel.
struct DomainConst {
  int nx, ny, nz, bc_x;
  long long ncell;
  long long ntile;    // 32-cell tiles of the population buffer
  float c, inv_c, half_inv_c, dt;
  float gm1;          // gamma - 1
  float gamma;
  float mu;           // reference viscosity
  float visc0;        // mu / tau_R
  float heat0;        // kappa / tau_q
  float inv_T_ref;
  float fmu_coef;     // 4 f_mu dt / dx^2 (Eq. 6)
  float C_sigma, J_min, omega_min;
  float src_R, src_q; // dS_k = src * Q_k for tau and q fields
  float rho_ref, E_ref;
  float scale[kF], inv_scale[kF];
  int sutherland, sensor_mode, collide;
  int sround;         // 16-bit storage rounds stochastically (1) or to nearest (0)
  int pf_tiles;       // L2 prefetch distance of the plain step kernel on whole-tile rows (0: off)
  int eso;            // storage map: 0 AA pattern, 1 esoteric twist (slots 2, 4, 6 shifted)
  double dx64;        // dx in FP64 (the diagnostics' gradient pass takes 1/dx from it)
  unsigned* check;    // checked builds: count of population addresses found outside the buffer
};

// Checked builds (-DLBM_CHECKED): every population tile and ghost-plane address is
// tested before use; one outside the buffer adds 1 to *P.check and the access is
// dropped (a load reads zero), so a bad index shows as a count instead of a fault.
// Other builds compile the test away.
#ifdef LBM_CHECKED
__device__ __forceinline__ bool lbm_check(const DomainConst& P, bool ok) {
  if (!ok && P.check) atomicAdd(P.check, 1u);
  return ok;
}
#define LBM_CHECK(P, cond) ::lbm::lbm_check((P), (cond))
#else
#define LBM_CHECK(P, cond) true
#endif

// ---------------------------------------------------------------- storage codecs
// Scalar codecs (dec/enc) and the vector forms used by the step kernel: V4 holds
// four consecutive fields of one direction of one cell, V2 two.
template <typename S>
struct Codec;

template <>
struct Codec<float> {
  using V4 = float4;
  using V2 = float2;
  static __device__ __forceinline__ float dec(float g, float) { return g; }
  static __device__ __forceinline__ float enc(float d, float) { return d; }
  static __device__ __forceinline__ double dec64(float g, double) { return (double)g; }
  static __device__ __forceinline__ void dec4(const V4& v, const float*, float o[4]) {
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
  static __device__ __forceinline__ void dec2(const V2& v, const float*, float o[2]) {
    o[0] = v.x; o[1] = v.y;
  }
  static __device__ __forceinline__ V4 enc4(const float i[4], const float*) {
    return make_float4(i[0], i[1], i[2], i[3]);
  }
  static __device__ __forceinline__ V2 enc2(const float i[2], const float*) {
    return make_float2(i[0], i[1]);
  }
};

// 16-bit codecs: pairs of values travel as one 32-bit word. kScaled: FP16 applies the
// per-field scale; BF16 has the exponent range of FP32 and stores unscaled (s = 1).
template <typename H, typename H2, bool kScaled>
struct Codec16 {
  using V4 = uint2;
  using V2 = unsigned;
  static __device__ __forceinline__ float2 to_f2(unsigned w);
  static __device__ __forceinline__ unsigned from_f2(float a, float b);
  static __device__ __forceinline__ void dec2w(unsigned w, const float* s, float* o) {
    const float2 f = to_f2(w);
    o[0] = kScaled ? f.x * s[0] : f.x;
    o[1] = kScaled ? f.y * s[1] : f.y;
  }
  static __device__ __forceinline__ void dec4(const V4& v, const float* s, float o[4]) {
    dec2w(v.x, s, o);
    dec2w(v.y, s + 2, o + 2);
  }
  static __device__ __forceinline__ void dec2(const V2& v, const float* s, float o[2]) {
    dec2w(v, s, o);
  }
  static __device__ __forceinline__ V4 enc4(const float i[4], const float* is) {
    if (!kScaled) return make_uint2(from_f2(i[0], i[1]), from_f2(i[2], i[3]));
    return make_uint2(from_f2(i[0] * is[0], i[1] * is[1]), from_f2(i[2] * is[2], i[3] * is[3]));
  }
  static __device__ __forceinline__ V2 enc2(const float i[2], const float* is) {
    if (!kScaled) return from_f2(i[0], i[1]);
    return from_f2(i[0] * is[0], i[1] * is[1]);
  }
  // Stochastic rounding of a pair (a to the low half, b to the high half): the
  // hardware conversion with random bits (cvt.rs, sm_100 and later) adds the low 16
  // bits of r below a's last kept place (FP16 uses 13 of them, BF16 all 16), the high
  // 16 bits below b's, and cuts what lies below. A value rounds away from zero with
  // probability equal to its distance from the value below, in ulps; FP16 subnormals
  // included.
  static __device__ __forceinline__ unsigned from_f2_sr(float a, float b, unsigned r);
  static __device__ __forceinline__ V4 enc4_sr(const float i[4], const float* is, unsigned r0,
                                               unsigned r1) {
    float a = i[0], b = i[1], c = i[2], e = i[3];
    if (kScaled) {
      a = a * is[0];
      b = b * is[1];
      c = c * is[2];
      e = e * is[3];
    }
    return make_uint2(from_f2_sr(a, b, r0), from_f2_sr(c, e, r1));
  }
  static __device__ __forceinline__ V2 enc2_sr(const float i[2], const float* is, unsigned r) {
    float a = i[0], b = i[1];
    if (kScaled) {
      a = a * is[0];
      b = b * is[1];
    }
    return from_f2_sr(a, b, r);
  }
};

template <>
__device__ __forceinline__ float2 Codec16<__half, __half2, true>::to_f2(unsigned w) {
  __half2 h;
  memcpy(&h, &w, 4);
  return __half22float2(h);
}
template <>
__device__ __forceinline__ unsigned Codec16<__half, __half2, true>::from_f2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  unsigned w;
  memcpy(&w, &h, 4);
  return w;
}
template <>
__device__ __forceinline__ unsigned Codec16<__half, __half2, true>::from_f2_sr(float a, float b,
                                                                               unsigned r) {
  unsigned w;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(w) : "f"(b), "f"(a), "r"(r));
  return w;
}
template <>
__device__ __forceinline__ float2 Codec16<__nv_bfloat16, __nv_bfloat162, false>::to_f2(unsigned w) {
  __nv_bfloat162 h;
  memcpy(&h, &w, 4);
  return __bfloat1622float2(h);
}
template <>
__device__ __forceinline__ unsigned Codec16<__nv_bfloat16, __nv_bfloat162, false>::from_f2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  unsigned w;
  memcpy(&w, &h, 4);
  return w;
}
template <>
__device__ __forceinline__ unsigned Codec16<__nv_bfloat16, __nv_bfloat162, false>::from_f2_sr(
    float a, float b, unsigned r) {
  unsigned w;
  asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(w) : "f"(b), "f"(a), "r"(r));
  return w;
}

template <>
struct Codec<__half> : Codec16<__half, __half2, true> {
  static __device__ __forceinline__ float dec(__half g, float s) { return __half2float(g) * s; }
  static __device__ __forceinline__ __half enc(float d, float inv_s) {
    return __float2half_rn(d * inv_s);
  }
  static __device__ __forceinline__ double dec64(__half g, double s) {
    return (double)__half2float(g) * s;
  }
};

template <>
struct Codec<__nv_bfloat16> : Codec16<__nv_bfloat16, __nv_bfloat162, false> {
  static __device__ __forceinline__ float dec(__nv_bfloat16 g, float s) {
    return __bfloat162float(g) * s;
  }
  static __device__ __forceinline__ __nv_bfloat16 enc(float d, float inv_s) {
    return __float2bfloat16_rn(d * inv_s);
  }
  static __device__ __forceinline__ double dec64(__nv_bfloat16 g, double s) {
    return (double)__bfloat162float(g) * s;
  }
};

// ---------------------------------------------------------------- layout
// Tiled, direction-major layout. Cells are grouped in tiles of 32 consecutive cell
// indices; a tile is one contiguous block of 98 x 32 elements holding, for each
// storage slot (direction) s = 0..6, the 14 fields of its 32 cells as four field
// groups: fields 0-3, 4-7, 8-11 as [lane][4] and fields 12-13 as [lane][2]. So a
// thread moves the 14 fields of one direction with three 4-wide and one 2-wide
// access (128/64-bit for FP32 storage), a warp's access covers contiguous bytes,
// and every address is a per-cell base plus a compile-time offset.
constexpr int kTile = 32;
constexpr int kSlotElems = kF * kTile;   // 448 elements per slot per tile
constexpr int kTileElems = kP * kTile;   // 3136 elements per tile

// Element offset of field group g (0..2: fields 4g..4g+3; 3: fields 12, 13) of slot s
// of lane `lane`, relative to the tile start.
__host__ __device__ constexpr int group_offset(int s, int g, int lane) {
  return s * kSlotElems + (g < 3 ? g * 4 * kTile + lane * 4 : 12 * kTile + lane * 2);
}

__host__ __device__ __forceinline__ long long tile_start(long long cell) {
  return (cell >> 5) * (long long)kTileElems;
}

__host__ __device__ __forceinline__ long long pop_index(long long cell, int k, int slot) {
  const int lane = (int)(cell & (kTile - 1));
  const int g = k < 12 ? k >> 2 : 3;
  const int j = k < 12 ? (k & 3) : k - 12;
  return tile_start(cell) + group_offset(slot, g, lane) + j;
}

// ---------------------------------------------------------------- AA index maps
// The state is one buffer of populations (k, slot, cell). After an even number of steps slot
// i of cell x holds f_i(x) (canonical). An even step reads its own slots and
// writes f*_i into slot opp(i) of the same cell; an odd step reads f_i(x) from
// slot opp(i) of cell x - e_i and writes f*_i into slot i of cell x + e_i. Every
// location is read and then written by the same thread, so the update is in place.
struct CellIndex {
  long long own;
  long long nb[kQ];  // nb[i] = cell x + e_i (periodic), nb[0] = own
  int x, plane;
};

__device__ __forceinline__ CellIndex make_index(const DomainConst& P, int x, int y, int z) {
  CellIndex c;
  const long long nx = P.nx, nxy = (long long)P.nx * P.ny;
  c.own = x + nx * ((long long)y + (long long)P.ny * z);
  c.x = x;
  c.plane = y + P.ny * z;
  c.nb[0] = c.own;
  c.nb[1] = c.own + (x + 1 < P.nx ? 1 : 1 - nx);
  c.nb[2] = c.own + (x > 0 ? -1 : nx - 1);
  c.nb[3] = c.own + (y + 1 < P.ny ? nx : nx - nxy);
  c.nb[4] = c.own + (y > 0 ? -nx : nxy - nx);
  c.nb[5] = c.own + (z + 1 < P.nz ? nxy : nxy - P.ncell);
  c.nb[6] = c.own + (z > 0 ? -nxy : P.ncell - nxy);
  return c;
}

// Esoteric twist (P.eso): the AA maps with slot s of logical cell x stored with cell
// x + e_x, x + e_y, x + e_z for s = 2, 4, 6 (the -x, -y, -z slots; periodic wrap), a
// fixed permutation of the buffer, so every result is the AA result bit for bit. Under
// it both parities touch the same cells: a step reads the incoming -x, -y, -z
// populations from the neighbours x + e_x, x + e_y, x + e_z and the rest from the own
// cell, and writes the outgoing +x, +y, +z populations into those neighbours and the
// rest into the own cell; the slots alternate as in the AA maps (even steps read slot
// i and write slot opp(i), odd steps read opp(i) and write i). Each location is still
// read and then written by one thread, so the update stays in place.
__device__ __forceinline__ bool eso_shifted(int i) { return i == 2 || i == 4 || i == 6; }

// Cell holding the incoming population of direction i at `parity` (its slot is i on
// even steps, opp(i) on odd ones).
__device__ __forceinline__ long long src_cell(const DomainConst& P, const CellIndex& c, int parity,
                                              int i) {
  if (P.eso) return eso_shifted(i) ? c.nb[i - 1] : c.own;
  return parity ? c.nb[opp(i)] : c.own;
}

// Cell receiving the outgoing population of direction i at `parity` (slot opp(i) on
// even steps, i on odd ones).
__device__ __forceinline__ long long dst_cell(const DomainConst& P, const CellIndex& c, int parity,
                                              int i) {
  if (P.eso) return (i == 1 || i == 3 || i == 5) ? c.nb[i] : c.own;
  return parity ? c.nb[i] : c.own;
}

// Cell and slot from which direction i of this cell is read at `parity`.
__device__ __forceinline__ long long read_pos(const DomainConst& P, const CellIndex& c, int parity,
                                              int k, int i) {
  long long cell = src_cell(P, c, parity, i);
  if (!LBM_CHECK(P, cell >= 0 && cell < P.ntile * kTile)) cell = 0;
  const int slot = parity ? opp(i) : i;
  return pop_index(cell, k, slot);
}

// Held x ends: the inward population of a boundary cell comes from the ghost
// layer, ghost[side][k][plane] (deviation, unscaled).
__device__ __forceinline__ bool from_ghost(const DomainConst& P, const CellIndex& c, int i) {
  return P.bc_x && ((i == 1 && c.x == 0) || (i == 2 && c.x == P.nx - 1));
}

__device__ __forceinline__ float ghost_value(const DomainConst& P, const float* ghost,
                                             const CellIndex& c, int k, int i) {
  const long long planes = (long long)P.ny * P.nz;
  const int side = (i == 1) ? 0 : 1;
  if (!LBM_CHECK(P, c.plane >= 0 && c.plane < planes)) return 0.0f;
  return ghost[((long long)side * kF + k) * planes + c.plane];
}

// Loads the 98 decoded deviations of this cell for a step of the given parity:
// per direction i the source cell and slot of the AA map (or the esoteric twist), then
// 4 + 4 + 4 + 2 fields.
template <int PARITY, bool HELD, typename S>
__device__ __forceinline__ void load_cell(const DomainConst& P, const S* __restrict__ pop,
                                          const float* __restrict__ ghost, const CellIndex& c,
                                          float (&d)[kF][kQ]) {
  using V4 = typename Codec<S>::V4;
  using V2 = typename Codec<S>::V2;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const long long cell = src_cell(P, c, PARITY, i);
    const int slot = PARITY ? opp(i) : i;
    if (!LBM_CHECK(P, cell >= 0 && cell < P.ntile * kTile)) {
#pragma unroll
      for (int k = 0; k < kF; ++k) d[k][i] = 0.0f;
      continue;
    }
    const S* base = pop + tile_start(cell);
    const int lane = (int)(cell & (kTile - 1));
    float v[kF];
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      const V4 w = *reinterpret_cast<const V4*>(base + group_offset(slot, g, lane));
      Codec<S>::dec4(w, P.scale + 4 * g, v + 4 * g);
    }
    const V2 w2 = *reinterpret_cast<const V2*>(base + group_offset(slot, 3, lane));
    Codec<S>::dec2(w2, P.scale + 12, v + 12);
#pragma unroll
    for (int k = 0; k < kF; ++k) d[k][i] = v[k];
    if (HELD && (i == 1 || i == 2) && from_ghost(P, c, i)) {
#pragma unroll
      for (int k = 0; k < kF; ++k) d[k][i] = ghost_value(P, ghost, c, k, i);
    }
  }
}

// Random words for stochastic rounding, one stream per cell and step: the seed mixes
// the cell's index with the bits of two of its post-collision populations (so the
// stream changes as the state evolves, and every kernel form draws the same words for
// the same cell) through a multiply-xorshift hash; the words are then a Weyl sequence
// (seed + k times the golden-ratio constant), one addition each. Every word is uniform
// because the seed is, so every rounding is unbiased; words of one cell differ by
// fixed offsets, which correlates roundings within a cell but biases none.
struct Dither {
  unsigned s;
  __device__ __forceinline__ Dither(long long cell, float a, float b) {
    unsigned x = (unsigned)cell * 0x9E3779B1u;
    x ^= __float_as_uint(a) * 0x85EBCA77u;
    x ^= __float_as_uint(b) * 0xC2B2AE3Du;
    x ^= x >> 15;
    x *= 0x2C1B3C6Du;
    x ^= x >> 13;
    x *= 0x297A2D39u;
    x ^= x >> 16;
    s = x;
  }
  __device__ __forceinline__ unsigned next() {
    s += 0x9E3779B9u;
    return s;
  }
};

// One direction's 14 fields into the 4 + 4 + 4 + 2 groups of slot `slot`, lane `lane`
// of the tile at `base`, rounded to nearest or (dz != nullptr) stochastically.
template <typename S>
__device__ __forceinline__ void store_dir(const DomainConst& P, S* base, int slot, int lane,
                                          const float (&d)[kF][kQ], int i, Dither* dz) {
  using V4 = typename Codec<S>::V4;
  using V2 = typename Codec<S>::V2;
  float v[kF];
#pragma unroll
  for (int k = 0; k < kF; ++k) v[k] = d[k][i];
  if constexpr (!std::is_same<S, float>::value) {
    if (dz) {
#pragma unroll
      for (int g = 0; g < 3; ++g) {
        const unsigned r0 = dz->next(), r1 = dz->next();
        *reinterpret_cast<V4*>(base + group_offset(slot, g, lane)) =
            Codec<S>::enc4_sr(v + 4 * g, P.inv_scale + 4 * g, r0, r1);
      }
      *reinterpret_cast<V2*>(base + group_offset(slot, 3, lane)) =
          Codec<S>::enc2_sr(v + 12, P.inv_scale + 12, dz->next());
      return;
    }
  }
#pragma unroll
  for (int g = 0; g < 3; ++g)
    *reinterpret_cast<V4*>(base + group_offset(slot, g, lane)) = Codec<S>::enc4(v + 4 * g, P.inv_scale + 4 * g);
  *reinterpret_cast<V2*>(base + group_offset(slot, 3, lane)) = Codec<S>::enc2(v + 12, P.inv_scale + 12);
}

// Stores the 98 post-collision deviations: direction i goes to the slot and cell of
// the AA map (own cell, slot opp(i) on even steps; cell x + e_i, slot i on odd steps),
// or of the esoteric twist.
// SR: stochastic rounding of 16-bit storage (a separate instantiation, so the
// round-to-nearest kernels carry none of its code).
template <int PARITY, typename S, bool SR = false>
__device__ __forceinline__ void store_cell(const DomainConst& P, S* __restrict__ pop,
                                           const CellIndex& c, const float (&d)[kF][kQ]) {
  [[maybe_unused]] Dither dz(0, 0.0f, 0.0f);
  if constexpr (SR) dz = Dither(c.own, d[0][0], d[4][0]);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const long long cell = dst_cell(P, c, PARITY, i);
    const int slot = PARITY ? i : opp(i);
    if (!LBM_CHECK(P, cell >= 0 && cell < P.ntile * kTile)) continue;
    store_dir<S>(P, pop + tile_start(cell), slot, (int)(cell & (kTile - 1)), d, i,
                 SR ? &dz : nullptr);
  }
}

// ---------------------------------------------------------------- rounding-exact arithmetic
// Every product, sum and fused multiply-add of the cell update is spelled out, so
// the compiler cannot contract or reorder them differently in different kernels:
// the single-domain kernels (both register budgets) and the batched kernel give
// bit-identical populations.
template <typename R> __device__ __forceinline__ R mul(R a, R b);
template <typename R> __device__ __forceinline__ R add(R a, R b);
template <typename R> __device__ __forceinline__ R sub(R a, R b);
template <typename R> __device__ __forceinline__ R fma_(R a, R b, R c);
template <> __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
template <> __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
template <> __device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
template <> __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
template <> __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
template <> __device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---------------------------------------------------------------- closure and flux
// Primitive state of one cell in precision R (float in the step, double in the
// initialisation and the moment outputs).
template <typename R>
struct Prim {
  R rho, inv_rho, m[3], u[3], E, p, T;
  R visc;     // mu_T / tau_R  (stress flux coefficient, Listing 1)
  R heat;     // kappa_T / tau_q (heat-flux flux coefficient, Listing 1)
  R mu_T;
  R tau[6];   // xx yy zz xy xz yz
  R q[3];
};

// Sutherland factor mu_T / mu = (1 + T_S) t^{3/2} / (t + T_S), t = T / T_ref.
template <typename R>
__device__ __forceinline__ R sutherland_ratio(R T, R inv_T_ref) {
  const R t = mul(T, inv_T_ref);
  return mul(mul((R)(1.0 + 0.4042), t), (R)sqrt(t)) / add(t, (R)0.4042);
}

// Sec. 2.1: u = (rho u)/rho, p = (gamma-1)(E - rho|u|^2/2), T = p/rho; Sutherland.
template <typename R>
__device__ __forceinline__ void closure(const R Q[kF], R gm1, R mu, R visc0, R heat0,
                                        R inv_T_ref, int sutherland, Prim<R>& s) {
  s.rho = Q[0];
  s.inv_rho = (R)1 / s.rho;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    s.m[a] = Q[1 + a];
    s.u[a] = mul(s.m[a], s.inv_rho);
  }
  s.E = Q[4];
  const R ke = mul((R)0.5, fma_(s.m[2], s.u[2], fma_(s.m[1], s.u[1], mul(s.m[0], s.u[0]))));
  s.p = mul(gm1, sub(s.E, ke));
  s.T = mul(s.p, s.inv_rho);
  const R r = sutherland ? sutherland_ratio<R>(s.T, inv_T_ref) : (R)1;
  s.mu_T = mul(mu, r);
  s.visc = mul(visc0, r);
  s.heat = mul(heat0, r);
#pragma unroll
  for (int j = 0; j < 6; ++j) s.tau[j] = Q[5 + j];
#pragma unroll
  for (int j = 0; j < 3; ++j) s.q[j] = Q[11 + j];
}

// Flux Phi_k (Eq. 2, Newtonian sign convention of tau) of field k, written out per
// component; Lambda_{bc,a} = delta_ab u_c + delta_ac u_b - 2/3 delta_bc u_a.
template <typename R>
__device__ __forceinline__ void field_flux(int k, const Prim<R>& s, R& fx, R& fy, R& fz) {
  const R ux = s.u[0], uy = s.u[1], uz = s.u[2];
  const R txx = s.tau[0], tyy = s.tau[1], tzz = s.tau[2];
  const R txy = s.tau[3], txz = s.tau[4], tyz = s.tau[5];
  const R v = s.visc;
  const R v23 = mul(v, (R)(2.0 / 3.0)), v43 = mul(v, (R)(4.0 / 3.0));
  switch (k) {
    case 0: fx = s.m[0]; fy = s.m[1]; fz = s.m[2]; break;
    case 1:
      fx = sub(fma_(s.m[0], ux, s.p), txx); fy = sub(mul(s.m[0], uy), txy); fz = sub(mul(s.m[0], uz), txz);
      break;
    case 2:
      fx = sub(mul(s.m[1], ux), txy); fy = sub(fma_(s.m[1], uy, s.p), tyy); fz = sub(mul(s.m[1], uz), tyz);
      break;
    case 3:
      fx = sub(mul(s.m[2], ux), txz); fy = sub(mul(s.m[2], uy), tyz); fz = sub(fma_(s.m[2], uz, s.p), tzz);
      break;
    case 4: {
      const R h = add(s.E, s.p);
      fx = add(sub(mul(h, ux), fma_(txz, uz, fma_(txy, uy, mul(txx, ux)))), s.q[0]);
      fy = add(sub(mul(h, uy), fma_(tyz, uz, fma_(tyy, uy, mul(txy, ux)))), s.q[1]);
      fz = add(sub(mul(h, uz), fma_(tzz, uz, fma_(tyz, uy, mul(txz, ux)))), s.q[2]);
      break;
    }
    case 5: fx = sub(mul(txx, ux), mul(v43, ux)); fy = fma_(v23, uy, mul(txx, uy)); fz = fma_(v23, uz, mul(txx, uz)); break;
    case 6: fx = fma_(v23, ux, mul(tyy, ux)); fy = sub(mul(tyy, uy), mul(v43, uy)); fz = fma_(v23, uz, mul(tyy, uz)); break;
    case 7: fx = fma_(v23, ux, mul(tzz, ux)); fy = fma_(v23, uy, mul(tzz, uy)); fz = sub(mul(tzz, uz), mul(v43, uz)); break;
    case 8: fx = sub(mul(txy, ux), mul(v, uy)); fy = sub(mul(txy, uy), mul(v, ux)); fz = mul(txy, uz); break;
    case 9: fx = sub(mul(txz, ux), mul(v, uz)); fy = mul(txz, uy); fz = sub(mul(txz, uz), mul(v, ux)); break;
    case 10: fx = mul(tyz, ux); fy = sub(mul(tyz, uy), mul(v, uz)); fz = sub(mul(tyz, uz), mul(v, uy)); break;
    case 11: fx = fma_(s.q[0], ux, mul(s.heat, s.T)); fy = mul(s.q[0], uy); fz = mul(s.q[0], uz); break;
    case 12: fx = mul(s.q[1], ux); fy = fma_(s.q[1], uy, mul(s.heat, s.T)); fz = mul(s.q[1], uz); break;
    default: fx = mul(s.q[2], ux); fy = mul(s.q[2], uy); fz = fma_(s.q[2], uz, mul(s.heat, s.T)); break;
  }
}

// ---------------------------------------------------------------- the cell update
struct SensorOut {
  float theta_dt;  // div u * dt (lattice units)
  float chi;
  float omega_h;
};

// The cell's own FP32 moments and closure as the step computes them, for the
// diagnostics (Sec. 3.2).
struct CellDiag {
  float D[5];      // zeroth-moment deviations of rho, rho u, E from the reference
  float rho, T, mu_T;
  float u[3], m[3];
  bool finite;     // all 14 zeroth moments finite
};

// Collides one cell in place on its decoded deviations d[k][i]. Returns the sum of
// the zeroth-moment deviations (a finiteness probe). With kSensor the sensor
// values are reported and the populations are left unchanged. With kDiag the
// moments and closure are also copied to *cd.
template <bool kSensor, bool kDiag = false>
__device__ __forceinline__ float collide_cell(const DomainConst& P, float (&d)[kF][kQ],
                                              SensorOut* so, CellDiag* cd = nullptr) {
  // Zeroth moments (Sec. 2.2: Q from the zeroth moment alone), i ascending.
  float D[kF];
#pragma unroll
  for (int k = 0; k < kF; ++k) {
    float s = d[k][0];
#pragma unroll
    for (int i = 1; i < kQ; ++i) s = add(s, d[k][i]);
    D[k] = s;
  }
  float Q[kF];
#pragma unroll
  for (int k = 0; k < kF; ++k) Q[k] = D[k];
  Q[0] = add(Q[0], P.rho_ref);
  Q[4] = add(Q[4], P.E_ref);
  Prim<float> s;
  closure<float>(Q, P.gm1, P.mu, P.visc0, P.heat0, P.inv_T_ref, P.sutherland, s);
  if constexpr (kDiag) {
    bool fin = true;
#pragma unroll
    for (int k = 0; k < kF; ++k) fin = fin && isfinite(D[k]);
#pragma unroll
    for (int k = 0; k < 5; ++k) cd->D[k] = D[k];
    cd->rho = s.rho;
    cd->T = s.T;
    cd->mu_T = s.mu_T;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cd->u[a] = s.u[a];
      cd->m[a] = s.m[a];
    }
    cd->finite = fin;
  }

  // Eq. 6: tau_base = 1/2 + 4 f_mu (mu_T/rho) dt/dx^2, omega = 1/tau_base.
  const float tau_b = fma_(mul(P.fmu_coef, s.mu_T), s.inv_rho, 0.5f);
  const float omega = 1.0f / tau_b;

  // Local dilatation from the cell's own non-equilibrium moments (pre-collision):
  //   fneq_{k,0} = d_{k,0} - D_k/4 = tau dt div(Phi_k)/4,
  //   m1_{rho,a} = c (d_{rho,+a} - d_{rho,-a}) - (rho u)_a
  //             = -tau dt (d_t (rho u)_a + (c^2/4) d_a rho),
  // so, in lattice units (theta dt) with tau = tau_base:
  //   theta dt = 4 omega / rho [fneq_{rho,0} - sum_a (u_a/c)(4 fneq_{rho u_a,0}/c
  //                                                   - (d_{rho,+a} - d_{rho,-a}) + m_a/c)].
  float acc = sub(d[0][0], mul(0.25f, D[0]));
  if (P.sensor_mode == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float fneq_m0 = sub(d[1 + a][0], mul(0.25f, D[1 + a]));
      const float g = fma_(s.m[a], P.inv_c, sub(mul(mul(4.0f, fneq_m0), P.inv_c),
                                                  sub(d[0][2 * a + 1], d[0][2 * a + 2])));
      acc = sub(acc, mul(mul(s.u[a], P.inv_c), g));
    }
  }
  const float theta_dt = mul(mul(mul(4.0f, omega), s.inv_rho), acc);
  // Eq. 3: s = max(0, -div u)/c_s with c_s = 1/2 in lattice units.
  const float smach = mul(2.0f, fmaxf(0.0f, -theta_dt));
  // Eq. 4 and Eq. 5.
  const float chi = (smach > P.J_min) ? fminf(mul(P.C_sigma, smach), 1.0f) : 0.0f;
  const float om = sub(omega, mul(chi, sub(omega, P.omega_min)));
  if constexpr (kSensor) {
    so->theta_dt = theta_dt;
    so->chi = chi;
    so->omega_h = om;
    return D[0];
  } else {
    // Collision, field by field: d* = d + omega_h (deq - d) + w_i dS_k with
    // deq_0 = D/4, deq_{+-a} = D/8 +- Phi_a / (2c).
#pragma unroll
    for (int k = 0; k < kF; ++k) {
      float fx, fy, fz;
      field_flux<float>(k, s, fx, fy, fz);
      const float e0 = mul(0.25f, D[k]), e1 = mul(0.125f, D[k]);
      const float ax = mul(P.half_inv_c, fx), ay = mul(P.half_inv_c, fy), az = mul(P.half_inv_c, fz);
      d[k][0] = fma_(om, sub(e0, d[k][0]), d[k][0]);
      d[k][1] = fma_(om, sub(add(e1, ax), d[k][1]), d[k][1]);
      d[k][2] = fma_(om, sub(sub(e1, ax), d[k][2]), d[k][2]);
      d[k][3] = fma_(om, sub(add(e1, ay), d[k][3]), d[k][3]);
      d[k][4] = fma_(om, sub(sub(e1, ay), d[k][4]), d[k][4]);
      d[k][5] = fma_(om, sub(add(e1, az), d[k][5]), d[k][5]);
      d[k][6] = fma_(om, sub(sub(e1, az), d[k][6]), d[k][6]);
      if (k >= 5) {  // the relaxation source of tau and q (zero for rho, rho u, E)
        const float dS = mul(k < 11 ? P.src_R : P.src_q, D[k]);
        const float s0 = mul(0.25f, dS), s1 = mul(0.125f, dS);
        d[k][0] = add(d[k][0], s0);
#pragma unroll
        for (int i = 1; i < kQ; ++i) d[k][i] = add(d[k][i], s1);
      }
    }
    float probe = 0.0f;
#pragma unroll
    for (int k = 0; k < kF; ++k) probe = add(probe, D[k]);
    return probe;
  }
}

}  // namespace lbm

// Device-side definitions shared by the CUDA translation units of liblbe:
// the D2Q9 velocity set, the per-instance descriptor and the population
// storage codecs.
//
// Population layout (one "arena" per instance and buffer): planes of
// ny rows x pitch elements, x fastest, pitch a multiple of 64 elements so
// that every row starts on a 128-byte boundary for every element size.  In a
// row, element XG + x holds cell x; the XG elements on either side are
// periodic ghost copies (cells nx-XG..nx-1 on the left, 0..XG-1 on the right)
// written with every store, so that a row segment [x0-XG, x0+w+XG) can be
// copied in one piece (TMA) for any strip start x0.
//   F64 : 27 planes, plane (k, i) at index k*9 + i (k = 0 f, 1 g, 2 hbar)
//   F32 : 9 pair planes holding (f_i, g_i) of a cell side by side (8 bytes
//         per cell), then 9 planes of hbar_i (so that a cell's f_i and g_i,
//         pulled from the same neighbour, load and store as one 8-byte word)
//   F16DEV / BF16DEV : 16-bit values (deviations, scaled): 8 pair planes
//               holding (f_i, g_i), i = 1..8, of a cell side by side
//               (4 bytes per cell), the f_0 plane (f0_off), 9 hbar planes
//               (h_off), then one FP32 plane holding g_0 (g0_off).
//   F16MIX : FP32 f with 16-bit (FP16) g and hbar deviations, the three
//               populations of a direction in one 8-byte word: 9 planes of
//               (f_i FP32, g_i FP16, hbar_i FP16) for i >= 1 and, for i = 0,
//               (f_0 FP32, hbar_0 FP16, the FP16 g_0 low part), then the FP32
//               g_0 plane (g0_off).  f carries the momentum, so u keeps the
//               precision of the FP32 form; 76 bytes per cell per buffer.
//   F32 and the 16-bit forms also keep the low part of g_0 (g_0 = hi + lo,
//   |lo| at most half an FP32 ulp of hi) as FP16 of lo * 2^24 in a plane at
//   byte offset g0lo_off, so that c = sum g_i (of which g_0 carries nearly
//   all) is held to about 1e-11 instead of the 6e-8 of one FP32 value.
// A buffer holds the post-collision populations of the previous step; the
// step kernel pulls P_i(x) = P*_i(x - xi_i) (with the wall rules) when it
// loads, so the two buffers ping-pong between steps.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace lbe {

// D2Q9: 0 (0,0), 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1), 5 (1,1), 6 (-1,1),
// 7 (-1,-1), 8 (1,-1).  constexpr so that unrolled loops fold them.
__host__ __device__ constexpr int EX(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int EY(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int OPP(int i) {
  return i == 0 ? 0 : i == 1 ? 3 : i == 2 ? 4 : i == 3 ? 1 : i == 4 ? 2
       : i == 5 ? 7 : i == 6 ? 8 : i == 7 ? 5 : 6;
}
// lattice weights (not listed in the paper; the standard D2Q9 set, c_s^2 = 1/3)
template <class C>
__host__ __device__ constexpr C WGT(int i) {
  return i == 0 ? C(4) / C(9) : (i < 5 ? C(1) / C(9) : C(1) / C(36));
}

enum Storage { ST_F64 = 0, ST_F32 = 1, ST_F16DEV = 2, ST_BF16DEV = 3, ST_F16MIX = 4 };

constexpr int XG = 4;  // periodic ghost columns on each side of a row

// Physical constants of one instance, derived on the host in double and
// kept in both precisions, so that the FP32 arithmetic never converts or
// computes in FP64 (a slow pipe on this GPU).
template <class C>
struct Phys {
  C rho, inv_rho, cv, rho_cv, inv_rho_cv;
  C rcs2, rcvcs2;          // rho c_s^2, rho c_v c_s^2
  C eta1, deta, lam1, dlam;
  C sigma0, sigmaT, Tref;
  C eps2, ea, beta2;       // eps^2, eps*alpha, 2 beta
  C omega_g, Gm;           // 1/tau_g, Gamma = M/(tau_g - 1/2)
  C Fbx, Fby;              // rho a
  C eta_n2;
  C hr0, hr1, dh;          // T_r(y) = hr0 + hr1 y; dh = rho c_v hr1
  C inv_s[3];              // 16-bit codec: 1/s_k (1 for the other storages)
  C drho;                  // rho2 - rho1 (0: uniform density; FP64 storage only)
  C ax, ay;                // body acceleration (the force rho(c) a)
  // variants (0: off): harmonic property law (with the phase-1 values and
  // the four reciprocals), wall temperature at the link's wall crossing,
  // wetting flux coefficient cos(theta) sqrt(2 beta) / eps
  C harm, eta2, lam2, ie1, ie2, il1, il2;
  C wmid;
  C kw;
};

// eta(c) or lambda(c) between the phase values a (c = 0) and b (c = 1):
// linear (a + c (b - a), d = b - a) or, with P.harm, harmonic
// 1/((1 - c)/a + c/b) (ia, ib: the reciprocals, used by the FP32 forms).
template <class C>
__device__ __forceinline__ C prop_at(const Phys<C>& P, C a, C d, C b, C ia, C ib, C c) {
  if (P.harm != C(0)) {
    if constexpr (sizeof(C) == 8)
      return C(1) / ((C(1) - c) / a + c / b);
    else
      return C(1) / ((C(1) - c) * ia + c * ib);
  }
  return a + c * d;
}

// Wetting walls: ghost row -1-j (or ny+j) of c from its mirror cell's c, the
// mirror value plus (2j+1) times the wall flux (sqrt(2 beta)/eps) cos(theta)
// c (1 - c) (Young's law through a cubic wall energy).
template <class C>
__device__ __forceinline__ C wet_ghost(const Phys<C>& P, C cm, int j) {
  return P.kw != C(0) ? cm + C(2 * j + 1) * P.kw * cm * (C(1) - cm) : cm;
}

// The density of a cell, linear in c: rho(c) = rho1 + c (rho2 - rho1).
template <class C>
__device__ __forceinline__ C rho_at(const Phys<C>& P, C c) {
  return P.drho != C(0) ? P.rho + c * P.drho : P.rho;
}

// Per-instance descriptor, built on the host, read by the kernels.
struct InstDev {
  int32_t nx, ny, pitch, tiles_x;
  int32_t tiles_y, storage;
  int64_t tile_begin;   // first global tile / work-item index of this instance
  uint64_t plane_bytes; // bytes between consecutive planes
  uint64_t g0_off;      // byte offset of the FP32 g_0 plane (16-bit forms)
  uint64_t g0lo_off;    // byte offset of the FP16 plane of the g_0 low part (16/32-bit)
  uint64_t pair_bytes;  // 16/32-bit: bytes of one (f_i, g_i) pair plane
  uint64_t h_off;       // 16/32-bit: byte offset of the first hbar plane
  uint64_t f0_off;      // 16-bit: byte offset of the f_0 plane
  char* buf[2];         // population arenas (ping-pong)
  const double* Tbot;   // [nx] wall temperature at y = -1/2
  const double* Ttop;   // [nx] wall temperature at y = ny - 1/2
  // deviation forms: T_w - T_r at the first row (bottom), last row (top),
  // and at the wall positions y = -1/2 (bottom) and y = ny - 1/2 (top)
  const float* wdev[4];
  Phys<double> pd;
  Phys<float> pf;
  float s[3];           // 16-bit codec scales s_k
  double hr0, hr1;      // T_r(y) = hr0 + hr1 y (double, for state conversion)
  uint32_t salt;        // the instance's index in its handle (random bits)
  double* pcorr;        // varying density: p of Eq. 13 with its correction, [ny][nx]
  double* uvel;         // dissipation term: u of every cell, [2][ny][nx] (FP64)
};

template <class C>
__device__ __forceinline__ const Phys<C>& phys(const InstDev& I);
template <>
__device__ __forceinline__ const Phys<double>& phys<double>(const InstDev& I) { return I.pd; }
template <>
__device__ __forceinline__ const Phys<float>& phys<float>(const InstDev& I) { return I.pf; }

// ------------------------------------------------------- stochastic rounding
// The 16-bit forms round the values they store stochastically: to one of the
// two neighbouring 16-bit values, with probabilities that make the expected
// stored value the exact one.  Rounded to nearest instead, a cell of a flow
// near steady state makes the same rounding error step after step, so the
// errors add up over the flow's relaxation time instead of averaging out.
// Random bits: a counter-based hash per cell and step (the finaliser of
// MurmurHash3 over the step counter, the instance and the cell), then, for
// population v = 9 k + i, term v of a linear congruential sequence started at
// that hash, reached in one multiply-add from closed-form constants, so that
// every kernel draws the same bits for a given value.
__host__ __device__ constexpr uint32_t mix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
// LCG s -> LCG_A s + LCG_C (Numerical Recipes' constants); term v from s:
// a_v s + c_v with a_v = LCG_A^v and c_v = LCG_C (1 + LCG_A + ... + LCG_A^(v-1)),
// tabulated at compile time for v = 0..27 (read with constant indices)
constexpr uint32_t LCG_A = 1664525u, LCG_C = 1013904223u;
struct LcgTable {
  uint32_t a[28], c[28];
};
constexpr LcgTable make_lcg_table() {
  LcgTable t{};
  t.a[0] = 1u;
  t.c[0] = 0u;
  for (int v = 1; v < 28; v++) {
    t.a[v] = LCG_A * t.a[v - 1];
    t.c[v] = LCG_A * t.c[v - 1] + LCG_C;
  }
  return t;
}
static __constant__ LcgTable LCG_TAB = make_lcg_table();
// hash of a step and an instance (uniform over a work item)
__device__ __forceinline__ uint32_t sr_step_key(uint32_t step, uint32_t salt) {
  return mix32(step * 0x9E3779B9u ^ mix32(salt + 0x632BE5ABu));
}
// the cell's hash
__device__ __forceinline__ uint32_t sr_cell(uint32_t step_key, uint32_t cell) {
  return mix32(step_key ^ (cell * 0x85EBCA77u));
}
// 32 random bits for population (k, i) of a cell (k and i fold to constants
// in the unrolled loops)
__device__ __forceinline__ uint32_t sr_bits(int k, int i, uint32_t cell_hash) {
  return LCG_TAB.a[9 * k + i + 1] * cell_hash + LCG_TAB.c[9 * k + i + 1];
}
// x with MB-bit target mantissa (10: FP16, 7: BF16) plus a random integer
// below the target's last mantissa bit, added to x's FP32 bit pattern (that
// is, to its magnitude): truncating the result toward zero to the target
// format rounds x up or down with probabilities proportional to the
// distances, wherever the target value is normal (for FP16 below 2^-14,
// where fewer mantissa bits remain, the rounding is partly toward zero).
template <int MB>
__device__ __forceinline__ float sr_dither(float x, uint32_t r) {
  return __uint_as_float(__float_as_uint(x) + (r >> (9 + MB)));
}
// (a, b) to a packed FP16 / BF16 pair (a in the low half), stochastically;
// the two dithers take bits 19-31 and 6-18 (FP16) or 16-31 and 0-15 (BF16)
// of one random word
__device__ __forceinline__ uint32_t sr_pack_half2(float a, float b, uint32_t r) {
  uint32_t out;
  asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(out) : "f"(sr_dither<10>(b, r << 13)),
      "f"(sr_dither<10>(a, r)));
  return out;
}
__device__ __forceinline__ uint32_t sr_pack_bf162(float a, float b, uint32_t r) {
  uint32_t out;
  asm("cvt.rz.bf16x2.f32 %0, %1, %2;" : "=r"(out) : "f"(sr_dither<7>(b, r << 16)),
      "f"(sr_dither<7>(a, r)));
  return out;
}
__device__ __forceinline__ __half sr_half(float x, uint32_t r) {
  return __float2half_rz(sr_dither<10>(x, r));
}
__device__ __forceinline__ __nv_bfloat16 sr_bf16(float x, uint32_t r) {
  return __float2bfloat16_rz(sr_dither<7>(x, r));
}

// ------------------------------------------------------------ storage codecs
// ld / st take (k, i) as template-folded constants through the unrolled loops.
// FP64 stores the populations as they are (parity mode).  The other forms
// store hbar as the deviation hbar_i - w_i rho c_v T_r(y) from the linear
// conduction profile T_r of the row the value is stored in; the kernels work
// with that deviation directly (the codec does not add the reference back).

struct StF64 {
  using C = double;
  static constexpr int kind = ST_F64;
  static constexpr bool SR = false;  // stores round to nearest
  __device__ static __forceinline__ C sr_value(const InstDev&, int, int, C v, uint32_t) {
    return v;
  }
  __device__ static __forceinline__ C ld(const InstDev& I, const Phys<C>&, const char* b, int k,
                                         int i, size_t idx) {
    return __ldg(reinterpret_cast<const double*>(b + (size_t)(k * 9 + i) * I.plane_bytes) + idx);
  }
  __device__ static __forceinline__ void st(const InstDev& I, char* b, int k, int i, size_t idx,
                                            C v) {
    reinterpret_cast<double*>(b + (size_t)(k * 9 + i) * I.plane_bytes)[idx] = v;
  }
};

struct StF32 {
  using C = float;
  static constexpr int kind = ST_F32;
  static constexpr bool SR = false;
  __device__ static __forceinline__ C sr_value(const InstDev&, int, int, C v, uint32_t) {
    return v;
  }
  __device__ static __forceinline__ C ld(const InstDev& I, const Phys<C>&, const char* b, int k,
                                         int i, size_t idx) {
    if (k < 2)
      return __ldg(reinterpret_cast<const float*>(b + (size_t)i * I.pair_bytes) + 2 * idx + k);
    return __ldg(reinterpret_cast<const float*>(b + I.h_off + (size_t)i * I.plane_bytes) + idx);
  }
  __device__ static __forceinline__ void st(const InstDev& I, char* b, int k, int i, size_t idx,
                                            C v) {
    if (k < 2)
      reinterpret_cast<float*>(b + (size_t)i * I.pair_bytes)[2 * idx + k] = v;
    else
      reinterpret_cast<float*>(b + I.h_off + (size_t)i * I.plane_bytes)[idx] = v;
  }
  // f_i and g_i of one cell as one 8-byte store
  __device__ static __forceinline__ void st_fg(const InstDev& I, char* b, int i, size_t idx,
                                               float fv, float gv) {
    reinterpret_cast<float2*>(b + (size_t)i * I.pair_bytes)[idx] = make_float2(fv, gv);
  }
};

// 16-bit forms: q = s_k v in fp16 / bf16 (v the value or, for hbar, the
// deviation); g_0 in FP32 (plus its low part, below).
template <class E, int KIND>
struct StDev {
  using C = float;
  static constexpr int kind = KIND;
  static constexpr bool SR = true;  // the 16-bit values round stochastically
  static constexpr bool BF = KIND == ST_BF16DEV;
  __device__ static __forceinline__ float cvt(__half q) { return __half2float(q); }
  __device__ static __forceinline__ float cvt(__nv_bfloat16 q) { return __bfloat162float(q); }
  // two adjacent 16-bit values (4-byte aligned) to FP32
  __device__ static __forceinline__ float2 cvt2(const __half* p) {
    return __half22float2(*reinterpret_cast<const __half2*>(p));
  }
  __device__ static __forceinline__ float2 cvt2(const __nv_bfloat16* p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
  }
  __device__ static __forceinline__ void put(__half* p, float v) { *p = __float2half_rn(v); }
  __device__ static __forceinline__ void put(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
  __device__ static __forceinline__ void put2(__half* p, float a, float b) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
  }
  __device__ static __forceinline__ void put2(__nv_bfloat16* p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
  }
  // element (k, i) of cell idx: its address in the pair / f_0 / hbar planes
  __device__ static __forceinline__ const E* at(const InstDev& I, const char* b, int k, int i,
                                                size_t idx) {
    if (k == 2) return reinterpret_cast<const E*>(b + I.h_off + (size_t)i * I.plane_bytes) + idx;
    if (i == 0) return reinterpret_cast<const E*>(b + I.f0_off) + idx;  // f_0
    return reinterpret_cast<const E*>(b + (size_t)(i - 1) * I.pair_bytes) + 2 * idx + k;
  }
  __device__ static __forceinline__ C ld(const InstDev& I, const Phys<C>& P, const char* b, int k,
                                         int i, size_t idx) {
    if (k == 1 && i == 0)
      return __ldg(reinterpret_cast<const float*>(b + I.g0_off) + idx);
    return cvt(*at(I, b, k, i, idx)) * P.inv_s[k];
  }
  __device__ static __forceinline__ void st(const InstDev& I, char* b, int k, int i, size_t idx,
                                            C v) {
    if (k == 1 && i == 0) {
      reinterpret_cast<float*>(b + I.g0_off)[idx] = v;
      return;
    }
    put(const_cast<E*>(at(I, b, k, i, idx)), v * I.s[k]);
  }
  // f_i and g_i (i >= 1) of one cell as one 4-byte store
  __device__ static __forceinline__ void st_fg(const InstDev& I, char* b, int i, size_t idx,
                                               float fv, float gv) {
    put2(reinterpret_cast<E*>(b + (size_t)(i - 1) * I.pair_bytes) + 2 * idx, fv * I.s[0],
         gv * I.s[1]);
  }
  // the same, stochastically rounded with the random word r; returns the
  // stored g_i scaled by s_1 (exact)
  __device__ static __forceinline__ float st_fg_sr(const InstDev& I, char* b, int i, size_t idx,
                                                   float fv, float gv, uint32_t r) {
    const uint32_t q = BF ? sr_pack_bf162(fv * I.s[0], gv * I.s[1], r)
                          : sr_pack_half2(fv * I.s[0], gv * I.s[1], r);
    *reinterpret_cast<uint32_t*>(reinterpret_cast<E*>(b + (size_t)(i - 1) * I.pair_bytes) +
                                 2 * idx) = q;
    if constexpr (BF)
      return __uint_as_float(q & 0xffff0000u);
    else
      return __half2float(__ushort_as_half((unsigned short)(q >> 16)));
  }
  // one 16-bit value (not g_0), stochastically rounded
  __device__ static __forceinline__ void st_sr(const InstDev& I, char* b, int k, int i, size_t idx,
                                               C v, uint32_t r) {
    E* p = const_cast<E*>(at(I, b, k, i, idx));
    if constexpr (BF)
      *p = sr_bf16(v * I.s[k], r);
    else
      *p = sr_half(v * I.s[k], r);
  }
  // the dither word of value (k, i) of a cell with hash hc: one word per
  // (f_i, g_i) pair (f from its top bits, g from the word shifted left, as
  // sr_pack_* take them), one per f_0 and per hbar_i
  __device__ static __forceinline__ uint32_t sr_word(int k, int i, uint32_t hc) {
    if (k == 1) return sr_bits(0, i, hc) << (BF ? 16 : 13);
    return sr_bits(k, i, hc);
  }
  // v rounded stochastically to a value the store then represents exactly
  // (g_0, kept in FP32, as it is)
  __device__ static __forceinline__ C sr_value(const InstDev& I, int k, int i, C v, uint32_t hc) {
    if (k == 1 && i == 0) return v;
    const uint32_t r = sr_word(k, i, hc);
    if constexpr (BF)
      return __bfloat162float(sr_bf16(v * I.s[k], r)) * I.pf.inv_s[k];
    else
      return __half2float(sr_half(v * I.s[k], r)) * I.pf.inv_s[k];
  }
};

// F16MIX: direction i of cell idx is the 8-byte word at pair plane i
// (pair_bytes apart): bytes 0-3 f_i (FP32); bytes 4-5 g_i (i >= 1) or
// hbar_0 (i = 0); bytes 6-7 hbar_i (i >= 1) or the g_0 low part (i = 0), as
// FP16 of s_k times the value.  g_0 itself is the FP32 plane at g0_off.
struct StMix {
  using C = float;
  static constexpr int kind = ST_F16MIX;
  static constexpr bool SR = true;  // the FP16 g_i and hbar_i round stochastically
  template <class B>  // const char or char
  __device__ static __forceinline__ B* word(const InstDev& I, B* b, int i, size_t idx) {
    return b + (size_t)i * I.pair_bytes + 8 * idx;
  }
  // byte offset of (k, i) in its word (k >= 1)
  __host__ __device__ static constexpr int half_at(int k, int i) {
    return (k == 1 || i == 0) ? 4 : 6;
  }
  __device__ static __forceinline__ C ld(const InstDev& I, const Phys<C>& P, const char* b, int k,
                                         int i, size_t idx) {
    if (k == 0) return __ldg(reinterpret_cast<const float*>(word(I, b, i, idx)));
    if (k == 1 && i == 0) return __ldg(reinterpret_cast<const float*>(b + I.g0_off) + idx);
    return __half2float(*reinterpret_cast<const __half*>(word(I, b, i, idx) + half_at(k, i))) *
           P.inv_s[k];
  }
  __device__ static __forceinline__ void st(const InstDev& I, char* b, int k, int i, size_t idx,
                                            C v) {
    char* w = word(I, b, i, idx);
    if (k == 0) {
      *reinterpret_cast<float*>(w) = v;
    } else if (k == 1 && i == 0) {
      reinterpret_cast<float*>(b + I.g0_off)[idx] = v;
    } else {
      *reinterpret_cast<__half*>(w + half_at(k, i)) = __float2half_rn(v * I.s[k]);
    }
  }
  // the dither word of value (k, i) of a cell with hash hc: one word per
  // (g_i, hbar_i) pair of a direction word (g from its top bits, hbar from
  // the word shifted left, as sr_pack_half2 takes them), one for hbar_0
  __device__ static __forceinline__ uint32_t sr_word(int k, int i, uint32_t hc) {
    if (i == 0) return sr_bits(2, 0, hc);
    return k == 1 ? sr_bits(1, i, hc) : sr_bits(1, i, hc) << 13;
  }
  // v rounded stochastically to a value the store then represents exactly
  // (the FP32 f_i and g_0 as they are)
  __device__ static __forceinline__ C sr_value(const InstDev& I, int k, int i, C v, uint32_t hc) {
    if (k == 0 || (k == 1 && i == 0)) return v;
    return __half2float(sr_half(v * I.s[k], sr_word(k, i, hc))) * I.pf.inv_s[k];
  }
};

// The low part of g_0 (16/32-bit storages).
constexpr float G0LO_SCALE = 16777216.0f;  // 2^24
constexpr float G0LO_INV = 1.0f / 16777216.0f;
template <class S>
__device__ __forceinline__ float ld_g0lo(const InstDev& I, const char* b, size_t idx) {
  if constexpr (S::kind == ST_F16MIX)
    return __half2float(*reinterpret_cast<const __half*>(b + 8 * idx + 6)) * G0LO_INV;
  else
    return __half2float(reinterpret_cast<const __half*>(b + I.g0lo_off)[idx]) * G0LO_INV;
}
template <class S>
__device__ __forceinline__ void st_g0lo(const InstDev& I, char* b, size_t idx, float lo) {
  if constexpr (S::kind == ST_F16MIX)
    *reinterpret_cast<__half*>(b + 8 * idx + 6) = __float2half_rn(lo * G0LO_SCALE);
  else
    reinterpret_cast<__half*>(b + I.g0lo_off)[idx] = __float2half_rn(lo * G0LO_SCALE);
}

using StF16 = StDev<__half, ST_F16DEV>;
using StBF16 = StDev<__nv_bfloat16, ST_BF16DEV>;

}  // namespace lbe

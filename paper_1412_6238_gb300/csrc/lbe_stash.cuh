// The fused step as a column-strip marching kernel with a stash of pulled
// populations (FP32 and 16-bit storages).
//
// A work item is a strip of NC output columns and a segment of rows [ya, yb)
// of one instance: a CTA of NC threads marches up the rows, thread t owning
// column x0 + t.  The stencils also need the moments of the two halo columns
// on each side (c at x0 - 2 .. x0 + NC + 1, p and T at x0 - 1 .. x0 + NC):
// four lanes of the last warp form those as extra work, so that no thread
// of the CTA is spent on a column it does not collide (NC a power of two:
// the strips tile power-of-two grids exactly).  Instead of staging whole
// source rows (as a TMA tiled row ring would, 7 rows for the pull and the
// stencils), the CTA stages, for
// each moment row m, what its cells pull: for each population row of the
// layout (FP32: the 9 (f_i, g_i) pair rows, the 9 hbar_i rows and the g_0 low
// part), the elements of source row m - xi_iy over the strip's columns and
// the pulls' reach (or, at a wall, the reversed population of row m itself),
// one bulk copy (cp.async.bulk, 16-byte aligned) per row, all completing on
// the slot's mbarrier.  A row's values stay in the stash from the time its
// moments are formed until it collides three iterations later: a 4-row
// stash (58 KB in FP32) instead of a 7-row ring, so that three CTAs fit on
// an SM.  A window that crosses the periodic edge is contiguous because
// every stored row repeats its first and last XG cells beyond its ends (the
// ghost columns): with OWN the kernel stores them with the cells' values,
// otherwise ghost_kernel refreshes them after the step.
//
// Iteration i (from ya - 4 to yb):
//   barrier; 1. collide row i-1 (S2-S9 of lbe_cell.cuh) from its stash slot
//      and the moment rings, and store its 27 values; every thread arrives
//      on the slot's empty mbarrier right after its pulls;
//   2. one elected lane of warp 0 waits for that empty barrier and issues
//      the copies of row i+3 into the slot (as early as possible: the
//      copies then have the rest of this iteration and the next collision
//      to land), while the other warps go on;
//   3. wait for the copies of row i+2 and form its moments c, p, T (S1) into
//      the rings (own columns, then the four halo columns); rows below the
//      bottom wall use the pulled values of their mirror row, rows above the
//      top wall copy the mirror rows in the rings;
//   barrier; 4. unit normal of row i+1 (S2).
// Every population is read from HBM once per step.  Every mbarrier wait is
// bounded (poll_lim polls): on the first time-out the CTA sets *err, issues
// no further copy, waits (bounded again) for the copies it has in flight and
// returns.  A drain wait that also runs out means a copy that was issued has
// not landed within the whole limit; the CTA returns all the same (it cannot
// wait forever), and the host then treats the handle's state as lost.
// withhold >= 0 is a test hook: the copies of source row `withhold` are not
// issued (their barrier still expects the bytes), so that the waits for that
// row run out with nothing in flight.
#pragma once

#include "lbe_tile.cuh"

namespace lbe {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Bounded wait for the phase with the given parity (at most `limit` polls);
// false on time-out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// One-dimensional bulk copy global -> shared (16-byte aligned addresses, a
// multiple of 16 bytes), completing on an mbarrier.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Threads (= output columns) of a strip CTA.
constexpr int STASH_NC = 128;

// Stash layout of one row for a storage form: population (k, i) has a row of
// EW = NC + 8 elements at byte offset off(k, i) of the slot, from storage
// element x0 (x0 a multiple of NC: 16-byte aligned in every form), covering
// the CTA's columns, the halo columns and the pulls' reach (columns x0 - 3
// .. x0 + NC + 2 are elements x0 + 1 .. x0 + NC + 6).  Every form adds the
// FP16 row of the g_0 low part at byte LO.
template <class S>
struct StashFmt;
// FP32: 9 rows of (f_i, g_i) pairs (EW cells x 8 bytes), 9 rows of hbar_i
// (EW x 4 bytes); off(k, i) is the byte offset of the row holding (k, i).
template <>
struct StashFmt<StF32> {
  using E = float;
  static constexpr int EW = STASH_NC + 8;             // cells per row
  static constexpr int PROW = EW * 8;                 // pair row bytes
  static constexpr int ROW = EW * 4;                  // hbar row bytes
  static constexpr int HOFF = 9 * PROW;
  static constexpr int LO = HOFF + 9 * ROW;           // the g_0 low-part row
  static constexpr int LOB = (STASH_NC + 8) * 2;      // its bytes
  static constexpr int SLOT_RAW = LO + LOB;           // bytes of one row
  static constexpr int MINB = 3;                      // resident CTAs per SM
  __host__ __device__ static constexpr int off(int k, int i) {
    return k < 2 ? i * PROW : HOFF + i * ROW;
  }
  static_assert(PROW % 16 == 0 && ROW % 16 == 0 && LO % 16 == 0 && LOB % 16 == 0,
                "bulk copies: 16-byte sizes and offsets");
};
// 16-bit: 8 rows of (f_i, g_i) pairs, i = 1..8, the f_0 row and 9 hbar rows
// (4 and 2 bytes per cell), the FP32 g_0 row.
template <class E16>
struct StashFmt16 {
  using E = E16;
  static constexpr int EW = STASH_NC + 8;
  static constexpr int PROW = EW * 4;
  static constexpr int ROW = EW * 2;
  static constexpr int F0 = 8 * PROW;
  static constexpr int HOFF = F0 + ROW;
  static constexpr int G0 = HOFF + 9 * ROW;
  static constexpr int G0B = EW * 4;
  static constexpr int LO = G0 + G0B;
  static constexpr int LOB = ROW;
  static constexpr int SLOT_RAW = LO + LOB;
  static constexpr int MINB = 4;
  __host__ __device__ static constexpr int off(int k, int i) {
    return k == 2 ? HOFF + i * ROW : (i == 0 ? (k == 0 ? F0 : G0) : (i - 1) * PROW);
  }
  static_assert(PROW % 16 == 0 && ROW % 16 == 0 && G0 % 16 == 0 && G0B % 16 == 0 &&
                    LO % 16 == 0,
                "bulk copies: 16-byte sizes and offsets");
};
// F16MIX: 9 rows of the 8-byte direction words (f_i FP32, two FP16 values)
// and the FP32 g_0 row; the g_0 low part travels in the words of row 0.
template <>
struct StashFmt<StMix> {
  using E = float;
  static constexpr int EW = STASH_NC + 8;
  static constexpr int WROW = EW * 8;  // word row bytes
  static constexpr int G0 = 9 * WROW;
  static constexpr int G0B = EW * 4;
  static constexpr int SLOT_RAW = G0 + G0B;
  static constexpr int MINB = 4;
  static_assert(WROW % 16 == 0 && G0B % 16 == 0, "bulk copies: 16-byte sizes and offsets");
};
template <>
struct StashFmt<StF16> : StashFmt16<__half> {};
template <>
struct StashFmt<StBF16> : StashFmt16<__nv_bfloat16> {};

template <class S, int NC>
struct StashCfg {
  using Fmt = StashFmt<S>;
  static_assert(NC == STASH_NC, "the stash formats are laid out for STASH_NC columns");
  static_assert(Fmt::SLOT_RAW % 16 == 0, "16-byte slots");
  static constexpr int NCO = NC;              // output columns
  static constexpr int NW = NC / 32;          // warps
  static constexpr int SR = 4;                // stash rows
  static constexpr int SLOT = Fmt::SLOT_RAW;  // bytes of one row
  static constexpr int TX = Fmt::SLOT_RAW;    // bytes copied per row
  static constexpr int CR = 5, PR = 5, NR = 4;  // moment / normal ring rows
  static_assert(CR == PR, "c, p and T rings share their row index");
  // ring row widths: c (and its low part) at x0 - 2 .. x0 + NC + 1, p, T
  // and the unit normal at x0 - 1 .. x0 + NC
  static constexpr int CW = NC + 4, QW = NC + 2;
  static constexpr int STASH = SR * SLOT;
  // FP32 rings of c, p, T, n_x, n_y and the FP16 ring of the c low part
  static constexpr int RINGS = (CR * CW + 2 * PR * QW + 2 * NR * QW) * 4 + CR * CW * 2;
  static_assert(RINGS % 8 == 0, "the slot barriers follow the rings");
  // a "full" (copies landed) and an "empty" (every thread done with the
  // slot) mbarrier per stash slot
  static constexpr int SMEM = STASH + RINGS + 2 * SR * 8;
  // resident CTAs per SM the kernel is compiled for (registers)
  static constexpr int MINB = Fmt::MINB;
  static_assert(NC % 32 == 0, "whole warps");
};

// The 9 pulled populations of lattice K at row y from a stash slot
// (thread t reads element t + 2 - xi_ix of population (K, i), or t + 2 where
// the wall substitution copied the reversed population of the cell itself),
// with the rules of pull9 (lbe_tile.cuh): anti-bounce-back for hbar at the
// walls, and the deviation offsets of hbar between rows.
template <class S>
__device__ __forceinline__ float stash_val(const char* slot, int k, int i, int col,
                                           const Phys<float>& P) {
  using Fmt = StashFmt<S>;
  if constexpr (sizeof(typename Fmt::E) == 4) {
    if (k < 2) return reinterpret_cast<const float*>(slot + Fmt::off(k, i))[2 * col + k];
    return reinterpret_cast<const float*>(slot + Fmt::off(k, i))[col];
  } else {
    if (k == 1 && i == 0) return reinterpret_cast<const float*>(slot + Fmt::off(1, 0))[col];
    const typename Fmt::E* r = reinterpret_cast<const typename Fmt::E*>(slot + Fmt::off(k, i));
    return S::cvt(k < 2 && i > 0 ? r[2 * col + k] : r[col]) * P.inv_s[k];
  }
}

// The 9 pulled populations of lattice K at row y from a stash slot.
// c0 is the element of the thread's own column in a population row (c0g in the
// FP32 g_0 row of the 16-bit forms); the pull reads c0 - xi_ix, or c0 where
// the wall substitution copied the reversed population of the cell itself.
// Rules of pull9 (lbe_tile.cuh): anti-bounce-back for hbar at the walls, and
// the deviation offsets of hbar between rows.
// RAW: in an interior row, the hbar deviations as stored, relative to their
// source rows' T_r, without the offsets +-w_i dh to this row's T_r: they
// cancel exactly in the moment, and collide() applies them through its
// source term.
// The wall temperature of the anti-bounce-back link of population i at
// column xw (Tw: the wall temperature at xw): with P.wmid, where the link
// crosses the wall, x - xi_ix/2, between the two columns.
template <class S>
__device__ __forceinline__ float link_T(const InstDev& I, const Phys<float>& P, int xw, int i,
                                        int which, float Tw) {
  if (P.wmid == 0.f || EX(i) == 0) return Tw;
  int xs = xw - EX(i);
  xs = xs < 0 ? xs + I.nx : (xs >= I.nx ? xs - I.nx : xs);
  return 0.5f * (Tw + wall_T<S>(I, xs, which));
}

template <class S, int K, bool RAW = false>
__device__ __forceinline__ void wstash_pull(const InstDev& I, const Phys<float>& P,
                                            const char* slot, int c0, int c0g, int y, int xw,
                                            float out[9]) {
  constexpr bool DEV = (K == 2) && dev_h<S>();
  const bool wb = (y == 0), wt = (y == I.ny - 1);
  auto col = [&](int i, bool shift) {
    const int base = (K == 1 && i == 0) ? c0g : c0;
    return shift ? base - EX(i) : base;
  };
  if (!wb && !wt) {
    // interior row: constant offsets
#pragma unroll
    for (int i = 0; i < 9; i++) {
      float v = stash_val<S>(slot, K, i, col(i, true), P);
      if (DEV && !RAW && EY(i) == 1) v -= WGT<float>(i) * P.dh;
      if (DEV && !RAW && EY(i) == -1) v += WGT<float>(i) * P.dh;
      out[i] = v;
    }
    return;
  }
  float Tw = 0.f;
  if (K == 2) Tw = wall_T<S>(I, xw, wb ? 0 : 1);
  const float dh = DEV ? P.dh : 0.f;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    const bool wall = (EY(i) == 1 && wb) || (EY(i) == -1 && wt);
    float v = wall ? stash_val<S>(slot, K, i, col(i, false), P)
                   : stash_val<S>(slot, K, i, col(i, true), P);
    if (K == 2) {
      if (wall) {
        v = -v + 2.f * WGT<float>(i) * P.rho * P.cv * link_T<S>(I, P, xw, i, wb ? 0 : 1, Tw);
      } else if (DEV && EY(i) == 1) {
        v -= WGT<float>(i) * dh;
      } else if (DEV && EY(i) == -1) {
        v += WGT<float>(i) * dh;
      }
    }
    out[i] = v;
  }
}

// FP32 pair layout: f_i and g_i of a pulled cell with one 8-byte load each
// (f and g follow the same bounce-back rule at the walls).
__device__ __forceinline__ void wstash_pull_fg(const InstDev& I, const char* slot, int c0, int y,
                                               float f[9], float g[9]) {
  using Fmt = StashFmt<StF32>;
  const bool wb = (y == 0), wt = (y == I.ny - 1);
  const float2* b = reinterpret_cast<const float2*>(slot) + c0;
  if (!wb && !wt) {  // interior row: constant offsets
#pragma unroll
    for (int i = 0; i < 9; i++) {
      const float2 v = b[i * Fmt::EW - EX(i)];
      f[i] = v.x;
      g[i] = v.y;
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 9; i++) {
    const bool wall = (EY(i) == 1 && wb) || (EY(i) == -1 && wt);
    const float2 v = wall ? b[i * Fmt::EW] : b[i * Fmt::EW - EX(i)];
    f[i] = v.x;
    g[i] = v.y;
  }
}

// 16-bit pair layout: f_i and g_i (i >= 1) of a pulled cell with one 4-byte
// load; f_0 from its row, g_0 from the FP32 row.
template <class S>
__device__ __forceinline__ void wstash_pull_fg16(const InstDev& I, const Phys<float>& P,
                                                 const char* slot, int c0, int c0g, int y,
                                                 float f[9], float g[9]) {
  using Fmt = StashFmt<S>;
  using E = typename Fmt::E;
  const bool wb = (y == 0), wt = (y == I.ny - 1);
  f[0] = S::cvt(reinterpret_cast<const E*>(slot + Fmt::F0)[c0]) * P.inv_s[0];
  g[0] = reinterpret_cast<const float*>(slot + Fmt::G0)[c0g];
  const bool interior = !wb && !wt;
#pragma unroll
  for (int i = 1; i < 9; i++) {
    const bool wall = !interior && ((EY(i) == 1 && wb) || (EY(i) == -1 && wt));
    const E* r = reinterpret_cast<const E*>(slot + (i - 1) * Fmt::PROW);
    const int col = wall ? c0 : c0 - EX(i);
    const float2 v = S::cvt2(r + 2 * col);
    f[i] = v.x * P.inv_s[0];
    g[i] = v.y * P.inv_s[1];
  }
}

// F16MIX: f_i, g_i and hbar_i of a pulled cell with one 8-byte load (the
// three follow the same neighbour, and the same wall rule but for the
// anti-bounce-back of hbar), with the rules of pull9 (lbe_tile.cuh) for
// hbar; g_0 from the FP32 row and its low part from word 0.  c0: the
// thread's own column in a row.  RAW: as in wstash_pull.
template <bool RAW>
__device__ __forceinline__ void wstash_pull_mix(const InstDev& I, const Phys<float>& P,
                                                const char* slot, int c0, int y, int xw,
                                                float f[9], float g[9], float h[9],
                                                float& g0lo) {
  using Fmt = StashFmt<StMix>;
  const bool wb = (y == 0), wt = (y == I.ny - 1);
  const uint2* b = reinterpret_cast<const uint2*>(slot) + c0;
  const float sg = P.inv_s[1], sh = P.inv_s[2];
  auto two = [](uint32_t u) {
    __half2 q;
    memcpy(&q, &u, 4);
    return __half22float2(q);
  };
  {
    const uint2 v = b[0];
    const float2 q = two(v.y);
    f[0] = __uint_as_float(v.x);
    h[0] = q.x * sh;
    g0lo = q.y * G0LO_INV;
    g[0] = reinterpret_cast<const float*>(slot + Fmt::G0)[c0];
  }
  if (!wb && !wt) {  // interior row: constant offsets
#pragma unroll
    for (int i = 1; i < 9; i++) {
      const uint2 v = b[i * Fmt::EW - EX(i)];
      const float2 q = two(v.y);
      f[i] = __uint_as_float(v.x);
      g[i] = q.x * sg;
      float hv = q.y * sh;
      if (!RAW && EY(i) == 1) hv -= WGT<float>(i) * P.dh;
      if (!RAW && EY(i) == -1) hv += WGT<float>(i) * P.dh;
      h[i] = hv;
    }
    return;
  }
  const float Tw = wall_T<StMix>(I, xw, wb ? 0 : 1);
#pragma unroll
  for (int i = 1; i < 9; i++) {
    const bool wall = (EY(i) == 1 && wb) || (EY(i) == -1 && wt);
    const uint2 v = wall ? b[i * Fmt::EW] : b[i * Fmt::EW - EX(i)];
    const float2 q = two(v.y);
    f[i] = __uint_as_float(v.x);
    g[i] = q.x * sg;
    float hv = q.y * sh;
    if (wall) {
      hv = -hv + 2.f * WGT<float>(i) * P.rho * P.cv * link_T<StMix>(I, P, xw, i, wb ? 0 : 1, Tw);
    } else if (EY(i) == 1) {
      hv -= WGT<float>(i) * P.dh;
    } else if (EY(i) == -1) {
      hv += WGT<float>(i) * P.dh;
    }
    h[i] = hv;
  }
}

// Moments c (two floats), p and T' of a cell of an interior row (no wall
// rule) of the 16-bit forms, from the stash: the 16-bit values are summed as
// stored and each sum is scaled once by its power-of-two 1/s_k, which gives
// the sums of the scaled values bit for bit (a power of two commutes with
// every rounding in the normal range) with 1/s_k applied to 3 sums instead
// of 26 values.  Same order of additions as sum9 and moment_c.
template <class S>
__device__ __forceinline__ void moments16_interior(const Phys<float>& P, const char* slot,
                                                   int c0, int c0g, float& c, float& clo,
                                                   float& p, float& Tp, float g0lo) {
  using Fmt = StashFmt<S>;
  using E = typename Fmt::E;
  float qf[9], qg[9], qh[9];
  qf[0] = S::cvt(reinterpret_cast<const E*>(slot + Fmt::F0)[c0]);
#pragma unroll
  for (int i = 1; i < 9; i++) {
    const E* r = reinterpret_cast<const E*>(slot + (i - 1) * Fmt::PROW);
    const float2 v = S::cvt2(r + 2 * (c0 - EX(i)));
    qf[i] = v.x;
    qg[i] = v.y;
  }
#pragma unroll
  for (int i = 0; i < 9; i++)
    qh[i] = S::cvt(reinterpret_cast<const E*>(slot + Fmt::off(2, i))[c0 - EX(i)]);
  p = sum9(qf) * P.inv_s[0];
  const float s8 = (((qg[1] + qg[2]) + (qg[3] + qg[4])) + ((qg[5] + qg[6]) + (qg[7] + qg[8]))) *
                   P.inv_s[1];
  const float g0 = reinterpret_cast<const float*>(slot + Fmt::G0)[c0g];
  float e;
  two_sum(g0, s8, c, e);
  clo = e + g0lo;
  Tp = dv(sum9(qh) * P.inv_s[2], P.rho_cv, P.inv_rho_cv);
}
// The same for F16MIX (f in FP32 as it is; g_i and the hbar deviations as
// stored, their sums scaled once).
__device__ __forceinline__ void moments_mix_interior(const Phys<float>& P, const char* slot, int c0,
                                                     float& c, float& clo, float& p, float& Tp) {
  using Fmt = StashFmt<StMix>;
  const uint2* b = reinterpret_cast<const uint2*>(slot) + c0;
  auto two = [](uint32_t u) {
    __half2 q;
    memcpy(&q, &u, 4);
    return __half22float2(q);
  };
  float f[9], qg[9], qh[9];
  float g0lo;
  {
    const uint2 v = b[0];
    const float2 q = two(v.y);
    f[0] = __uint_as_float(v.x);
    qh[0] = q.x;
    g0lo = q.y * G0LO_INV;
  }
#pragma unroll
  for (int i = 1; i < 9; i++) {
    const uint2 v = b[i * Fmt::EW - EX(i)];
    const float2 q = two(v.y);
    f[i] = __uint_as_float(v.x);
    qg[i] = q.x;
    qh[i] = q.y;
  }
  p = sum9(f);
  const float s8 = (((qg[1] + qg[2]) + (qg[3] + qg[4])) + ((qg[5] + qg[6]) + (qg[7] + qg[8]))) *
                   P.inv_s[1];
  const float g0 = reinterpret_cast<const float*>(slot + Fmt::G0)[c0];
  float e;
  two_sum(g0, s8, c, e);
  clo = e + g0lo;
  Tp = dv(sum9(qh) * P.inv_s[2], P.rho_cv, P.inv_rho_cv);
}

// True in exactly one lane of the (converged) warp.
__device__ __forceinline__ bool elect_one() {
  uint32_t e;
  asm volatile(
      "{\n .reg .b32 r;\n .reg .pred p;\n elect.sync r|p, 0xffffffff;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(e));
  return e != 0;
}

// Warp-uniform source addresses of a CTA's copies in one item: the start of
// its column window (from element x0, or x0 rounded down to a multiple of 8
// for 16-bit rows) in row 0 of the first pair plane, of the first hbar plane,
// of the f_0 and g_0 planes (16-bit forms) and of the g_0 low part; the row
// strides in bytes (elements of 8, 4 and 2 bytes) and the plane strides.
// Built from values broadcast from lane 0, so that the copies' operands stay
// in uniform registers and one elected lane issues each copy as one
// instruction.
struct CopyPlan {
  const char *pair, *h, *f0, *g0, *lo;
  int64_t row8, row4, row2, pp, pb;
};
__device__ __forceinline__ int64_t bcast64(int64_t v) {
  return (int64_t)__shfl_sync(0xffffffffu, (unsigned long long)v, 0);
}
__device__ __forceinline__ CopyPlan copy_plan(const InstDev& I, int parity, int x0) {
  const char* src = reinterpret_cast<const char*>(
      __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(I.buf[parity]), 0));
  const int64_t pitch = bcast64(I.pitch);
  const int e16 = x0 & ~7;
  const bool w16 = I.storage == ST_F16DEV || I.storage == ST_BF16DEV;
  CopyPlan c;
  c.row8 = pitch * 8;
  c.row4 = pitch * 4;
  c.row2 = pitch * 2;
  c.pp = bcast64((int64_t)I.pair_bytes);
  c.pb = bcast64((int64_t)I.plane_bytes);
  c.pair = src + (w16 ? (int64_t)e16 * 4 : (int64_t)x0 * 8);
  c.h = src + bcast64((int64_t)I.h_off) + (w16 ? (int64_t)e16 * 2 : (int64_t)x0 * 4);
  c.f0 = src + bcast64((int64_t)I.f0_off) + (int64_t)e16 * 2;
  c.g0 = src + bcast64((int64_t)I.g0_off) + (int64_t)x0 * 4;
  c.lo = src + bcast64((int64_t)I.g0lo_off) + (int64_t)e16 * 2;
  return c;
}

// The copies of one row: the populations pulled by the cells of moment row
// mr (or, at a wall, the reversed populations of row mr itself), as calls
// copy(byte offset in the stash slot, source address, bytes).
//   FP32 (19 copies): the 9 (f_i, g_i) pair rows, the 9 hbar_i rows, the
//     g_0 low part.
//   16-bit (20 copies): the 8 pair rows (i = 1..8), f_0, the 9 hbar_i rows,
//     the FP32 g_0 row, the g_0 low part.
//   F16MIX (10 copies): the 9 rows of direction words, the FP32 g_0 row.
// WALL: mr is the first or the last row (else the pulls need no wall rule).
template <class S, bool WALL, class Copy>
__device__ __forceinline__ void row_copies(const CopyPlan& c, int mr, int ny, Copy&& copy) {
  using Fmt = StashFmt<S>;
  const bool wb = WALL && mr == 0, wt = WALL && mr == ny - 1;
  // source row and plane of population i (the reversed one at a wall)
  auto at = [&](int i, int64_t row) -> int64_t {
    const bool wall = (EY(i) == 1 && wb) || (EY(i) == -1 && wt);
    return wall ? (int64_t)mr * row : (int64_t)(mr - EY(i)) * row;
  };
  auto pl = [&](int i) {
    const bool wall = (EY(i) == 1 && wb) || (EY(i) == -1 && wt);
    return wall ? OPP(i) : i;
  };
  if constexpr (S::kind == ST_F16MIX) {
#pragma unroll
    for (int i = 0; i < 9; i++)
      copy(i * Fmt::WROW, c.pair + pl(i) * c.pp + at(i, c.row8), Fmt::WROW);
    copy(Fmt::G0, c.g0 + (int64_t)mr * c.row4, Fmt::G0B);
  } else if constexpr (S::kind == ST_F32) {
#pragma unroll
    for (int i = 0; i < 9; i++)
      copy(Fmt::off(0, i), c.pair + pl(i) * c.pp + at(i, c.row8), Fmt::PROW);
#pragma unroll
    for (int i = 0; i < 9; i++)
      copy(Fmt::off(2, i), c.h + pl(i) * c.pb + at(i, c.row4), Fmt::ROW);
  } else {
#pragma unroll
    for (int i = 1; i < 9; i++)
      copy(Fmt::off(0, i), c.pair + (pl(i) - 1) * c.pp + at(i, c.row4), Fmt::PROW);
    copy(Fmt::F0, c.f0 + (int64_t)mr * c.row2, Fmt::ROW);
#pragma unroll
    for (int i = 0; i < 9; i++)
      copy(Fmt::off(2, i), c.h + pl(i) * c.pb + at(i, c.row2), Fmt::ROW);
    copy(Fmt::G0, c.g0 + (int64_t)mr * c.row4, Fmt::G0B);
  }
  if constexpr (S::kind != ST_F16MIX) copy(Fmt::LO, c.lo + (int64_t)mr * c.row2, Fmt::LOB);
}

// The row's copies into the stash slot at shared address dst, completing on
// the slot's barrier bar.
template <class S, bool WALL>
__device__ __forceinline__ void issue_row(const CopyPlan& c, uint32_t dst, uint32_t bar, int mr,
                                          int ny) {
  row_copies<S, WALL>(c, mr, ny, [&](int off, const char* src, int bytes) {
    bulk_load(dst + (uint32_t)off, src, (uint32_t)bytes, bar);
  });
}

// VAR: the boundary and property variants (harmonic law, wall temperature
// at the link's wall crossing, wetting walls) compiled in; without them the
// kernel carries none of their registers.
// OWN: the kernel writes the periodic ghost columns of its output itself
// (a compile-time choice: compiled in, the ghost stores cost the main
// stores about 1 % even where no lane takes them).
template <class S, int NC, bool VAR, bool OWN>
__global__ void __launch_bounds__(NC, (StashCfg<S, NC>::MINB))
stash_kernel(const InstDev* __restrict__ insts, int n_inst, int64_t total_items, int seg_rows,
             int parity, int* __restrict__ err, int poll_lim, int withhold,
             const uint32_t* __restrict__ seed) {
  using Cfg = StashCfg<S, NC>;
  using Fmt = typename Cfg::Fmt;
  using C = float;
  constexpr bool W16 = sizeof(typename Fmt::E) == 2;
  constexpr bool MIX = S::kind == ST_F16MIX;
  extern __shared__ __align__(128) char smem[];
  constexpr int CW = Cfg::CW, QW = Cfg::QW;
  // ring entry of column x0 + j: c (and its low part) at j + 2, p, T, n at j + 1
  C* cring = reinterpret_cast<C*>(smem + Cfg::STASH);  // [CR][CW]
  C* pring = cring + Cfg::CR * CW;                       // [PR][QW]
  C* Tring = pring + Cfg::PR * QW;                       // [PR][QW]
  C* nxr = Tring + Cfg::PR * QW;                         // [NR][QW]
  C* nyr = nxr + Cfg::NR * QW;
  __half* clr = reinterpret_cast<__half*>(nyr + Cfg::NR * QW);  // [CR][CW], lo * 2^24
  // [SR] full barriers, then [SR] empty barriers
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::STASH + Cfg::RINGS);
  __shared__ int s_abort;
  const int t = threadIdx.x;
  const int wu = __shfl_sync(0xffffffffu, t >> 5, 0);  // the warp index, warp-uniform
  // halo lanes: lanes 0..3 of the last warp form the moments of columns
  // x0 - 2, x0 - 1, x0 + NC, x0 + NC + 1 (offset hj from x0)
  const int lane = t & 31;
  const bool halo = wu == Cfg::NW - 1 && lane < 4;
  const int hj = lane < 2 ? lane - 2 : NC - 2 + lane;
  const uint32_t stash_u = smem_u32(smem);
  const uint32_t bars_u = smem_u32(bars);
  const uint32_t empty_u = bars_u + 8 * Cfg::SR;
  // the slots' barriers are initialised once; every copy issued in an item is
  // waited for in that item, so the phase bits carry over between items
  if (t == 0) {
    for (int s = 0; s < Cfg::SR; s++) {
      mbar_init(bars_u + 8 * s, 1);
      mbar_init(empty_u + 8 * s, NC);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  unsigned phase = 0;    // bit s: parity of the next completion of slot s
  unsigned ephase = 0;   // bit s: parity of the next release of slot s
  unsigned pending = 0;  // bit s: slot s has copies not yet waited for
  // the handle's step counter (random bits of the stochastic rounding)
  const uint32_t step = S::SR ? __ldg(seed) : 0u;

  // Work assignment.  seg_rows > 0: items of seg_rows rows of one strip
  // (tile_begin counts items), taken round-robin.  seg_rows <= 0: the rows
  // of all strips of all instances as one sequence (tile_begin counts strip
  // rows), cut into gridDim.x contiguous ranges of equal length; a CTA's
  // items are the pieces of its range in each strip it meets, so that every
  // CTA marches over the same number of rows whatever the mix of grid sizes
  // (fixed items leave a partial last wave); seg_rows < 0 cuts the pieces
  // further, to at most -seg_rows rows each.  The sequence runs through an
  // instance band by band (bands of tiles_y rows), and through a band strip
  // by strip: neighbouring CTAs then march side by side over the same rows,
  // so that the rows read at one time are whole rows of the planes (in the
  // strip-by-strip order they were 1 KB pieces of rows hundreds apart, and
  // the step ran 2.4 % slower).
  const bool balanced = seg_rows <= 0;
  const int64_t piece = seg_rows < 0 ? -(int64_t)seg_rows : 0;  // 0: uncut
  int64_t g = balanced ? (int64_t)blockIdx.x * total_items / gridDim.x : (int64_t)blockIdx.x;
  const int64_t gend =
      balanced ? (int64_t)(blockIdx.x + 1) * total_items / gridDim.x : total_items;
  while (g < gend) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (insts[mid].tile_begin <= g) lo = mid; else hi = mid - 1;
    }
    const InstDev& I = insts[lo];
    const int64_t local = g - I.tile_begin;
    // the item's scalars, broadcast from lane 0 so that the compiler knows
    // them to be warp-uniform (and so the row loop and the copy operands)
    const int nx = I.nx, ny = __shfl_sync(0xffffffffu, I.ny, 0);
    int strip, ya, yb;
    if (balanced) {
      const int ns = I.tiles_x, B = I.tiles_y;  // strips, band height
      const int64_t band = min(local / ((int64_t)ns * B), (int64_t)(ny - 1) / B);
      const int y0 = (int)band * B, bh = min(B, ny - y0);
      const int64_t rem = local - band * ns * B;
      strip = (int)(rem / bh);
      ya = y0 + (int)(rem - (int64_t)strip * bh);
      int64_t lim = min((int64_t)(y0 + bh), (int64_t)ya + (gend - g));
      if (piece > 0) lim = min(lim, (int64_t)ya + piece);
      yb = (int)lim;
      // (never taken: every piece holds at least one row of the strip; a
      // guard against a work loop that would not advance or leave the grid)
      if (yb <= ya || ya < 0 || yb > ny || strip >= ns) {
        if (threadIdx.x == 0) atomicOr(err, 2);
        break;
      }
      g += yb - ya;
    } else {
      strip = (int)(local % I.tiles_x);
      ya = (int)(local / I.tiles_x) * seg_rows;
      yb = min(ya + seg_rows, ny);
      g += gridDim.x;
    }
    const int x0 = __shfl_sync(0xffffffffu, strip * Cfg::NCO, 0);
    ya = __shfl_sync(0xffffffffu, ya, 0);
    yb = __shfl_sync(0xffffffffu, yb, 0);
    char* __restrict__ dst = I.buf[parity ^ 1];
    Phys<C> P = phys<C>(I);
    if constexpr (!VAR) {  // the variants are off: known to the compiler
      P.harm = C(0);
      P.wmid = C(0);
      P.kw = C(0);
    }
    const C en2 = P.eta_n2;
    const uint32_t skey = S::SR ? sr_step_key(step, I.salt) : 0u;
    const size_t pitch = (size_t)I.pitch;
    const int x = x0 + t;
    const int xw = wrapx(x, nx);
    const bool collides = x < nx;
    // OWN: the periodic ghost copies are written by the owner of the cell,
    // element XG + x + nx for x < XG (right ghosts), XG + x - nx for
    // x >= nx - XG (left ghosts), both for 4 <= nx < 2 XG; otherwise
    // ghost_kernel refreshes them after the step
    const bool gR = OWN && collides && x < XG;
    const bool gL = OWN && collides && x >= nx - XG;
    const int ndst = 1 + (int)gR + (int)gL;
    // staged elements of the strip's population rows (storage element e
    // holds column e - XG): column x0 + j is element j + XG of a stash row,
    // which starts at element x0 (a multiple of NC: 16-byte aligned).
    const int e16 = x0 & ~7;
    static_assert(XG == 4, "stash columns: column x0 + j at element j + 4 of a row");
    const int c0 = (W16 ? x0 - e16 : 0) + t + XG;  // own column in a population row
    const int c0g = t + XG;                         // own column in the FP32 g_0 row
    const int c0lo = x0 - e16 + t + XG;             // own column in the g_0 low-part row
    const int hd = hj - t;                          // halo lanes: column offset from own
    const int hxw = wrapx(x0 + hj, nx);
    const CopyPlan cp = copy_plan(I, parity, x0);
    __syncthreads();  // the previous item is done with the rings and stashes
    if (t == 0) s_abort = 0;

    auto slot = [&](int m) { return smem + (m & (Cfg::SR - 1)) * Cfg::SLOT; };
    auto rrow = [](int m) { return ((m % Cfg::CR) + Cfg::CR) % Cfg::CR; };
    auto nr = [](int m) { return (m & (Cfg::NR - 1)) * QW; };
    auto loadable = [&](int m) { return m <= yb + 1 && m < ny; };
    // the copies of the populations pulled by moment row m (the mirror row's
    // below the bottom wall), issued by one elected lane of warp 0.  In the
    // row loop the slot is that of the row collided in the same iteration:
    // the lane first waits (bounded) for the slot's empty barrier, on which
    // every thread arrives once per iteration after its last read of the
    // slot (release = false: the slot is free already, at an item start).
    auto issue = [&](int m, bool release) {
      const int sl = m & (Cfg::SR - 1);
      const unsigned epar = (ephase >> sl) & 1u;
      if (release) ephase ^= 1u << sl;  // one release of this slot per iteration
      if (!loadable(m)) return;
      pending |= 1u << sl;
      if (wu != 0) return;
      __syncwarp();
      if (elect_one()) {
        if (release && !mbar_wait(empty_u + 8 * sl, epar, poll_lim)) {
          // no copy issued after a failed wait (the slot may still be read)
          s_abort = 1;
          atomicOr(err, 1);
          return;
        }
        const uint32_t bar = bars_u + (uint32_t)(sl * 8);
        const uint32_t dstw = stash_u + (uint32_t)(sl * Cfg::SLOT);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, Cfg::TX);
        const int mr = m >= 0 ? m : -1 - m;
        if (mr == withhold) {
          // test hook: nothing issued, the wait for this slot runs out
        } else if (mr > 0 && mr < ny - 1)
          issue_row<S, false>(cp, dstw, bar, mr, ny);
        else
          issue_row<S, true>(cp, dstw, bar, mr, ny);
      }
    };
    auto wait_row = [&](int m) -> bool {
      if (!loadable(m)) return true;
      const int s = m & (Cfg::SR - 1);
      const bool ok = mbar_wait(bars_u + 8 * s, (phase >> s) & 1u, poll_lim);
      if (ok) {
        phase ^= 1u << s;
        pending &= ~(1u << s);
      }
      return ok;
    };

    issue(ya - 2, false);
    int i5 = (((ya - 4) % Cfg::CR) + Cfg::CR) % Cfg::CR;  // i mod CR
    for (int i = ya - 4; i <= yb; i++, i5 = (i5 == Cfg::CR - 1) ? 0 : i5 + 1) {
      // ring row of i + d (|d| < CR)
      auto rr = [&](int d) {
        int v = i5 + d;
        return v < 0 ? v + Cfg::CR : (v >= Cfg::CR ? v - Cfg::CR : v);
      };
      __syncthreads();
      if (s_abort) break;

      // ---- 1. collide row r = i - 1 (every thread then releases its slot)
      const int r = i - 1;
      const uint32_t ebar = empty_u + 8u * (uint32_t)(r & (Cfg::SR - 1));
      if (r >= ya && r < yb && collides) {
        const char* s = slot(r);
        C f[9], g[9], h[9], g0lo;
        // hbar as pulled (without the change of reference row in interior
        // rows, which collide() applies through the source term)
        if constexpr (MIX) {
          wstash_pull_mix<true>(I, P, s, c0, r, x, f, g, h, g0lo);
        } else {
          if constexpr (!W16) {
            wstash_pull_fg(I, s, c0, r, f, g);
          } else {
            wstash_pull_fg16<S>(I, P, s, c0, c0g, r, f, g);
          }
          wstash_pull<S, 2, true>(I, P, s, c0, c0g, r, x, h);
          g0lo = __half2float(reinterpret_cast<const __half*>(s + Fmt::LO)[c0lo]) * G0LO_INV;
        }
        mbar_arrive(ebar);  // done with the slot (the arrive orders the reads before it)
        const int ps = rr(-2), p0 = rr(-1), pn = rr(0);  // rows r-1, r, r+1
        // rows of the rings from column x0 (index t: the own column)
        const C* cs = cring + ps * CW + 2;
        const C* c0 = cring + p0 * CW + 2;
        const C* cn = cring + pn * CW + 2;
        const C cc = c0[t];
        const C clo = lo_at(clr + p0 * CW + 2, t);
        const C* Ts = Tring + ps * QW + 1;
        const C* T0 = Tring + p0 * QW + 1;
        const C* Tn = Tring + pn * QW + 1;
        const C* qs = pring + ps * QW + 1;
        const C* q0 = pring + p0 * QW + 1;
        const C* qn = pring + pn * QW + 1;
        const C pp = q0[t], TT = T0[t];
        Stencils<C> st;
        grad3(cs, c0, cn, t, st.gcx, st.gcy);
        st.lapc = lap3(cs, c0, cn, t);
        grad3(Ts, T0, Tn, t, st.gTx, st.gTy);
        if (dev_h<S>()) st.gTy += P.hr1;
        grad3(qs, q0, qn, t, st.gpx, st.gpy);
        const int ns = nr(r - 1) + 1, n0 = nr(r) + 1, nn = nr(r + 1) + 1;
        C d1, d2, dum;
        grad3(nxr + ns, nxr + n0, nxr + nn, t, d1, dum);
        grad3(nyr + ns, nyr + n0, nyr + nn, t, dum, d2);
        st.kappa = d1 + d2;
        const Drive<S> d = drive<S>(P, r, f, cc, TT, st);
        C o[27];
        C lo_out = C(0);
        const C dhc = (r > 0 && r < I.ny - 1) ? P.dh : C(0);
        collide<S>(P, f, g, h, cc, pp, TT, st.gpx, st.gpy, d,
                   [&](int k, int ii, C v) { o[k * 9 + ii] = v; }, g0lo, clo, &lo_out, dhc);
        // 16-bit forms: the cell's random bits for the stochastic rounding
        const uint32_t hc = S::SR ? sr_cell(skey, (uint32_t)r * (uint32_t)nx + (uint32_t)x) : 0u;
        // the cell's values stored at its element and, with OWN, by the lanes
        // of the periodic edge columns at its ghost copies (the 16-bit forms
        // round them again, with the same random bits: the same values)
        auto store_at = [&](const size_t e) {
          if constexpr (MIX) {
            // word i: (f_i, g_i, hbar_i); word 0: (f_0, hbar_0, g_0 low part)
            const float s1 = I.s[1], s2 = I.s[2];
            auto word = [&](int ii, float fv, uint32_t u) {
              reinterpret_cast<uint2*>(dst + (size_t)ii * I.pair_bytes)[e] =
                  make_uint2(__float_as_uint(fv), u);
            };
            float gs = 0.f;  // the stored g_i, times s_1
#pragma unroll
            for (int ii = 1; ii < 9; ii++) {
              const uint32_t q =
                  sr_pack_half2(o[9 + ii] * s1, o[18 + ii] * s2, S::sr_word(1, ii, hc));
              gs += __half2float(__ushort_as_half((unsigned short)(q & 0xffffu)));
              word(ii, o[ii], q);
            }
            float g0h, g0l;
            g0_remainder(cc, clo, gs * P.inv_s[1], g0h, g0l);
            word(0, o[0],
                 (uint32_t)__half_as_ushort(sr_half(o[18] * s2, S::sr_word(2, 0, hc))) |
                     ((uint32_t)__half_as_ushort(__float2half_rn(g0l * G0LO_SCALE)) << 16));
            reinterpret_cast<float*>(dst + I.g0_off)[e] = g0h;
          } else if constexpr (!W16) {
            st_g0lo<S>(I, dst, e, lo_out);
#pragma unroll
            for (int ii = 0; ii < 9; ii++) S::st_fg(I, dst, ii, e, o[ii], o[9 + ii]);
#pragma unroll
            for (int ii = 0; ii < 9; ii++) S::st(I, dst, 2, ii, e, o[18 + ii]);
          } else {
            S::st_sr(I, dst, 0, 0, e, o[0], S::sr_word(0, 0, hc));
            float gs = 0.f;  // the stored g_i, times s_1
#pragma unroll
            for (int ii = 1; ii < 9; ii++)
              gs += S::st_fg_sr(I, dst, ii, e, o[ii], o[9 + ii], S::sr_word(0, ii, hc));
            float g0h, g0l;
            g0_remainder(cc, clo, gs * P.inv_s[1], g0h, g0l);
            S::st(I, dst, 1, 0, e, g0h);
            st_g0lo<S>(I, dst, e, g0l);
#pragma unroll
            for (int ii = 0; ii < 9; ii++)
              S::st_sr(I, dst, 2, ii, e, o[18 + ii], S::sr_word(2, ii, hc));
          }
        };
        store_at((size_t)r * pitch + XG + x);
        if constexpr (OWN) {
          if (ndst > 1) {
#pragma unroll 1
            for (int dq = 1; dq < ndst; dq++)
              store_at((size_t)r * pitch + (XG + x + ((dq == 1 && gR) ? nx : -nx)));
          }
        }
      } else {
        mbar_arrive(ebar);
      }

      // ---- 2. the copies of row i + 3 into the slot of row i - 1, once
      // every thread has released it (no CTA barrier: the other warps go on
      // to the moments of row i + 2, which touch neither that slot nor the
      // ring rows the collision reads)
      issue(i + 3, true);

      // ---- 3. moments of row m = i + 2
      const int m = i + 2;
      if (!wait_row(m)) {
        s_abort = 1;
        atomicOr(err, 1);
      }
      if (m <= yb + 1) {
        const int rm = rr(2);
        // moments of the column at offset dj from the own one into ring
        // entries ci (c) and, if pt, pi (p, T)
        auto moments = [&](int dj, int cxw, int ci, int pi, bool pt) {
          if (m < ny) {
            const int mr = m >= 0 ? m : -1 - m;
            const char* s = slot(m);
            C v[9], vf[9];
            bool done = false;
            if constexpr (MIX || W16) {
              if (mr > 0 && mr < ny - 1) {
                // interior row of a 16-bit form: sums of the stored values
                C cv, clo, pv, Tv;
                if constexpr (MIX) {
                  moments_mix_interior(P, s, c0 + dj, cv, clo, pv, Tv);
                } else {
                  const C g0lo =
                      __half2float(reinterpret_cast<const __half*>(s + Fmt::LO)[c0lo + dj]) *
                      G0LO_INV;
                  moments16_interior<S>(P, s, c0 + dj, c0g + dj, cv, clo, pv, Tv, g0lo);
                }
                cring[ci] = m < 0 ? wet_ghost(P, cv, -1 - m) : cv;
                clr[ci] = __float2half_rn(clo * G0LO_SCALE);
                if (pt) {
                  pring[pi] = pv;
                  Tring[pi] = m < 0 ? ghost_T<S>(I, cxw, true, Tv) : Tv;
                }
                done = true;
              }
            }
            if (done) {
            } else if constexpr (MIX) {
              C vh[9], g0lo, clo;
              wstash_pull_mix<true>(I, P, s, c0 + dj, mr, cxw, vf, v, vh, g0lo);
              cring[ci] = moment_c(v, g0lo, clo);
              if (m < 0) cring[ci] = wet_ghost(P, cring[ci], -1 - m);
              clr[ci] = __float2half_rn(clo * G0LO_SCALE);
              if (pt) {
                pring[pi] = sum9(vf);
                C T = dv(sum9(vh), P.rho_cv, P.inv_rho_cv);
                if (m < 0) T = ghost_T<S>(I, cxw, true, T);
                Tring[pi] = T;
              }
            } else {
              if constexpr (!W16) {
                wstash_pull_fg(I, s, c0 + dj, mr, vf, v);
              } else {
                wstash_pull_fg16<S>(I, P, s, c0 + dj, c0g + dj, mr, vf, v);
              }
              const C g0lo =
                  __half2float(reinterpret_cast<const __half*>(s + Fmt::LO)[c0lo + dj]) *
                  G0LO_INV;
              C clo;
              cring[ci] = moment_c(v, g0lo, clo);
              if (m < 0) cring[ci] = wet_ghost(P, cring[ci], -1 - m);
              clr[ci] = __float2half_rn(clo * G0LO_SCALE);
              if (pt) {
                pring[pi] = sum9(vf);
                wstash_pull<S, 2, true>(I, P, s, c0 + dj, c0g + dj, mr, cxw, v);
                C T = dv(sum9(v), P.rho_cv, P.inv_rho_cv);
                if (m < 0) T = ghost_T<S>(I, cxw, true, T);
                Tring[pi] = T;
              }
            }
          } else {
            // above the top wall: the mirror row's moments
            const int mm = rrow(2 * ny - 1 - m);
            const int cm = ci - rm * CW + mm * CW, pm = pi - rm * QW + mm * QW;
            cring[ci] = wet_ghost(P, cring[cm], m - ny);
            clr[ci] = clr[cm];
            if (pt) {
              pring[pi] = pring[pm];
              Tring[pi] = ghost_T<S>(I, cxw, false, Tring[pm]);
            }
          }
        };
        moments(0, xw, rm * CW + t + 2, rm * QW + t + 1, true);
        // the halo columns: c of all four, p and T of x0 - 1 and x0 + NC
        if (halo)
          moments(hd, hxw, rm * CW + hj + 2, rm * QW + hj + 1, lane == 1 || lane == 2);
      }
      __syncthreads();
      if (s_abort) break;

      // ---- 4. unit normal of row i + 1
      const int mn = i + 1;
      if (mn >= ya - 1 && mn <= yb) {
        const C* ca = cring + rr(0) * CW;
        const C* cb = cring + rr(1) * CW;
        const C* cc2 = cring + rr(2) * CW;
        normal3(ca, cb, cc2, t + 2, en2, nxr[nr(mn) + t + 1], nyr[nr(mn) + t + 1]);
        // the halo columns x0 - 1 and x0 + NC
        if (halo && (lane == 1 || lane == 2))
          normal3(ca, cb, cc2, hj + 2, en2, nxr[nr(mn) + hj + 1], nyr[nr(mn) + hj + 1]);
      }
    }
    __syncthreads();
    if (s_abort) {
      // no copy is issued after the failed wait (the loop left at the barrier
      // that followed it); bounded wait for the copies still in flight, then
      // stop.  Every thread tracks the same pending slots.
      for (int sl = 0; sl < Cfg::SR; sl++)
        if (pending & (1u << sl)) mbar_wait(bars_u + 8 * sl, (phase >> sl) & 1u, poll_lim);
      __syncthreads();
      return;
    }
  }
}

}  // namespace lbe

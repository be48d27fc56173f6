// The fused step as a column-strip marching kernel with TMA row staging.
//
// A work item is a strip of NC columns [x0, x0+NC) and a segment of rows
// [ya, yb) of one instance.  One CTA of NC threads (one column each) marches
// up the rows.  The source rows it needs (all 27 population planes of row q,
// columns x0-XG .. x0+NC+XG) are copied into a ring of R shared-memory slots
// by one TMA tiled load per row (cp.async.bulk.tensor, completion on an
// mbarrier per slot), issued up to two rows ahead of use.  Per output row r:
//   1. moments c, p, T of row r+2 (S1), pulled from the staged rows r+1..r+3
//      (rows beyond a wall are ghosts: mirror for c and p, 2 T_w - T for T);
//      a ring of the last 5 moment rows feeds the stencils;
//   2. unit normal of row r+1 (S2) into a ring of 3 rows;
//   3. the stencils, force, velocity and three collisions of row r (S2-S9,
//      lbe_cell.cuh) from the staged rows r-1..r+1 and the rings, and the 27
//      stores of the post-collision values with their periodic ghost copies.
// Every moment and normal is computed once per strip (only 4 halo columns are
// recomputed by the neighbouring strip), every population is read from HBM
// once per step, and the per-cell arithmetic is that of the tile kernel, so
// the two kernels produce bitwise-equal results.
//
// Every mbarrier wait is bounded; on time-out the kernel sets *err, waits
// (bounded) for its own copies in flight and returns.
#pragma once

#include <cuda.h>

#include "lbe_tile.cuh"

namespace lbe {

// Tensor maps of one instance: m[buffer][0] covers the 27 (FP32) or 26
// (16-bit) population planes as a 3D tensor {pitch, ny, planes}; m[buffer][1]
// the FP32 g_0 plane of the 16-bit forms as a 2D tensor {pitch, ny}.
struct alignas(64) TmapSet {
  CUtensorMap m[2][2];
};

template <class S>
struct RowFmt;
template <>
struct RowFmt<StF32> {
  using E = float;
  static constexpr int planes = 27;
  static constexpr bool g0 = false;
};
template <>
struct RowFmt<StF16> {
  using E = __half;
  static constexpr int planes = 26;
  static constexpr bool g0 = true;
};
template <>
struct RowFmt<StBF16> {
  using E = __nv_bfloat16;
  static constexpr int planes = 26;
  static constexpr bool g0 = true;
};

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
// Bounded wait for the phase with the given parity; false on time-out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
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
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

template <class S, int NC, int R>
struct Strip {
  using C = typename S::C;
  using F = RowFmt<S>;
  using E = typename F::E;
  static constexpr int BW = NC + 2 * XG;  // staged columns x0-XG .. x0+NC+XG-1
  static constexpr int MAIN = F::planes * BW * (int)sizeof(E);
  static constexpr int G0OFF = (MAIN + 127) / 128 * 128;
  static constexpr int ROW_BYTES = MAIN + (F::g0 ? BW * 4 : 0);  // TMA bytes per row
  static constexpr int SLOT = (G0OFF + (F::g0 ? BW * 4 : 0) + 127) / 128 * 128;
  static constexpr int RW = NC + 4;  // moment ring columns x0-2 .. x0+NC+1
  static constexpr int QW = NC + 2;  // normal ring columns x0-1 .. x0+NC
  static constexpr int SMEM = R * SLOT + 5 * RW * 3 * (int)sizeof(C) +
                              3 * QW * 2 * (int)sizeof(C) + R * 8 + 16;

  // population (k, i) at staged column col of a slot
  __device__ static __forceinline__ C sld(const Phys<C>& P, const char* slot, int k, int i,
                                          int col) {
    if constexpr (S::kind == ST_F32) {
      return reinterpret_cast<const float*>(slot)[(k * 9 + i) * BW + col];
    } else {
      if (k == 1 && i == 0) return reinterpret_cast<const float*>(slot + G0OFF)[col];
      return S::cvt(reinterpret_cast<const E*>(slot)[dev_plane(k, i) * BW + col]) * P.inv_s[k];
    }
  }

  // Pull of lattice K at staged column col, row y, from the slots holding
  // rows y-1 (sm), y (s0), y+1 (sp); same rules and arithmetic as pull9.
  template <int K>
  __device__ static __forceinline__ void spull9(const InstDev& I, const Phys<C>& P, const char* sm,
                                                const char* s0, const char* sp, int col, int y,
                                                int xw, C out[9]) {
    constexpr bool DEV = (K == 2) && dev_h<S>();
    const bool wb = (y == 0), wt = (y == I.ny - 1);
    C Tw = C(0);
    if (K == 2 && (wb || wt)) Tw = wall_T<S>(I, xw, wb ? 0 : 1);
    const C dh = DEV ? P.dh : C(0);
    auto bb = [&](int i) -> C {
      C v = sld(P, s0, K, OPP(i), col);
      if (K == 2) return -v + C(2) * WGT<C>(i) * P.rho * P.cv * Tw;
      return v;
    };
    out[0] = sld(P, s0, K, 0, col);
    out[1] = sld(P, s0, K, 1, col - 1);
    out[3] = sld(P, s0, K, 3, col + 1);
    if (wb) {
      out[2] = bb(2);
      out[5] = bb(5);
      out[6] = bb(6);
    } else {
      out[2] = sld(P, sm, K, 2, col);
      out[5] = sld(P, sm, K, 5, col - 1);
      out[6] = sld(P, sm, K, 6, col + 1);
      if (DEV) {
        out[2] -= WGT<C>(2) * dh;
        out[5] -= WGT<C>(5) * dh;
        out[6] -= WGT<C>(6) * dh;
      }
    }
    if (wt) {
      out[4] = bb(4);
      out[7] = bb(7);
      out[8] = bb(8);
    } else {
      out[4] = sld(P, sp, K, 4, col);
      out[7] = sld(P, sp, K, 7, col + 1);
      out[8] = sld(P, sp, K, 8, col - 1);
      if (DEV) {
        out[4] += WGT<C>(4) * dh;
        out[7] += WGT<C>(7) * dh;
        out[8] += WGT<C>(8) * dh;
      }
    }
  }
};

template <class S, int NC, int R>
__global__ void __launch_bounds__(NC)
strip_kernel(const InstDev* __restrict__ insts, const TmapSet* __restrict__ maps, int n_inst,
             int64_t total_items, int seg_rows, int parity, int* __restrict__ err) {
  using St = Strip<S, NC, R>;
  using C = typename S::C;
  extern __shared__ __align__(128) char smem[];
  char* slots = smem;
  C* cring = reinterpret_cast<C*>(smem + R * St::SLOT);  // [5][RW]
  C* pring = cring + 5 * St::RW;
  C* Tring = pring + 5 * St::RW;
  C* nxr = Tring + 5 * St::RW;  // [3][QW]
  C* nyr = nxr + 3 * St::QW;
  uint64_t* bars = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(nyr + 3 * St::QW) + 15) & ~uintptr_t(15));
  __shared__ int s_abort;
  const int t = threadIdx.x;
  constexpr int RW = St::RW, QW = St::QW;

  for (int64_t item = blockIdx.x; item < total_items; item += gridDim.x) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (insts[mid].tile_begin <= item) lo = mid; else hi = mid - 1;
    }
    const InstDev& I = insts[lo];
    const CUtensorMap* map0 = &maps[lo].m[parity][0];
    const CUtensorMap* map1 = &maps[lo].m[parity][1];
    const int64_t local = item - I.tile_begin;
    const int nx = I.nx, ny = I.ny;
    const int x0 = (int)(local % I.tiles_x) * NC;
    const int ya = (int)(local / I.tiles_x) * seg_rows;
    const int yb = min(ya + seg_rows, ny);
    const int src_lo = max(ya - 3, 0), src_hi = min(yb + 2, ny - 1);
    char* __restrict__ dst = I.buf[parity ^ 1];
    const Phys<C> P = phys<C>(I);  // constants in registers for the whole item
    const C en2 = P.eta_n2;

    __syncthreads();  // previous item fully done with the slots and barriers
    if (t == 0) {
      s_abort = 0;
      for (int s = 0; s < R; s++) mbar_init(smem_u32(&bars[s]), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    int next = src_lo;          // next source row to issue (thread 0)
    int waited = src_lo - 1;    // highest source row waited for
    auto issue_upto = [&](int lim) {
      if (t != 0) return;
      lim = min(lim, src_hi);
      for (; next <= lim; next++) {
        const int s = (next - src_lo) % R;
        const uint32_t bar = smem_u32(&bars[s]);
        const uint32_t dsts = smem_u32(slots + s * St::SLOT);
        mbar_expect_tx(bar, St::ROW_BYTES);
        tma_load_3d(dsts, map0, x0, next, 0, bar);
        if (RowFmt<S>::g0) tma_load_2d(dsts + St::G0OFF, map1, x0, next, bar);
      }
    };
    auto wait_upto = [&](int y) -> bool {
      y = min(y, src_hi);
      for (; waited < y; waited++) {
        const int q = waited + 1;
        if (!mbar_wait(smem_u32(&bars[(q - src_lo) % R]), ((q - src_lo) / R) & 1)) {
          s_abort = 1;
          atomicOr(err, 1);
          return false;
        }
      }
      return true;
    };
    auto slot_of = [&](int q) -> const char* {
      int d = (q - src_lo) % R;
      if (d < 0) d += R;
      return slots + d * St::SLOT;
    };
    auto ring5 = [](int m) { return ((m % 5) + 5) % 5; };
    auto ring3 = [](int m) { return ((m % 3) + 3) % 3; };

    // moments c, p, T of row m (0 <= m < ny) at staged column col
    auto moments = [&](int m, int col, int xw, C& c, C& p, C& T) {
      const char* s0 = slot_of(m);
      const char* sm = m > 0 ? slot_of(m - 1) : s0;
      const char* sp = m < ny - 1 ? slot_of(m + 1) : s0;
      C v[9];
      St::template spull9<1>(I, P, sm, s0, sp, col, m, xw, v);
      c = sum9(v);
      St::template spull9<0>(I, P, sm, s0, sp, col, m, xw, v);
      p = sum9(v);
      St::template spull9<2>(I, P, sm, s0, sp, col, m, xw, v);
      T = dv(sum9(v), P.rho_cv, P.inv_rho_cv);
    };

    // per-thread constants of the item: own column and the halo columns the
    // edge threads also compute
    const int x = x0 + t;
    const bool own_active = x < nx;
    const bool edge_ghost = own_active && (x < XG || x >= nx - XG);
    int rcs[3], nrc = 0;
    rcs[nrc++] = t + 2;
    if (t == 0) {
      rcs[nrc++] = 0;
      rcs[nrc++] = 1;
    } else if (t == NC - 1) {
      rcs[nrc++] = NC + 2;
      rcs[nrc++] = NC + 3;
    }
    int xws[3];
    for (int j = 0; j < nrc; j++) xws[j] = wrapx(x0 - 2 + rcs[j], nx);
    const size_t pitch = (size_t)I.pitch;

    for (int r = ya - 4; r < yb; r++) {
      __syncthreads();
      if (s_abort) break;
      issue_upto(max(r - 2, src_lo - 1) + R);

      // ---- moments of row m = r + 2 at ring columns t+2 (+ halo columns)
      const int m = r + 2;
      if (m <= yb + 1) {
        const int ridx = ring5(m) * RW;
        if (m < ny) {
          const int mr = m >= 0 ? m : -1 - m;  // bottom ghost rows: the mirror row
          if (wait_upto(mr + 1)) {
            for (int j = 0; j < nrc; j++) {
              const int rc = rcs[j];
              C c, p, T;
              moments(mr, rc - 2 + XG, xws[j], c, p, T);
              if (m < 0) T = ghost_T<S>(I, xws[j], true, T);
              cring[ridx + rc] = c;
              pring[ridx + rc] = p;
              Tring[ridx + rc] = T;
            }
          }
        } else {
          // top ghost rows from the mirror rows still in the ring
          const int sidx = ring5(2 * ny - 1 - m) * RW;
          for (int rc = t; rc < RW; rc += NC) {
            const int xw = wrapx(x0 - 2 + rc, nx);
            cring[ridx + rc] = cring[sidx + rc];
            pring[ridx + rc] = pring[sidx + rc];
            Tring[ridx + rc] = ghost_T<S>(I, xw, false, Tring[sidx + rc]);
          }
        }
      }
      __syncthreads();
      if (s_abort) break;

      // ---- unit normal of row r + 1 at normal-ring columns t+1 (+ halo)
      const int mn = r + 1;
      if (mn >= ya - 1 && mn <= yb) {
        const C* cs = cring + ring5(mn - 1) * RW;
        const C* c0 = cring + ring5(mn) * RW;
        const C* cn = cring + ring5(mn + 1) * RW;
        const int nidx = ring3(mn) * QW;
        normal3(cs, c0, cn, t + 2, en2, nxr[nidx + t + 1], nyr[nidx + t + 1]);
        if (t == 0) normal3(cs, c0, cn, 1, en2, nxr[nidx], nyr[nidx]);
        if (t == NC - 1) normal3(cs, c0, cn, NC + 2, en2, nxr[nidx + NC + 1], nyr[nidx + NC + 1]);
      }
      __syncthreads();
      if (s_abort) break;

      // ---- collide row r at column x0 + t
      if (r >= ya && own_active) {
        const int col = t + XG;
        const char* s0 = slot_of(r);
        const char* sm = r > 0 ? slot_of(r - 1) : s0;
        const char* sp = r < ny - 1 ? slot_of(r + 1) : s0;
        C f[9], g[9], h[9];
        St::template spull9<0>(I, P, sm, s0, sp, col, r, x, f);
        St::template spull9<1>(I, P, sm, s0, sp, col, r, x, g);
        St::template spull9<2>(I, P, sm, s0, sp, col, r, x, h);
        const int rs5 = ring5(r - 1) * RW, r05 = ring5(r) * RW, rn5 = ring5(r + 1) * RW;
        const C* cs = cring + rs5;
        const C* c0 = cring + r05;
        const C* cn = cring + rn5;
        const C cc = c0[t + 2];
        const C pp = pring[r05 + t + 2], TT = Tring[r05 + t + 2];
        Stencils<C> st;
        grad3(cs, c0, cn, t + 2, st.gcx, st.gcy);
        st.lapc = lap3(cs, c0, cn, t + 2);
        grad3(Tring + rs5, Tring + r05, Tring + rn5, t + 2, st.gTx, st.gTy);
        if (dev_h<S>()) st.gTy += P.hr1;
        grad3(pring + rs5, pring + r05, pring + rn5, t + 2, st.gpx, st.gpy);
        const int ns = ring3(r - 1) * QW, n0 = ring3(r) * QW, nn = ring3(r + 1) * QW;
        C d1, d2, dum;
        grad3(nxr + ns, nxr + n0, nxr + nn, t + 1, d1, dum);
        grad3(nyr + ns, nyr + n0, nyr + nn, t + 1, dum, d2);
        st.kappa = d1 + d2;
        const Drive<S> d = drive<S>(P, r, f, cc, TT, st);
        C o[27];
        collide<S>(P, f, g, h, cc, pp, TT, st.gpx, st.gpy, d,
                   [&](int k, int i, C v) { o[k * 9 + i] = v; });
        const size_t e0 = (size_t)r * pitch + XG + x;
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
          for (int i = 0; i < 9; i++) S::st(I, dst, k, i, e0, o[k * 9 + i]);
        if (edge_ghost) {
          // periodic ghost copies of the first / last XG cells of the row
#pragma unroll
          for (int k = 0; k < 3; k++)
#pragma unroll
            for (int i = 0; i < 9; i++) {
              if (x < XG) S::st(I, dst, k, i, e0 + nx, o[k * 9 + i]);
              if (x >= nx - XG) S::st(I, dst, k, i, e0 - nx, o[k * 9 + i]);
            }
        }
      }
    }
    __syncthreads();
    if (s_abort) {
      // bounded wait for this CTA's copies still in flight, then stop
      if (t == 0)
        for (int q = waited + 1; q < next; q++)
          mbar_wait(smem_u32(&bars[(q - src_lo) % R]), ((q - src_lo) / R) & 1);
      __syncthreads();
      return;
    }
  }
}

}  // namespace lbe

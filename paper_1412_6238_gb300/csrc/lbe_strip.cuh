// The fused step as a column-strip marching kernel with TMA row staging.
//
// A work item is a strip of NC - 4 output columns [x0, x0 + NC - 4) and a
// segment of rows [ya, yb) of one instance.  One CTA of NC threads marches up
// the rows; thread t owns column x0 - 2 + t, so the two halo columns on each
// side that the stencils need are ordinary threads (no divergent halo work).
// The source rows (all population planes of row q, columns x0-3 .. x0+NC-2)
// are copied into a ring of R shared-memory slots by one TMA tiled load per
// row (cp.async.bulk.tensor, completion on an mbarrier per slot), issued
// R - 6 rows ahead of use.  Iteration i has two phases separated by a
// barrier:
//   phase 1, two independent pieces of work the compiler interleaves:
//     - every thread: moments c, p, T of row i+2 at its column (S1), pulled
//       from the staged rows i+1..i+3 (rows beyond a wall are ghosts: mirror
//       for c and p, 2 T_w - T for T) into rings of the last moment rows;
//     - threads 2..NC-3: stencils, force, velocity and the three collisions
//       of row i-1 (S2-S9, lbe_cell.cuh) from the staged rows i-2..i and the
//       rings, and the 27 stores (plus periodic ghost copies at row ends);
//   phase 2, threads 1..NC-2: unit normal of row i+1 (S2) into a ring.
// Every population is read from HBM once per step; moments and normals are
// computed once per strip column (4 halo columns overlap the neighbour).
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

// Staged row width (elements) of a strip kernel with nc threads: cells
// x0-3 .. x0+nc-2 from a start element rounded down to 16 bytes.
__host__ __device__ constexpr int strip_bw(int nc, int esz) {
  return ((nc + 2 + 16 / esz - 1) + 16 / esz - 1) / (16 / esz) * (16 / esz);
}

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
  static constexpr int NCO = NC - 4;                       // output columns
  static constexpr int A = 16 / (int)sizeof(E);            // TMA x alignment (elements)
  static constexpr int BW = strip_bw(NC, (int)sizeof(E));  // staged columns
  static constexpr int MAIN = F::planes * BW * (int)sizeof(E);
  static constexpr int G0OFF = (MAIN + 127) / 128 * 128;
  static constexpr int ROW_BYTES = MAIN + (F::g0 ? BW * 4 : 0);  // TMA bytes per row
  static constexpr int SLOT = (G0OFF + (F::g0 ? BW * 4 : 0) + 127) / 128 * 128;
  // rings of moment rows (c: 6, p and T: 5) and normal rows (4)
  static constexpr int CR = 6, PR = 5, NR = 4;
  static constexpr int SMEM = R * SLOT + (CR + 2 * PR) * NC * (int)sizeof(C) +
                              NR * NC * 2 * (int)sizeof(C) + R * 8 + 16;
  static_assert(R >= 7, "the ring holds rows i-2..i+3 plus at least one prefetched row");

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
  // rows y-1 (sm), y (s0), y+1 (sp); same rules as pull9 (lbe_tile.cuh).
  template <int K>
  __device__ static __forceinline__ void spull9(const InstDev& I, const Phys<C>& P, const char* sm,
                                                const char* s0, const char* sp, int col, int y,
                                                int ny, int xw, C out[9]) {
    constexpr bool DEV = (K == 2) && dev_h<S>();
    const bool wb = (y == 0), wt = (y == ny - 1);
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
  C* cring = reinterpret_cast<C*>(smem + R * St::SLOT);  // [CR][NC]
  C* pring = cring + St::CR * NC;                           // [PR][NC]
  C* Tring = pring + St::PR * NC;                           // [PR][NC]
  C* nxr = Tring + St::PR * NC;                             // [NR][NC]
  C* nyr = nxr + St::NR * NC;
  uint64_t* bars = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(nyr + St::NR * NC) + 15) & ~uintptr_t(15));
  __shared__ int s_abort;
  const int t = threadIdx.x;

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
    const int x0 = (int)(local % I.tiles_x) * St::NCO;
    const int ya = (int)(local / I.tiles_x) * seg_rows;
    const int yb = min(ya + seg_rows, ny);
    const int src_lo = max(ya - 3, 0), src_hi = min(yb + 2, ny - 1);
    // staged row: elements e0 .. e0+BW-1 (element XG + c holds cell c)
    const int e0 = (x0 + 1) / St::A * St::A;
    const int col = (x0 + 1 - e0) + 1 + t;  // staged column of this thread's cell
    char* __restrict__ dst = I.buf[parity ^ 1];
    const Phys<C> P = phys<C>(I);  // constants in registers for the whole item
    const C en2 = P.eta_n2;
    const size_t pitch = (size_t)I.pitch;
    const int x = x0 - 2 + t;
    const int xw = wrapx(x, nx);
    const bool collides = t >= 2 && t < NC - 2 && x < nx;
    const bool edge_ghost = collides && (x < XG || x >= nx - XG);

    __syncthreads();  // previous item fully done with the slots and barriers
    if (t == 0) {
      s_abort = 0;
      for (int s = 0; s < R; s++) mbar_init(smem_u32(&bars[s]), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    int next = src_lo;        // next source row to issue (thread 0)
    int waited = src_lo - 1;  // highest source row waited for
    auto issue_upto = [&](int lim) {
      if (t != 0) return;
      lim = min(lim, src_hi);
      for (; next <= lim; next++) {
        const int s = (next - src_lo) % R;
        const uint32_t bar = smem_u32(&bars[s]);
        const uint32_t dsts = smem_u32(slots + s * St::SLOT);
        mbar_expect_tx(bar, St::ROW_BYTES);
        tma_load_3d(dsts, map0, e0, next, 0, bar);
        if (RowFmt<S>::g0) tma_load_2d(dsts + St::G0OFF, map1, e0, next, bar);
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
    auto cr = [](int m) { return (((m % St::CR) + St::CR) % St::CR) * NC; };
    auto pr = [](int m) { return (((m % St::PR) + St::PR) % St::PR) * NC; };
    auto nr = [](int m) { return (m & (St::NR - 1)) * NC; };

    for (int i = ya - 4; i <= yb; i++) {
      __syncthreads();
      if (s_abort) break;
      // rows <= i-3 are done (the collision of row i-2 used rows i-3..i-1)
      issue_upto(max(i - 3, src_lo - 1) + R);

      // ---- phase 1a: moments of row m = i + 2 at this thread's column
      const int m = i + 2;
      if (m <= yb + 1) {
        const int ci = cr(m) + t, pi = pr(m) + t;
        if (m < ny) {
          const int mr = m >= 0 ? m : -1 - m;  // bottom ghost rows: the mirror row
          if (wait_upto(mr + 1)) {
            const char* s0 = slot_of(mr);
            const char* sm = mr > 0 ? slot_of(mr - 1) : s0;
            const char* sp = mr < ny - 1 ? slot_of(mr + 1) : s0;
            C v[9];
            St::template spull9<1>(I, P, sm, s0, sp, col, mr, ny, xw, v);
            {
              // the g_0 low part is read from the buffer (it is not staged)
              C clo_unused;
              const C g0lo = ld_g0lo(I, I.buf[parity], (size_t)mr * pitch + XG + xw);
              cring[ci] = moment_c(v, g0lo, clo_unused);
            }
            St::template spull9<0>(I, P, sm, s0, sp, col, mr, ny, xw, v);
            pring[pi] = sum9(v);
            St::template spull9<2>(I, P, sm, s0, sp, col, mr, ny, xw, v);
            C T = dv(sum9(v), P.rho_cv, P.inv_rho_cv);
            if (m < 0) T = ghost_T<S>(I, xw, true, T);
            Tring[pi] = T;
          }
        } else {
          // top ghost rows from the mirror rows still in the rings
          const int mm = 2 * ny - 1 - m;
          cring[ci] = cring[cr(mm) + t];
          pring[pi] = pring[pr(mm) + t];
          Tring[pi] = ghost_T<S>(I, xw, false, Tring[pr(mm) + t]);
        }
      }

      // ---- phase 1b: collide row r = i - 1
      const int r = i - 1;
      if (r >= ya && r < yb && collides) {
        const char* s0 = slot_of(r);
        const char* sm = r > 0 ? slot_of(r - 1) : s0;
        const char* sp = r < ny - 1 ? slot_of(r + 1) : s0;
        C f[9], g[9], h[9];
        St::template spull9<0>(I, P, sm, s0, sp, col, r, ny, x, f);
        St::template spull9<1>(I, P, sm, s0, sp, col, r, ny, x, g);
        St::template spull9<2>(I, P, sm, s0, sp, col, r, ny, x, h);
        const C* cs = cring + cr(r - 1);
        const C* c0 = cring + cr(r);
        const C* cn = cring + cr(r + 1);
        const int ps = pr(r - 1), p0 = pr(r), pn = pr(r + 1);
        const C cc = c0[t];
        const C pp = pring[p0 + t], TT = Tring[p0 + t];
        Stencils<C> st;
        grad3(cs, c0, cn, t, st.gcx, st.gcy);
        st.lapc = lap3(cs, c0, cn, t);
        grad3(Tring + ps, Tring + p0, Tring + pn, t, st.gTx, st.gTy);
        if (dev_h<S>()) st.gTy += P.hr1;
        grad3(pring + ps, pring + p0, pring + pn, t, st.gpx, st.gpy);
        const int ns = nr(r - 1), n0 = nr(r), nn = nr(r + 1);
        C d1, d2, dum;
        grad3(nxr + ns, nxr + n0, nxr + nn, t, d1, dum);
        grad3(nyr + ns, nyr + n0, nyr + nn, t, dum, d2);
        st.kappa = d1 + d2;
        const Drive<S> d = drive<S>(P, r, f, cc, TT, st);
        C o[27];
        // two-float g_0 and c of this cell (the low part read from the buffer)
        const C g0lo = ld_g0lo(I, I.buf[parity], (size_t)r * pitch + XG + x);
        C clo;
        (void)moment_c(g, g0lo, clo);
        C lo_out = C(0);
        collide<S>(P, f, g, h, cc, pp, TT, st.gpx, st.gpy, d,
                   [&](int k, int ii, C v) { o[k * 9 + ii] = v; }, g0lo, clo, &lo_out);
        const size_t e = (size_t)r * pitch + XG + x;
        st_cell_g0lo(I, dst, (size_t)r * pitch, x, lo_out);
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
          for (int ii = 0; ii < 9; ii++) S::st(I, dst, k, ii, e, o[k * 9 + ii]);
        if (edge_ghost) {
          // periodic ghost copies of the first / last XG cells of the row
#pragma unroll
          for (int k = 0; k < 3; k++)
#pragma unroll
            for (int ii = 0; ii < 9; ii++) {
              if (x < XG) S::st(I, dst, k, ii, e + nx, o[k * 9 + ii]);
              if (x >= nx - XG) S::st(I, dst, k, ii, e - nx, o[k * 9 + ii]);
            }
        }
      }
      __syncthreads();
      if (s_abort) break;

      // ---- phase 2: unit normal of row i + 1
      const int mn = i + 1;
      if (mn >= ya - 1 && mn <= yb && t >= 1 && t < NC - 1) {
        const C* c0 = cring + cr(mn);
        const int ni = nr(mn) + t;
        normal3(cring + cr(mn - 1), c0, cring + cr(mn + 1), t, en2, nxr[ni], nyr[ni]);
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

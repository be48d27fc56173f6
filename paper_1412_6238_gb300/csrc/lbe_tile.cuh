// The fused step of the three coupled D2Q9 lattices, one CTA tile at a time
// (the general kernel: any grid size, every storage including FP64), and the
// field-export variant that shares its front half.
//
// Per tile of TX x TY cells, per time step:
//   S1  pull the 27 pre-collision populations of each cell from the previous
//       post-collision buffer, P_i(x) = P*_i(x - xi_i), with halfway
//       bounce-back (f, g) and anti-bounce-back (hbar) at the walls; moments
//       c = sum g_i (Eq. 28), p = sum f_i (Eq. 13), T = sum hbar_i/(rho c_v)
//       (Eq. aEq13).  The same moments are recomputed on a ring of 2 cells
//       (c) / 1 cell (p, T) around the tile into shared memory; rows beyond
//       the walls are ghosts (c, p mirrored; T antisymmetric about T_w).
//   S2  isotropic D2Q9 stencils from shared memory: grad c, lap c, grad T,
//       grad p; n = grad c / sqrt(|grad c|^2 + eta_n^2) on a ring of 1;
//       kappa = div n (Eq. 3).
//   S3-S9  properties, mu, force, velocity and the three collisions
//       (lbe_cell.cuh).
//   S10 store the 27 post-collision values at the cell (the pull of the next
//       step streams them).
// At uniform density the grad(rho c_s^2) terms of Eq. 12, Eq. 13 and Fbar
// vanish; with a density varying with c (FP64 storage) p is corrected by
// (dt/2) u.grad(rho c_s^2) in a pass of its own (MODE 2), since the
// gradient of p needs the correction at the neighbours too.
#pragma once

#include "lbe_cell.cuh"

namespace lbe {

template <class S>
struct Cell {
  int x, xm, xp, y;  // wrapped column, its neighbours, row (0 <= y < ny)
};

// Pull the 9 pre-collision populations of lattice K at (x, y) from global
// memory.  For hbar in deviation form the result is relative to T_r of row
// y: a value pulled from row y - xi_iy was stored relative to
// T_r(y - xi_iy), which differs by w_i rho c_v hr1 xi_iy; at a wall the
// anti-bounce-back reads -P*_ibar + 2 w_i rho c_v (T_w - T_r(y)).
template <class S>
__device__ __forceinline__ typename S::C wall_T(const InstDev& I, int x, int which) {
  // which: 0 bottom row, 1 top row (for the anti-bounce-back), 2 bottom wall,
  // 3 top wall (for the ghost rows); deviation forms read T_w - T_r there
  if constexpr (dev_h<S>()) {
    return I.wdev[which][x];
  } else {
    return (which == 0 || which == 2) ? I.Tbot[x] : I.Ttop[x];
  }
}

// RAW: in an interior row, the hbar deviations as stored (relative to their
// source rows' T_r), for the moment T' (whose offsets cancel) and for
// collide() with dhc = dh.
// rho_cell: the cell's density (of its pulled c) for hbar's anti-bounce-back
// with a varying density; ignored at uniform density.
template <class S, int K, bool RAW = false>
__device__ __forceinline__ void pull9(const InstDev& I, const Phys<typename S::C>& P,
                                      const char* __restrict__ src, const Cell<S>& q,
                                      typename S::C out[9], typename S::C rho_cell = 0) {
  using C = typename S::C;
  const size_t pitch = (size_t)I.pitch;
  const size_t r0 = (size_t)q.y * pitch + XG;
  const bool wb = (q.y == 0), wt = (q.y == I.ny - 1);
  const bool DEV = (K == 2) && dev_h<S>() && (!RAW || wb || wt);
  C Tw = C(0);
  if (K == 2 && (wb || wt)) Tw = wall_T<S>(I, q.x, wb ? 0 : 1);
  const C dh = DEV ? P.dh : C(0);  // rho c_v (T_r(y) - T_r(y-1))
  auto bb = [&](int i) -> C {
    C v = S::ld(I, P, src, K, OPP(i), r0 + q.x);
    if (K == 2) {
      // the wall temperature where the link crosses the wall (x - xi_x/2,
      // between the columns) when P.wmid, else at the cell's column
      C Twi = Tw;
      if (P.wmid != C(0) && EX(i) != 0) {
        int xs = q.x - EX(i);
        xs = xs < 0 ? xs + I.nx : (xs >= I.nx ? xs - I.nx : xs);
        Twi = C(0.5) * (Tw + wall_T<S>(I, xs, wb ? 0 : 1));
      }
      return -v + C(2) * WGT<C>(i) * (P.drho != C(0) ? rho_cell : P.rho) * P.cv * Twi;
    }
    return v;
  };
  out[0] = S::ld(I, P, src, K, 0, r0 + q.x);
  out[1] = S::ld(I, P, src, K, 1, r0 + q.xm);
  out[3] = S::ld(I, P, src, K, 3, r0 + q.xp);
  if (wb) {
    out[2] = bb(2);
    out[5] = bb(5);
    out[6] = bb(6);
  } else {
    const size_t rm = r0 - pitch;
    out[2] = S::ld(I, P, src, K, 2, rm + q.x);
    out[5] = S::ld(I, P, src, K, 5, rm + q.xm);
    out[6] = S::ld(I, P, src, K, 6, rm + q.xp);
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
    const size_t rp = r0 + pitch;
    out[4] = S::ld(I, P, src, K, 4, rp + q.x);
    out[7] = S::ld(I, P, src, K, 7, rp + q.xp);
    out[8] = S::ld(I, P, src, K, 8, rp + q.xm);
    if (DEV) {
      out[4] += WGT<C>(4) * dh;
      out[7] += WGT<C>(7) * dh;
      out[8] += WGT<C>(8) * dh;
    }
  }
}

__device__ __forceinline__ int wrapx(int gx, int nx) {
  int x = gx % nx;
  return x < 0 ? x + nx : x;
}

template <class S>
__device__ __forceinline__ Cell<S> make_cell(int x, int y, int nx) {
  Cell<S> q;
  q.x = x;
  q.xm = (x == 0) ? nx - 1 : x - 1;
  q.xp = (x == nx - 1) ? 0 : x + 1;
  q.y = y;
  return q;
}

// Ghost temperature beyond a wall: T(-1-j) = 2 T_w - T(j); in deviation form
// (T_r linear) T'(-1-j) = 2 (T_w - T_r(wall)) - T'(j) with T_r(wall) at
// y = -1/2 or y = ny - 1/2.
template <class S>
__device__ __forceinline__ typename S::C ghost_T(const InstDev& I, int x, bool bottom,
                                                 typename S::C T) {
  using C = typename S::C;
  return C(2) * wall_T<S>(I, x, bottom ? 2 : 3) - T;
}

// c, p, T at an arbitrary tile-region position: x wraps, rows beyond the
// walls (gy in [-2, -1] or [ny, ny+1]) are ghosts.
template <class S>
__device__ __forceinline__ void region_values(const InstDev& I, const Phys<typename S::C>& P,
                                              const char* __restrict__ src, int gx, int gy,
                                              bool need_pT, bool use_pcorr,
                                              typename S::C& c, typename S::C& p,
                                              typename S::C& T) {
  using C = typename S::C;
  const int nx = I.nx, ny = I.ny;
  int ghost = 0, y = gy;
  if (y < 0) {
    y = -1 - y;
    ghost = -1;
  } else if (y >= ny) {
    y = 2 * ny - 1 - y;
    ghost = 1;
  }
  const Cell<S> q = make_cell<S>(wrapx(gx, nx), y, nx);
  C v[9];
  pull9<S, 1>(I, P, src, q, v);
  const C cm = sum9(v);  // c of the cell (of the mirror cell for a ghost row)
  // ghost rows of c: the mirror, plus the wetting flux at a wetting wall
  c = ghost != 0 ? wet_ghost(P, cm, ghost < 0 ? y : ny - 1 - y) : cm;
  if (need_pT) {
    const C rc = rho_at(P, cm);
    pull9<S, 0>(I, P, src, q, v);
    // p of Eq. 13: with a varying density, the corrected p of pcorr
    p = (use_pcorr && P.drho != C(0)) ? (C)I.pcorr[(size_t)y * nx + q.x] : sum9(v);
    pull9<S, 2, true>(I, P, src, q, v, rc);
    T = P.drho != C(0) ? dv(sum9(v), rc * P.cv, C(1)) : dv(sum9(v), P.rho_cv, P.inv_rho_cv);
    if (ghost != 0) T = ghost_T<S>(I, q.x, ghost < 0, T);
  } else {
    p = C(0);
    T = C(0);
  }
}

// Tile work.  MODE 0: full step (collide and store into the other buffer).
// MODE 1: export c, p, ux, uy, T of the current state into out[5][ny][nx].
// MODE 2 (varying density): the corrected p of Eq. 13 of every cell into
// I.pcorr, which MODE 0 then reads for p and its gradient.
template <class S, int TX, int TY, int MODE>
struct Tile {
  using C = typename S::C;
  static constexpr int NT = TX * TY;
  static constexpr int RW = TX + 4, RH = TY + 4;  // c region (ring of 2)
  static constexpr int QW = TX + 2, QH = TY + 2;  // p, T, n region (ring of 1)
  static constexpr int RING = RW * RH - TX * TY;

  struct Smem {
    C c[RH * RW];
    C p[QH * QW];
    C T[QH * QW];
    C nx[QH * QW];
    C ny[QH * QW];
  };

  __device__ static void run(const InstDev& I, int64_t tile, int parity, Smem& sm,
                             double* __restrict__ out, uint32_t step) {
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int nx = I.nx, ny = I.ny;
    const int x0 = (int)(tile % I.tiles_x) * TX;
    const int y0 = (int)(tile / I.tiles_x) * TY;
    const char* __restrict__ src = I.buf[parity];
    const Phys<C> P = phys<C>(I);  // constants in registers for the whole tile
    // the pre-pass has nothing to do for an instance without a varying
    // density (pcorr) or the dissipation term (uvel); the whole CTA leaves
    // together
    const bool wants_p = P.drho != C(0) && I.pcorr != nullptr;
    if (MODE == 2 && !wants_p && I.uvel == nullptr) return;

    // ---- S1: own cell
    const int gx = x0 + tx, gy = y0 + ty;
    const bool active = (gx < nx) && (gy < ny);
    C f[9], g[9], h[9];
    C cc = C(0), pp = C(0), TT = C(0);
    C g0lo = C(0), clo = C(0);  // low parts of g_0 and c (16/32-bit forms)
    Cell<S> q = make_cell<S>(active ? gx : 0, active ? gy : 0, nx);
    if (active) {
      pull9<S, 0>(I, P, src, q, f);
      pull9<S, 1>(I, P, src, q, g);
      if constexpr (S::kind != ST_F64) {
        g0lo = ld_g0lo<S>(I, src, (size_t)gy * I.pitch + XG + gx);
        cc = moment_c(g, g0lo, clo);
      } else {
        cc = sum9(g);
      }
      const C rc = rho_at(P, cc);
      pull9<S, 2, true>(I, P, src, q, h, rc);
      // p of Eq. 13 (with a varying density the corrected p, MODE 2 / pcorr)
      pp = (P.drho != C(0) && MODE == 0) ? (C)I.pcorr[(size_t)gy * nx + gx] : sum9(f);
      TT = P.drho != C(0) ? dv(sum9(h), rc * P.cv, C(1)) : dv(sum9(h), P.rho_cv, P.inv_rho_cv);
    } else if (gy <= ny + 1) {
      region_values<S>(I, P, src, gx, gy, true, MODE == 0, cc, pp, TT);
    }
    sm.c[(ty + 2) * RW + tx + 2] = cc;
    sm.p[(ty + 1) * QW + tx + 1] = pp;
    sm.T[(ty + 1) * QW + tx + 1] = TT;

    // ---- S1: ring around the tile (2 rows above/below, 2 columns left/right)
    for (int r = tid; r < RING; r += NT) {
      int rx, ry;
      if (r < 2 * RW) {
        ry = r / RW;
        rx = r % RW;
      } else if (r < 4 * RW) {
        ry = TY + 2 + (r - 2 * RW) / RW;
        rx = (r - 2 * RW) % RW;
      } else {
        const int s = r - 4 * RW;  // 4 columns x TY rows
        ry = 2 + s / 4;
        const int col = s % 4;
        rx = col < 2 ? col : TX + col;
      }
      const int hx = x0 - 2 + rx, hy = y0 - 2 + ry;
      const bool inner = rx >= 1 && rx <= TX + 2 && ry >= 1 && ry <= TY + 2;
      C vc = C(0), vp = C(0), vT = C(0);
      if (hy >= -2 && hy <= ny + 1)
        region_values<S>(I, P, src, hx, hy, inner, MODE == 0, vc, vp, vT);
      sm.c[ry * RW + rx] = vc;
      if (inner) {
        sm.p[(ry - 1) * QW + rx - 1] = vp;
        sm.T[(ry - 1) * QW + rx - 1] = vT;
      }
    }
    __syncthreads();

    // ---- S2: unit normal on the (TX+2) x (TY+2) region
    const C en2 = P.eta_n2;
    for (int r = tid; r < QW * QH; r += NT) {
      const int qx = r % QW, qy = r / QW;
      const C* c0 = sm.c + (qy + 1) * RW;
      normal3(c0 - RW, c0, c0 + RW, qx + 1, en2, sm.nx[r], sm.ny[r]);
    }
    __syncthreads();

    if (active) {
      Stencils<C> st;
      C d1, d2, dum;
      const C* c0 = sm.c + (ty + 2) * RW;
      grad3(c0 - RW, c0, c0 + RW, tx + 2, st.gcx, st.gcy);
      st.lapc = lap3(c0 - RW, c0, c0 + RW, tx + 2);
      const int qo = (ty + 1) * QW;
      grad3(sm.T + qo - QW, sm.T + qo, sm.T + qo + QW, tx + 1, st.gTx, st.gTy);
      // deviation form: grad T = grad T' + (0, hr1) (exact for the linear T_r)
      if (dev_h<S>()) st.gTy += P.hr1;
      grad3(sm.p + qo - QW, sm.p + qo, sm.p + qo + QW, tx + 1, st.gpx, st.gpy);
      grad3(sm.nx + qo - QW, sm.nx + qo, sm.nx + qo + QW, tx + 1, d1, dum);
      grad3(sm.ny + qo - QW, sm.ny + qo, sm.ny + qo + QW, tx + 1, dum, d2);
      st.kappa = d1 + d2;
      const Drive<S> d = drive<S>(P, gy, f, cc, TT, st);

      // Eq. 13 with a varying density: p = sum f_i + (dt/2) u.grad(rho c_s^2)
      const C pcor = P.drho != C(0) ? pp + C(0.5) * (d.ux * d.dRx + d.uy * d.dRy) : pp;
      if (MODE == 2) {  // the corrected p and u for the step that follows
        const size_t k = (size_t)gy * nx + gx;
        if (wants_p) I.pcorr[k] = (double)pcor;
        if (I.uvel) {
          I.uvel[k] = (double)d.ux;
          I.uvel[(size_t)nx * ny + k] = (double)d.uy;
        }
        return;
      }
      if (MODE == 1) {
        const size_t N = (size_t)nx * ny, k = (size_t)gy * nx + gx;
        out[k] = (double)cc + (double)clo;
        out[N + k] = (double)pcor;
        out[2 * N + k] = (double)d.ux;
        out[3 * N + k] = (double)d.uy;
        out[4 * N + k] = dev_h<S>() ? (double)TT + (I.hr0 + I.hr1 * gy) : (double)TT;
        return;
      }

      char* __restrict__ dst = I.buf[parity ^ 1];
      const size_t rowbase = (size_t)gy * I.pitch;
      C lo_out = C(0);
      // 16-bit forms: the cell's random bits for the stochastic rounding
      const uint32_t hc =
          S::SR ? sr_cell(sr_step_key(step, I.salt), (uint32_t)gy * (uint32_t)nx + (uint32_t)gx)
                : 0u;
      C gs = C(0);  // 16-bit forms: the stored moving g_i
      // the dissipation term: velocity gradients from the pre-pass's u
      // (isotropic stencil in index order; no slip: the ghost rows hold
      // minus the mirror cell's u)
      C du[4] = {C(0), C(0), C(0), C(0)};
      if (I.uvel != nullptr) {
        const size_t N = (size_t)nx * ny;
        C s0 = C(0), s1 = C(0), s2 = C(0), s3 = C(0);
        for (int i = 1; i < 9; i++) {
          int xx = gx + EX(i), yy = gy + EY(i);
          xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
          C sg = C(1);
          if (yy < 0) {
            yy = -1 - yy;
            sg = C(-1);
          } else if (yy >= ny) {
            yy = 2 * ny - 1 - yy;
            sg = C(-1);
          }
          const size_t kk = (size_t)yy * nx + xx;
          const C vx = sg * (C)I.uvel[kk], vy = sg * (C)I.uvel[N + kk];
          s0 += WGT<C>(i) * C(EX(i)) * vx;
          s1 += WGT<C>(i) * C(EY(i)) * vx;
          s2 += WGT<C>(i) * C(EX(i)) * vy;
          s3 += WGT<C>(i) * C(EY(i)) * vy;
        }
        du[0] = dv(s0, cs2<C>(), C(3));
        du[1] = dv(s1, cs2<C>(), C(3));
        du[2] = dv(s2, cs2<C>(), C(3));
        du[3] = dv(s3, cs2<C>(), C(3));
      }
      collide<S>(P, f, g, h, cc, pp, TT, st.gpx, st.gpy, d,
                 [&](int k, int i, C v) {
                   if constexpr (S::SR) {
                     v = S::sr_value(I, k, i, v, hc);
                     if (k == 1 && i > 0) gs += v;
                   }
                   st_cell<S>(I, dst, k, i, rowbase, gx, v);
                 },
                 g0lo, clo, &lo_out, (gy > 0 && gy < ny - 1) ? P.dh : C(0),
                 I.uvel != nullptr ? du : nullptr);
      if constexpr (S::SR) {
        // g_0 as c minus the stored g_i (as the strip kernel stores it)
        float g0h, g0l;
        g0_remainder(cc, clo, gs, g0h, g0l);
        st_cell<S>(I, dst, 1, 0, rowbase, gx, g0h);
        lo_out = g0l;
      }
      if constexpr (S::kind != ST_F64) st_cell_g0lo<S>(I, dst, rowbase, gx, (float)lo_out);
    }
  }
};

// Persistent kernel over a tile list spanning one or more instances.
template <class S, int TX, int TY, int MODE>
__global__ void __launch_bounds__(TX * TY, (S::kind == ST_F64 || TX * TY >= 512) ? 1 : 2)
tile_kernel(const InstDev* __restrict__ insts, int n_inst, int64_t total_tiles, int parity,
            double* __restrict__ out, const uint32_t* __restrict__ seed) {
  using T = Tile<S, TX, TY, MODE>;
  __shared__ typename T::Smem sm;
  // the step counter of the handle (random bits of the stochastic rounding)
  const uint32_t step = (S::SR && MODE == 0) ? __ldg(seed) : 0u;
  for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (insts[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    const InstDev& I = insts[lo];
    T::run(I, t - I.tile_begin, parity, sm, out, step);
    __syncthreads();
  }
}

}  // namespace lbe

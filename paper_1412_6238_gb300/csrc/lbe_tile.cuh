// The fused step of the three coupled D2Q9 lattices (one CTA tile at a time)
// and the field-export variant that shares its front half.
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
//   S3  eta(c), lambda(c) linear in c; tau_f = eta/(rho c_s^2) + 1/2;
//       tau_h = lambda/(rho c_v c_s^2), omega_T = 2/(2 tau_h + 1) (Eq. aEq12,
//       Eq. aEq14); sigma(T) = sigma0 - sigmaT (T - Tref) (Eq. aEq3).
//   S4  mu = 2 beta c (c-1)(2c-1) - eps^2 lap c (Sec. II, Eq. 16).
//   S5  F = eps alpha [-sigma kappa |grad c| grad c
//                      - sigmaT (|grad c|^2 grad T - (grad c.grad T) grad c)] + rho a
//       (Eq. 3: delta = eps alpha |grad c|^2, n = grad c/|grad c|).
//   S6  u = sum xi_i f_i/(rho c_s^2) + F/(2 rho) (Eq. 13).
//   S7  f: BGK + (1 - omega_f/2) F.(xi_i - u) Gamma_i(u) (Eq. 12, Eq. 5, Eq. 6).
//   S8  g: BGK to g_eq of Eq. 21-22 + (1 - omega_g/2) c (xi_i - u).(F - grad p)
//       Gamma_i(u)/(rho c_s^2) (Eq. 27).
//   S9  hbar: BGK to h_eq = rho c_v T Gamma_i(u) + (1 - omega_T/2)
//       Fbar.(xi_i - u) h_eq/(rho c_s^2), Fbar = F - grad p (Eq. aEq12).
//   S10 store the 27 post-collision values at the cell (the pull of the next
//       step streams them).
// Density is uniform, so the grad(rho c_s^2) terms of Eq. 12, Eq. 13 and Fbar
// vanish.
#pragma once

#include "lbe_common.cuh"

namespace lbe {

template <class S>
struct Cell {
  using C = typename S::C;
  int x, xm, xp, y;  // wrapped column, its neighbours, row (0 <= y < ny)
};

// hbar is handled as the deviation hbar_i - w_i rho c_v T_r(y) from the linear
// conduction profile T_r(y) = hr0 + hr1 y in every storage but FP64 (which
// keeps the full populations, like the FP64 reference).
template <class S>
__device__ __forceinline__ constexpr bool dev_h() { return S::kind != ST_F64; }

// Pull the 9 pre-collision populations of lattice K at (x, y).  For hbar in
// deviation form the result is relative to T_r of row y: a value pulled from
// row y - xi_iy was stored relative to T_r(y - xi_iy), which differs by
// w_i rho c_v hr1 xi_iy; at a wall the anti-bounce-back reads
// -P*_ibar + 2 w_i rho c_v (T_w - T_r(y)).
template <class S, int K>
__device__ __forceinline__ void pull9(const InstDev& I, const char* __restrict__ src,
                                      const Cell<S>& q, typename S::C out[9]) {
  using C = typename S::C;
  constexpr bool DEV = (K == 2) && dev_h<S>();
  const size_t pitch = (size_t)I.pitch;
  const size_t r0 = (size_t)q.y * pitch;
  const bool wb = (q.y == 0), wt = (q.y == I.ny - 1);
  C Tw = C(0);
  if (K == 2 && (wb || wt)) {
    const double tw = wb ? I.Tbot[q.x] : I.Ttop[q.x];
    Tw = DEV ? C(tw - (I.hr0 + I.hr1 * q.y)) : C(tw);
  }
  const C dh = DEV ? C(I.rho_cv * I.hr1) : C(0);  // rho c_v (T_r(y) - T_r(y-1))
  auto bb = [&](int i) -> C {
    C v = S::ld(I, src, K, OPP(i), r0 + q.x);
    if (K == 2) return -v + C(2) * WGT<C>(i) * C(I.rho) * C(I.cv) * Tw;
    return v;
  };
  out[0] = S::ld(I, src, K, 0, r0 + q.x);
  out[1] = S::ld(I, src, K, 1, r0 + q.xm);
  out[3] = S::ld(I, src, K, 3, r0 + q.xp);
  if (wb) {
    out[2] = bb(2);
    out[5] = bb(5);
    out[6] = bb(6);
  } else {
    const size_t rm = r0 - pitch;
    out[2] = S::ld(I, src, K, 2, rm + q.x);
    out[5] = S::ld(I, src, K, 5, rm + q.xm);
    out[6] = S::ld(I, src, K, 6, rm + q.xp);
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
    out[4] = S::ld(I, src, K, 4, rp + q.x);
    out[7] = S::ld(I, src, K, 7, rp + q.xp);
    out[8] = S::ld(I, src, K, 8, rp + q.xm);
    if (DEV) {
      out[4] += WGT<C>(4) * dh;
      out[7] += WGT<C>(7) * dh;
      out[8] += WGT<C>(8) * dh;
    }
  }
}

// Sum over i = 0..8 in index order (the order the moments of Eq. 13, Eq. 28
// and Eq. aEq13 are accumulated in FP64 parity mode as well).
template <class C>
__device__ __forceinline__ C sum9(const C v[9]) {
  C s = v[0];
#pragma unroll
  for (int i = 1; i < 9; i++) s += v[i];
  return s;
}

// a / b: a true division in FP64 (parity mode rounds like the FP64
// reference); a product with the precomputed reciprocal in FP32.
__device__ __forceinline__ double dv(double a, double b, double) { return a / b; }
__device__ __forceinline__ float dv(float a, float, float inv_b) { return a * inv_b; }

// c_s^2 = 1/3 of D2Q9
template <class C>
__device__ __forceinline__ C cs2() { return C(1.0 / 3.0); }

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

// c, p, T at an arbitrary tile-region position: x wraps, rows beyond the
// walls (gy in [-2, -1] or [ny, ny+1]) are ghosts.
template <class S>
__device__ __forceinline__ void region_values(const InstDev& I, const char* __restrict__ src,
                                              int gx, int gy, bool need_pT,
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
  pull9<S, 1>(I, src, q, v);
  c = sum9(v);
  if (need_pT) {
    pull9<S, 0>(I, src, q, v);
    p = sum9(v);
    pull9<S, 2>(I, src, q, v);
    T = dv(sum9(v), C(I.rho_cv), C(I.inv_rho_cv));
    if (ghost != 0) {
      // T(-1-j) = 2 T_w - T(j); in deviation form T_r is linear, so
      // T'(-1-j) = 2 (T_w - T_r(wall)) - T'(j), T_r(wall) = T_r(-1/2) or T_r(ny-1/2)
      const double tw = ghost < 0 ? I.Tbot[q.x] : I.Ttop[q.x];
      const C Tw = dev_h<S>() ? C(tw - (I.hr0 + I.hr1 * (ghost < 0 ? -0.5 : ny - 0.5)))
                              : C(tw);
      T = C(2) * Tw - T;
    }
  } else {
    p = C(0);
    T = C(0);
  }
}

// Isotropic gradient (1/c_s^2) sum_{i>=1} w_i xi_i phi(x + xi_i) and Laplacian
// (2/c_s^2) sum_{i>=1} w_i (phi(x + xi_i) - phi(x)) of a shared-memory array
// of row width WD at (rx, ry); the terms are summed in index order
// i = 1 (E), 2 (N), 3 (W), 4 (S), 5 (NE), 6 (NW), 7 (SW), 8 (SE), terms with
// xi_ia = 0 being exact zeros.
template <class C, int WD>
__device__ __forceinline__ void grad_iso(const C* s, int rx, int ry, C& gx, C& gy) {
  const C* r0 = s + ry * WD + rx;
  const C vE = r0[1], vW = r0[-1], vN = r0[WD], vS = r0[-WD];
  const C vNE = r0[WD + 1], vNW = r0[WD - 1], vSE = r0[-WD + 1], vSW = r0[-WD - 1];
  const C wa = WGT<C>(1), wd = WGT<C>(5);
  C sx = wa * vE;
  sx = sx - wa * vW;
  sx = sx + wd * vNE;
  sx = sx - wd * vNW;
  sx = sx - wd * vSW;
  sx = sx + wd * vSE;
  C sy = wa * vN;
  sy = sy - wa * vS;
  sy = sy + wd * vNE;
  sy = sy + wd * vNW;
  sy = sy - wd * vSW;
  sy = sy - wd * vSE;
  gx = dv(sx, cs2<C>(), C(3));
  gy = dv(sy, cs2<C>(), C(3));
}
template <class C, int WD>
__device__ __forceinline__ C lap_iso(const C* s, int rx, int ry) {
  const C* r0 = s + ry * WD + rx;
  const C v0 = r0[0];
  const C wa = WGT<C>(1), wd = WGT<C>(5);
  C t = wa * (r0[1] - v0);
  t = t + wa * (r0[WD] - v0);
  t = t + wa * (r0[-1] - v0);
  t = t + wa * (r0[-WD] - v0);
  t = t + wd * (r0[WD + 1] - v0);
  t = t + wd * (r0[WD - 1] - v0);
  t = t + wd * (r0[-WD - 1] - v0);
  t = t + wd * (r0[-WD + 1] - v0);
  return dv(C(2) * t, cs2<C>(), C(3));
}

// Tile work.  MODE 0: full step (collide and store into the other buffer).
// MODE 1: export c, p, ux, uy, T of the current state into out[5][ny][nx].
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
                             double* __restrict__ out) {
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int nx = I.nx, ny = I.ny;
    const int x0 = (int)(tile % I.tiles_x) * TX;
    const int y0 = (int)(tile / I.tiles_x) * TY;
    const char* __restrict__ src = I.buf[parity];

    // ---- S1: own cell
    const int gx = x0 + tx, gy = y0 + ty;
    const bool active = (gx < nx) && (gy < ny);
    C f[9], g[9], h[9];
    C cc = C(0), pp = C(0), TT = C(0);
    Cell<S> q = make_cell<S>(active ? gx : 0, active ? gy : 0, nx);
    if (active) {
      pull9<S, 0>(I, src, q, f);
      pull9<S, 1>(I, src, q, g);
      pull9<S, 2>(I, src, q, h);
      cc = sum9(g);
      pp = sum9(f);
      TT = dv(sum9(h), C(I.rho_cv), C(I.inv_rho_cv));
    } else if (gy <= ny + 1) {
      region_values<S>(I, src, gx, gy, true, cc, pp, TT);
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
      if (hy >= -2 && hy <= ny + 1) region_values<S>(I, src, hx, hy, inner, vc, vp, vT);
      sm.c[ry * RW + rx] = vc;
      if (inner) {
        sm.p[(ry - 1) * QW + rx - 1] = vp;
        sm.T[(ry - 1) * QW + rx - 1] = vT;
      }
    }
    __syncthreads();

    // ---- S2: unit normal on the (TX+2) x (TY+2) region
    const C en2 = C(I.eta_n2);
    for (int r = tid; r < QW * QH; r += NT) {
      const int qx = r % QW, qy = r / QW;
      C gxv, gyv;
      grad_iso<C, RW>(sm.c, qx + 1, qy + 1, gxv, gyv);
      const C inv = C(1) / sqrt(gxv * gxv + gyv * gyv + en2);
      sm.nx[r] = gxv * inv;
      sm.ny[r] = gyv * inv;
    }
    __syncthreads();

    if (active) {
      C gcx, gcy, gTx, gTy, gpx, gpy, d1, d2, dum;
      grad_iso<C, RW>(sm.c, tx + 2, ty + 2, gcx, gcy);
      const C lapc = lap_iso<C, RW>(sm.c, tx + 2, ty + 2);
      grad_iso<C, QW>(sm.T, tx + 1, ty + 1, gTx, gTy);
      // deviation form: T = T' + T_r(y), grad T = grad T' + (0, hr1) (the
      // isotropic gradient of a linear profile is exact)
      const C Trow = dev_h<S>() ? C(I.hr0 + I.hr1 * gy) : C(0);
      if (dev_h<S>()) gTy += C(I.hr1);
      grad_iso<C, QW>(sm.p, tx + 1, ty + 1, gpx, gpy);
      grad_iso<C, QW>(sm.nx, tx + 1, ty + 1, d1, dum);
      grad_iso<C, QW>(sm.ny, tx + 1, ty + 1, dum, d2);
      const C kappa = d1 + d2;

      // S4, S5
      const C mu = C(I.beta2) * cc * (cc - C(1)) * (C(2) * cc - C(1)) - C(I.eps2) * lapc;
      const C sigma = dev_h<S>() ? C(I.sigma0) - C(I.sigmaT) * (TT + C(I.hr0 + I.hr1 * gy - I.Tref))
                                 : C(I.sigma0) - C(I.sigmaT) * (TT - C(I.Tref));
      const C g2 = gcx * gcx + gcy * gcy;
      const C gabs = sqrt(g2);
      const C cdT = gcx * gTx + gcy * gTy;
      const C ea = C(I.ea);
      const C cap = -sigma * kappa * ea * gabs;
      const C mar = -C(I.sigmaT) * ea;
      const C Fx = cap * gcx + mar * (g2 * gTx - cdT * gcx) + C(I.Fbx);
      const C Fy = cap * gcy + mar * (g2 * gTy - cdT * gcy) + C(I.Fby);

      // S6 (Eq. 13): first moments summed in index order
      const C f0 = f[0];
      (void)f0;
      C jx = f[1] - f[3];
      jx = jx + f[5];
      jx = jx - f[6];
      jx = jx - f[7];
      jx = jx + f[8];
      C jy = f[2] - f[4];
      jy = jy + f[5];
      jy = jy + f[6];
      jy = jy - f[7];
      jy = jy - f[8];
      const C rho = C(I.rho);
      const C inv_rho = C(I.inv_rho);
      const C rcs2 = C(I.rcs2);          // rho c_s^2
      const C inv_rcs2 = C(3) * inv_rho;
      const C ux = dv(jx, rcs2, inv_rcs2) + dv(C(0.5) * Fx, rho, inv_rho);
      const C uy = dv(jy, rcs2, inv_rcs2) + dv(C(0.5) * Fy, rho, inv_rho);

      if (MODE == 1) {
        const size_t N = (size_t)nx * ny, k = (size_t)gy * nx + gx;
        out[k] = (double)cc;
        out[N + k] = (double)pp;
        out[2 * N + k] = (double)ux;
        out[3 * N + k] = (double)uy;
        out[4 * N + k] = dev_h<S>() ? (double)TT + (I.hr0 + I.hr1 * gy) : (double)TT;
        return;
      }

      // S3: properties, linear in c
      const C eta = C(I.eta1) + cc * C(I.deta);
      const C lam = C(I.lam1) + cc * C(I.dlam);
      const C tau_f = dv(eta, rcs2, inv_rcs2) + C(0.5);
      const C omega_f = C(1) / tau_f;
      const C tau_h = dv(lam, C(I.rcvcs2), C(3) * C(I.inv_rho_cv));
      const C omega_T = C(2) / (C(2) * tau_h + C(1));
      const C omega_g = C(I.omega_g);
      const C af = C(1) - C(0.5) * omega_f;
      const C ag = C(1) - C(0.5) * omega_g;
      const C aT = C(1) - C(0.5) * omega_T;
      // Gamma_i(u) = w_i (1 + xi.u/c_s^2 + ((xi.u/c_s^2)^2 - u^2/c_s^2)/2) (Eq. 6)
      const C uu = dv(ux * ux + uy * uy, cs2<C>(), C(3));
      const C Gm = C(I.Gm);
      // H_i of Eq. 22
      const C Hi = dv(Gm * mu, cs2<C>(), C(3));
      const C H0 = dv(cc - dv((C(1) - WGT<C>(0)) * Gm * mu, cs2<C>(), C(3)), WGT<C>(0),
                      C(9) / C(4));
      const C Gx = Fx - gpx, Gy = Fy - gpy;  // F - grad p (= Fbar, uniform rho)
      const C rcvT = C(I.rho) * C(I.cv) * (TT + Trow);  // rho c_v T (full T)
      const C rcvTr = C(I.rho_cv) * Trow;                // rho c_v T_r(y)
      const C rcvTd = C(I.rho_cv) * TT;                  // rho c_v T'

      char* __restrict__ dst = I.buf[parity ^ 1];
      const size_t idx = (size_t)gy * I.pitch + gx;
#pragma unroll
      for (int i = 0; i < 9; i++) {
        const C W = WGT<C>(i);
        const C xu = dv(C(EX(i)) * ux + C(EY(i)) * uy, cs2<C>(), C(3));
        const C hq = C(0.5) * (xu * xu - uu);
        const C G = W * (C(1) + xu + hq);
        const C q = xu + hq;  // velocity part, without the cancelling w_i
        const C dx = C(EX(i)) - ux, dy = C(EY(i)) - uy;
        // f (Eq. 12 with Eq. 5)
        const C feq = W * (pp + rcs2 * q);
        const C fs = (Fx * dx + Fy * dy) * G;
        const C fn = f[i] - omega_f * (f[i] - feq) + af * fs;
        // g (Eq. 27 with Eq. 21-22)
        const C geq = W * ((i == 0 ? H0 : Hi) + cc * q);
        const C gs = dv(cc * (dx * Gx + dy * Gy), rcs2, inv_rcs2) * G;
        const C gn = g[i] - omega_g * (g[i] - geq) + ag * gs;
        // hbar (Eq. aEq12 with Eq. aEq9)
        const C heq = rcvT * G;
        const C hs = dv(Gx * dx + Gy * dy, rcs2, inv_rcs2) * heq;
        // deviation form: h_eq - w_i rho c_v T_r = rho c_v (T' Gamma_i + T_r w_i q_i)
        const C heqd = dev_h<S>() ? rcvTd * G + rcvTr * (W * q) : heq;
        const C hn = h[i] - omega_T * (h[i] - heqd) + aT * hs;
        S::st(I, dst, 0, i, idx, fn);
        S::st(I, dst, 1, i, idx, gn);
        S::st(I, dst, 2, i, idx, hn);
      }
    }
  }
};

// Persistent kernel over a tile list spanning one or more instances.
template <class S, int TX, int TY, int MODE>
__global__ void __launch_bounds__(TX * TY, (S::kind == ST_F64) ? 1 : 2)
tile_kernel(const InstDev* __restrict__ insts, int n_inst, int64_t total_tiles, int parity,
            double* __restrict__ out) {
  using T = Tile<S, TX, TY, MODE>;
  __shared__ typename T::Smem sm;
  for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (insts[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    const InstDev& I = insts[lo];
    T::run(I, t - I.tile_begin, parity, sm, out);
    __syncthreads();
  }
}

}  // namespace lbe

// Per-cell arithmetic of the fused step, shared by the tile kernel and the
// strip kernel: isotropic stencils, chemical potential, CSF + Marangoni force,
// velocity and the three forced BGK collisions (steps S2-S9).  Expressions are
// evaluated in the operation order of the FP64 CPU reference; divisions are
// true divisions in FP64 and products with a reciprocal in FP32 (dv()).
#pragma once

#include "lbe_common.cuh"

namespace lbe {

// a / b: a true division in FP64 (parity mode rounds like the FP64
// reference); a product with the precomputed reciprocal in FP32.
__device__ __forceinline__ double dv(double a, double b, double) { return a / b; }
__device__ __forceinline__ float dv(float a, float, float inv_b) { return a * inv_b; }

// c_s^2 = 1/3 of D2Q9
template <class C>
__device__ __forceinline__ C cs2() { return C(1.0 / 3.0); }

// Sum over i = 0..8: in index order in FP64 (the order of the FP64
// reference), as a pairwise tree in FP32 (shorter dependency chains).
__device__ __forceinline__ double sum9(const double v[9]) {
  double s = v[0];
#pragma unroll
  for (int i = 1; i < 9; i++) s += v[i];
  return s;
}
__device__ __forceinline__ float sum9(const float v[9]) {
  return (((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) + v[8];
}

// Error-free transformations for the two-float g_0 and c of the 16/32-bit
// forms: a + b = s + e exactly (Knuth's two-sum; the fast variant needs
// |a| >= |b|).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// c = sum g_i (Eq. 28) with g_0 = g[0] + g0lo, as hi + lo: the eight small
// moving populations are summed first, then added to g_0 exactly.
__device__ __forceinline__ float moment_c(const float g[9], float g0lo, float& clo) {
  const float s8 = ((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8]));
  float ch, e;
  two_sum(g[0], s8, ch, e);
  clo = e + g0lo;
  return ch;
}

// hbar is handled as the deviation hbar_i - w_i rho c_v T_r(y) from the linear
// conduction profile T_r(y) = hr0 + hr1 y in every storage but FP64 (which
// keeps the full populations, like the FP64 reference).
template <class S>
__device__ __forceinline__ constexpr bool dev_h() { return S::kind != ST_F64; }

// Isotropic gradient (1/c_s^2) sum_{i>=1} w_i xi_i phi(x + xi_i) and Laplacian
// (2/c_s^2) sum_{i>=1} w_i (phi(x + xi_i) - phi(x)) from three rows (south,
// centre, north) at column x.  FP64: the terms are summed in index order
// i = 1 (E), 2 (N), 3 (W), 4 (S), 5 (NE), 6 (NW), 7 (SW), 8 (SE), terms with
// xi_ia = 0 being exact zeros (the order of the FP64 reference).
template <class C>
__device__ __forceinline__ void grad3(const C* rs, const C* rc, const C* rn, int x, C& gx, C& gy) {
  const C vE = rc[x + 1], vW = rc[x - 1], vN = rn[x], vS = rs[x];
  const C vNE = rn[x + 1], vNW = rn[x - 1], vSE = rs[x + 1], vSW = rs[x - 1];
  const C wa = WGT<C>(1), wd = WGT<C>(5);
  if constexpr (sizeof(C) == 4) {
    // FP32: differences of opposite neighbours first (exact when they are
    // within a factor 2, Sterbenz), then the weights, so that a small
    // gradient of an O(1) field keeps its relative precision instead of
    // inheriting the rounding of the O(1) products w_i phi(x + xi_i)
    const C dEW = vE - vW, dNS = vN - vS;
    const C d1 = vNE - vSW, d2 = vSE - vNW;  // xi = (1, 1) and (1, -1)
    gx = dv(wa * dEW + wd * (d1 + d2), cs2<C>(), C(3));
    gy = dv(wa * dNS + wd * (d1 - d2), cs2<C>(), C(3));
  } else {
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
}

template <class C>
__device__ __forceinline__ C lap3(const C* rs, const C* rc, const C* rn, int x) {
  const C v0 = rc[x];
  const C wa = WGT<C>(1), wd = WGT<C>(5);
  C t = wa * (rc[x + 1] - v0);
  t = t + wa * (rn[x] - v0);
  t = t + wa * (rc[x - 1] - v0);
  t = t + wa * (rs[x] - v0);
  t = t + wd * (rn[x + 1] - v0);
  t = t + wd * (rn[x - 1] - v0);
  t = t + wd * (rs[x - 1] - v0);
  t = t + wd * (rs[x + 1] - v0);
  return dv(C(2) * t, cs2<C>(), C(3));
}

// Unit normal n = grad c / sqrt(|grad c|^2 + eta_n^2) (Eq. 3).
template <class C>
__device__ __forceinline__ void normal3(const C* rs, const C* rc, const C* rn, int x, C en2, C& nx,
                                        C& ny) {
  C gx, gy;
  grad3(rs, rc, rn, x, gx, gy);
  const C inv = C(1) / sqrt(gx * gx + gy * gy + en2);
  nx = gx * inv;
  ny = gy * inv;
}

// The same stencils for c = hi + lo (16/32-bit forms): hi rows in FP32, lo
// rows as FP16 of lo * 2^24; differences of hi and of lo are taken first.
__device__ __forceinline__ float lo_at(const __half* r, int x) {
  return __half2float(r[x]) * G0LO_INV;
}
__device__ __forceinline__ void grad3c(const float* rs, const float* rc, const float* rn,
                                       const __half* ls, const __half* lc, const __half* ln, int x,
                                       float& gx, float& gy) {
  const float wa = WGT<float>(1), wd = WGT<float>(5);
  const float dEW = (rc[x + 1] - rc[x - 1]) + (lo_at(lc, x + 1) - lo_at(lc, x - 1));
  const float dNS = (rn[x] - rs[x]) + (lo_at(ln, x) - lo_at(ls, x));
  const float d1 = (rn[x + 1] - rs[x - 1]) + (lo_at(ln, x + 1) - lo_at(ls, x - 1));
  const float d2 = (rs[x + 1] - rn[x - 1]) + (lo_at(ls, x + 1) - lo_at(ln, x - 1));
  gx = dv(wa * dEW + wd * (d1 + d2), cs2<float>(), 3.f);
  gy = dv(wa * dNS + wd * (d1 - d2), cs2<float>(), 3.f);
}
__device__ __forceinline__ float lap3c(const float* rs, const float* rc, const float* rn,
                                       const __half* ls, const __half* lc, const __half* ln,
                                       int x) {
  const float v0 = rc[x], l0 = lo_at(lc, x);
  const float wa = WGT<float>(1), wd = WGT<float>(5);
  auto d = [&](const float* r, const __half* l, int xx) { return (r[xx] - v0) + (lo_at(l, xx) - l0); };
  float t = wa * d(rc, lc, x + 1);
  t = t + wa * d(rn, ln, x);
  t = t + wa * d(rc, lc, x - 1);
  t = t + wa * d(rs, ls, x);
  t = t + wd * d(rn, ln, x + 1);
  t = t + wd * d(rn, ln, x - 1);
  t = t + wd * d(rs, ls, x - 1);
  t = t + wd * d(rs, ls, x + 1);
  return dv(2.f * t, cs2<float>(), 3.f);
}
__device__ __forceinline__ void normal3c(const float* rs, const float* rc, const float* rn,
                                         const __half* ls, const __half* lc, const __half* ln,
                                         int x, float en2, float& nx, float& ny) {
  float gx, gy;
  grad3c(rs, rc, rn, ls, lc, ln, x, gx, gy);
  const float inv = 1.f / sqrtf(gx * gx + gy * gy + en2);
  nx = gx * inv;
  ny = gy * inv;
}

// Stencil results at one cell.
template <class C>
struct Stencils {
  C gcx, gcy, lapc, gTx, gTy, gpx, gpy, kappa;
};

// Force, chemical potential and velocity (S4-S6).  TT is T, or T' = T - T_r(y)
// in the deviation forms (then gTy already includes dT_r/dy).
template <class S>
struct Drive {
  using C = typename S::C;
  C mu, Fx, Fy, ux, uy, Trow;
  // varying density (FP64): rho(c) and grad(rho c_s^2) = c_s^2 (rho2 - rho1)
  // grad c (the isotropic gradient of the interpolated density)
  C rho, dRx, dRy;
  // rho c_s^2 u = j + c_s^2 F / 2, the first moment the f equilibrium must
  // have (FP32 forms, which build its odd part from it), as two floats
  // J = Jx + Jxl; c_s^2 F / 2 is formed as (w_axis + 2 w_diag) F with the
  // weights of the forcing term, so that it is half the forcing term's first
  // moment in the FP32 constants
  C Jx, Jy, Jxl, Jyl;
};

template <class S>
__device__ __forceinline__ Drive<S> drive(const Phys<typename S::C>& P, int gy,
                                          const typename S::C f[9], typename S::C cc,
                                          typename S::C TT, const Stencils<typename S::C>& s) {
  using C = typename S::C;
  Drive<S> d;
  d.Trow = dev_h<S>() ? P.hr0 + P.hr1 * C(gy) : C(0);
  // S4: mu = 2 beta c (c-1)(2c-1) - eps^2 lap c
  d.mu = P.beta2 * cc * (cc - C(1)) * (C(2) * cc - C(1)) - P.eps2 * s.lapc;
  // S5: sigma(T) (Eq. aEq3) and F (Eq. 3)
  const C sigma = dev_h<S>() ? P.sigma0 - P.sigmaT * (TT + (d.Trow - P.Tref))
                             : P.sigma0 - P.sigmaT * (TT - P.Tref);
  const C g2 = s.gcx * s.gcx + s.gcy * s.gcy;
  const C gabs = sqrt(g2);
  const C cdT = s.gcx * s.gTx + s.gcy * s.gTy;
  const C ea = P.ea;
  const C cap = -sigma * s.kappa * ea * gabs;
  const C mar = -P.sigmaT * ea;
  // varying density (FP64 storage only): rho(c) in the body force, u, the
  // relaxation times, the equilibria and the sources
  const bool vr = sizeof(C) == 8 && P.drho != C(0);
  d.rho = vr ? rho_at(P, cc) : P.rho;
  d.dRx = vr ? (cs2<C>() * P.drho) * s.gcx : C(0);
  d.dRy = vr ? (cs2<C>() * P.drho) * s.gcy : C(0);
  d.Fx = cap * s.gcx + mar * (g2 * s.gTx - cdT * s.gcx) + (vr ? d.rho * P.ax : P.Fbx);
  d.Fy = cap * s.gcy + mar * (g2 * s.gTy - cdT * s.gcy) + (vr ? d.rho * P.ay : P.Fby);
  // S6 (Eq. 13): first moments.  FP64: summed in index order (the order of
  // the FP64 reference).  FP32: differences of opposite populations first,
  // each exact (Sterbenz: the two are within a factor 2 of each other), then
  // their sum, so that j is rounded at its own scale; summed in index order,
  // every partial sum is of the size of f and rounds at that scale, an error
  // that is large next to a small j (slow flow, where f is mostly w_i p) and
  // repeats step after step where the flow is steady.
  C jx, jy, jxl = C(0), jyl = C(0);
  if constexpr (sizeof(C) == 4) {
    // j exactly, as two floats: the three differences are exact, their sums
    // by error-free two-sums
    const C d13 = f[1] - f[3], d24 = f[2] - f[4], d57 = f[5] - f[7], d86 = f[8] - f[6];
    C sx, ex, sy, ey, e2;
    two_sum(d57, d86, sx, ex);
    two_sum(d13, sx, jx, e2);
    jxl = ex + e2;
    two_sum(d57, -d86, sy, ey);
    two_sum(d24, sy, jy, e2);
    jyl = ey + e2;
  } else {
    jx = f[1] - f[3];
    jx = jx + f[5];
    jx = jx - f[6];
    jx = jx - f[7];
    jx = jx + f[8];
    jy = f[2] - f[4];
    jy = jy + f[5];
    jy = jy + f[6];
    jy = jy - f[7];
    jy = jy - f[8];
  }
  const C rho = d.rho, inv_rho = P.inv_rho;
  const C rcs2 = vr ? d.rho * C(1.0 / 3.0) : P.rcs2, inv_rcs2 = C(3) * inv_rho;
  d.ux = dv(jx, rcs2, inv_rcs2) + dv(C(0.5) * d.Fx, rho, inv_rho);
  d.uy = dv(jy, rcs2, inv_rcs2) + dv(C(0.5) * d.Fy, rho, inv_rho);
  const C wa = WGT<C>(1), wd2 = C(2) * WGT<C>(5);
  if constexpr (sizeof(C) == 4) {
    // J = j + (w_axis + 2 w_diag) F as two floats (the force term, small
    // next to j where the momentum matters, is rounded at its own scale)
    const C cFx = fmaf(wa, d.Fx, wd2 * d.Fx), cFy = fmaf(wa, d.Fy, wd2 * d.Fy);
    C e;
    two_sum(jx, cFx, d.Jx, e);
    d.Jxl = e + jxl;
    two_sum(jy, cFy, d.Jy, e);
    d.Jyl = e + jyl;
  } else {
    d.Jx = (jx + wa * d.Fx) + wd2 * d.Fx;
    d.Jy = (jy + wa * d.Fy) + wd2 * d.Fy;
    d.Jxl = d.Jyl = C(0);
  }
  return d;
}

// S3, S7-S9: the three forced BGK collisions.  out(k, i, value) receives the
// post-collision value of population (k, i) (hbar as a deviation in the
// deviation forms).  16/32-bit forms: g_0 = g[0] + g0lo and c = cc + clo
// enter as two-float values and the post-collision g_0 leaves as
// out(1, 0, hi) and *g0lo_out = lo.  hbar (16/32-bit forms): h[] as pulled,
// without the change of reference row (from the source row's T_r to this
// row's) when dhc = rho c_v dT_r/dy, or already in this row's reference when
// dhc = 0 (the wall rows); the change, w_i xi_iy dhc, enters through the
// source term instead, (1 - omega_T) times (see below).
template <class S, class Out>
__device__ __forceinline__ void collide(const Phys<typename S::C>& P, const typename S::C f[9],
                                        const typename S::C g[9], const typename S::C h[9],
                                        typename S::C cc, typename S::C pp, typename S::C TT,
                                        typename S::C gpx, typename S::C gpy, const Drive<S>& d,
                                        Out&& out, typename S::C g0lo = 0, typename S::C clo = 0,
                                        typename S::C* g0lo_out = nullptr,
                                        typename S::C dhc = 0,
                                        const typename S::C* wdu = nullptr) {
  using C = typename S::C;
  const bool vr = sizeof(C) == 8 && P.drho != C(0);  // varying density (FP64)
  const C inv_rho = P.inv_rho;
  const C rcs2 = vr ? d.rho * C(1.0 / 3.0) : P.rcs2, inv_rcs2 = C(3) * inv_rho;
  // S3: properties, linear in c
  const C eta = prop_at(P, P.eta1, P.deta, P.eta2, P.ie1, P.ie2, cc);
  const C lam = prop_at(P, P.lam1, P.dlam, P.lam2, P.il1, P.il2, cc);
  const C tau_f = dv(eta, rcs2, inv_rcs2) + C(0.5);
  const C omega_f = C(1) / tau_f;
  const C tau_h = dv(lam, vr ? (d.rho * P.cv) * C(1.0 / 3.0) : P.rcvcs2, C(3) * P.inv_rho_cv);
  const C omega_T = C(2) / (C(2) * tau_h + C(1));
  const C omega_g = P.omega_g;
  const C af = C(1) - C(0.5) * omega_f;
  const C ag = C(1) - C(0.5) * omega_g;
  const C aT = C(1) - C(0.5) * omega_T;
  const C ux = d.ux, uy = d.uy, Fx = d.Fx, Fy = d.Fy;
  // Gamma_i(u) = w_i (1 + xi.u/c_s^2 + ((xi.u/c_s^2)^2 - u^2/c_s^2)/2) (Eq. 6)
  const C uu = dv(ux * ux + uy * uy, cs2<C>(), C(3));
  const C Gm = P.Gm;
  // H_i of Eq. 22 (H_0 below, in the FP64 branch)
  const C Hi = dv(Gm * d.mu, cs2<C>(), C(3));
  const C Gx = Fx - gpx, Gy = Fy - gpy;  // F - grad p (= Fbar, uniform rho)
  const C rcvT = (vr ? d.rho : P.rho) * P.cv * (TT + d.Trow);  // rho c_v T (full T)
  const C rcvTr = P.rho_cv * d.Trow;            // rho c_v T_r(y)
  const C rcvTd = P.rho_cv * TT;                // rho c_v T'
  if constexpr (sizeof(C) == 4) {
    // FP32: the same terms regrouped.  With a = xi_i.u/c_s^2 and
    // q = a + ((a^2 - u^2/c_s^2)/2), Gamma_i = w_i (1 + q); opposite
    // directions share (a^2 - u^2/c_s^2)/2; F.(xi_i - u) = F.xi_i - F.u.
    // The eight moving directions come first and the rest direction takes
    // the remainder of the p, c and rho c_v T equilibria (the moment minus
    // the sum of the other eight; the same value in exact arithmetic).
    // Computed directly, w_0 carries the FP32 representation error of 4/9 in
    // the same direction at every bulk cell, a systematic drift of the
    // conserved sums over long runs.
    // The odd part of the f equilibrium, w_i rho c_s^2 xi_i.u/c_s^2 =
    // 3 w_i xi_i.J with J = rho c_s^2 u, is formed from J with weights
    // K_axis = fl(1/3) and K_diag = (1 - 2 K_axis)/4, whose first-moment sum
    // 2 K_axis + 4 K_diag is exactly 1: the equilibrium then carries the
    // momentum J itself.  From u with the FP32 values of w_i and rho c_s^2
    // it carried J (1 + 3.7e-8) at every cell, which relaxation turns into a
    // growth of the momentum by 3e-8 per step: over the viscous time of a
    // flow near steady state, a bias of 1e-4 of the velocity.  J enters as
    // two floats and the relaxation f_i + omega (f_eq,i - f_i) + source is
    // formed as f_i + (omega (((S - f_i) +- A_hi) +- A_lo) + source): the
    // difference S - f_i is exact, so every rounding before the last falls
    // at the scale of the increment, and the equilibrium momentum is J to
    // its two-float precision (rounded to one float, J alone left a 3e-6
    // velocity error after the 40 000 steps of the 512 x 1024 drop).
    const C Fdu = Fx * ux + Fy * uy, Gdu = Gx * ux + Gy * uy;
    const C sg = cc * inv_rcs2;  // c / (rho c_s^2)
    const C agsg = ag * sg, aTi = aT * inv_rcs2;
    const C ux3 = C(3) * ux, uy3 = C(3) * uy;
    C sge = C(0), she = C(0);  // sums of the moving g and hbar equilibria
    static_assert(dev_h<S>(), "the FP32 forms keep hbar as a deviation");
    const C wa = WGT<C>(1), wd = WGT<C>(5);
    const C hu = C(-0.5) * uu;
    // The opposite directions (i, j) of a pair run as the two lanes of packed
    // FP32 arithmetic (fma.rn.f32x2: each lane rounds like the scalar
    // operation): q_i = a + hq, q_j = hq - a with a = xi_i.u/c_s^2.
    const float2 rcs2v = make_float2(rcs2, rcs2), ppv = make_float2(pp, pp);
    const float2 ccv = make_float2(cc, cc), Hiv = make_float2(Hi, Hi);
    const float2 rTd = make_float2(rcvTd, rcvTd), rTr = make_float2(rcvTr, rcvTr);
    const float2 rT = make_float2(rcvT, rcvT);
    const float2 omf = make_float2(omega_f, omega_f), afv = make_float2(af, af);
    const float2 omg = make_float2(omega_g, omega_g), omT = make_float2(omega_T, omega_T);
    const float2 agsgv = make_float2(agsg, agsg), aTiv = make_float2(aTi, aTi);
    const float2 m1 = make_float2(-1.f, -1.f);
    C dfs = C(0), dhs = C(0);  // sums of the moving f and hbar increments
    const float2 omTc = make_float2(omega_T - C(1), omega_T - C(1));
    C ws[9], ws0 = C(0);  // the dissipation term (below)
    auto dir2 = [&](int i, int j, C W, C K, C a, C hq, C Ja, C Jal, C Fxi, C Gxi, C offi) {
      const float2 Wv = make_float2(W, W);
      const float2 q = make_float2(a + hq, hq - a);
      const float2 G = __ffma2_rn(Wv, q, Wv);                          // Gamma_i
      // Eq. 5: even part w_i (p + rho c_s^2 hq), odd part K_i xi_i.J (two
      // floats: the product's rounding error recovered by an FMA)
      const float Sf = W * fmaf(rcs2, hq, pp), Af = K * Ja;
      const float Afl = fmaf(K, Ja, -Af) + K * Jal;
      const float2 geq = __fmul2_rn(Wv, __ffma2_rn(ccv, q, Hiv));       // Eq. 21
      const float2 heqd = __ffma2_rn(rTd, G, __fmul2_rn(rTr, __fmul2_rn(Wv, q)));
      sge += geq.x + geq.y;
      she += heqd.x + heqd.y;
      const float2 fv = make_float2(f[i], f[j]);
      const float2 gv = make_float2(g[i], g[j]);
      const float2 hv = make_float2(h[i], h[j]);
      const float2 Fd = make_float2(Fxi - Fdu, -Fxi - Fdu);  // F.(xi - u)
      const float2 gd = make_float2(Gxi - Gdu, -Gxi - Gdu);  // (F - grad p).(xi - u)
      const float2 fdel = make_float2(((Sf - fv.x) + Af) + Afl, ((Sf - fv.y) - Af) - Afl);
      const float2 finc = __ffma2_rn(omf, fdel, __fmul2_rn(afv, __fmul2_rn(Fd, G)));
      const float2 fo = __fadd2_rn(fv, finc);
      float2 go = __ffma2_rn(omg, __ffma2_rn(gv, m1, geq), gv);
      go = __ffma2_rn(__fmul2_rn(agsgv, gd), G, go);
      float2 ho = __ffma2_rn(omT, __ffma2_rn(hv, m1, heqd), hv);
      // source plus the change of reference row of a raw pulled value,
      // -(1 - omega_T) xi_iy w_i dhc: relaxing (h_raw - off) gives
      // h_raw + omega (heq - h_raw) + source - (1 - omega) off
      const float2 sT = __ffma2_rn(omTc, make_float2(offi, -offi),
                                   __fmul2_rn(__fmul2_rn(aTiv, gd), __fmul2_rn(rT, G)));
      ho = __fadd2_rn(ho, sT);
      if (wdu) {  // the dissipation term: isotropic part whole, the rest (1 - omega_T/2)
        ho.x += aT * (ws[i] - W * ws0) + W * ws0;
        ho.y += aT * (ws[j] - W * ws0) + W * ws0;
      }
      // increments, whose sum the rest direction takes with the opposite sign
      dfs += finc.x + finc.y;
      dhs += (ho.x - hv.x) + (ho.y - hv.y);
      out(0, i, fo.x);
      out(0, j, fo.y);
      out(1, i, go.x);
      out(1, j, go.y);
      out(2, i, ho.x);
      out(2, j, ho.y);
    };
    constexpr float Ka = 1.0f / 3.0f;                 // fl(1/3)
    constexpr float Kd = (1.0f - 2.0f * Ka) / 4.0f;  // exact: 2 Ka + 4 Kd = 1
    const C Jx = d.Jx, Jy = d.Jy, Jxl = d.Jxl, Jyl = d.Jyl;
    C Jp, Jpl, Jm, Jml;  // Jx + Jy and Jy - Jx as two floats
    two_sum(Jx, Jy, Jp, Jpl);
    Jpl += Jxl + Jyl;
    two_sum(Jy, -Jx, Jm, Jml);
    Jml += Jyl - Jxl;
    // the dissipation term of Eq. aEq7 (wdu given; as in the FP64 branch):
    // fbar_i = rho Gamma_i - 3 (1 - omega_f/2) (f_eq,i - f_i), with f_eq,i - f_i
    // formed as the f relaxation forms it (two floats for the odd part), not
    // as the difference of fbar and rho Gamma, whose cancellation would lose
    // three digits of the stress; q_0 = 0
    if (wdu) {
      auto pair = [&](int i, int j, C W, C K, C a, C hq, C Ja, C Jal) {
        const C Sf = W * fmaf(rcs2, hq, pp), Af = K * Ja;
        const C Afl = fmaf(K, Ja, -Af) + K * Jal;
        const C d_i = ((Sf - f[i]) + Af) + Afl, d_j = ((Sf - f[j]) - Af) - Afl;
        const C Gi = W * (C(1) + (a + hq)), Gj = W * (C(1) + (hq - a));
        auto one = [&](int k, C G, C dl) {
          const C ex = C(EX(k)), ey = C(EY(k));
          const C fph = d.rho * G - C(3) * af * dl;
          const C q = (ex - ux) * (ex * wdu[0] + ey * wdu[1]) +
                      (ey - uy) * (ex * wdu[2] + ey * wdu[3]);
          ws[k] = -fph * q;
        };
        one(i, Gi, d_i);
        one(j, Gj, d_j);
      };
      C a0 = ux3, hq0 = C(0.5) * (a0 * a0 - uu);
      pair(1, 3, wa, Ka, a0, hq0, Jx, Jxl);
      a0 = uy3;
      hq0 = C(0.5) * (a0 * a0 - uu);
      pair(2, 4, wa, Ka, a0, hq0, Jy, Jyl);
      a0 = ux3 + uy3;
      hq0 = C(0.5) * (a0 * a0 - uu);
      pair(5, 7, wd, Kd, a0, hq0, Jp, Jpl);
      a0 = uy3 - ux3;
      hq0 = C(0.5) * (a0 * a0 - uu);
      pair(6, 8, wd, Kd, a0, hq0, Jm, Jml);
      ws[0] = C(0);
#pragma unroll
      for (int i = 1; i < 9; i++) ws0 += ws[i];
    }
    C a = ux3, hq = C(0.5) * (a * a - uu);
    dir2(1, 3, wa, Ka, a, hq, Jx, Jxl, Fx, Gx, C(0));
    a = uy3;
    hq = C(0.5) * (a * a - uu);
    dir2(2, 4, wa, Ka, a, hq, Jy, Jyl, Fy, Gy, wa * dhc);
    a = ux3 + uy3;
    hq = C(0.5) * (a * a - uu);
    dir2(5, 7, wd, Kd, a, hq, Jp, Jpl, Fx + Fy, Gx + Gy, wd * dhc);
    a = uy3 - ux3;
    hq = C(0.5) * (a * a - uu);
    dir2(6, 8, wd, Kd, a, hq, Jm, Jml, Fy - Fx, Gy - Gx, wd * dhc);
    const C W0 = WGT<C>(0);
    const C G0 = W0 + W0 * hu;
    // rest direction: f and hbar take minus the sum of the moving increments
    // (the collision conserves sum f and sum hbar and the sources have no
    // zeroth moment, so this is the relaxation of f_0 and hbar_0 in exact
    // arithmetic): the cell's mass and energy then change only by the
    // rounding of its stored values, not by the rounding of p or T' (a
    // bias that repeats step after step where the fields are steady); g_0
    // in two-float arithmetic (g_0 + omega_g (g_eq,0 - g_0) + source,
    // g_eq,0 = c - sum of the moving g_eq), so that c keeps the precision of
    // its two-float moment
    (void)she;
    out(0, 0, f[0] - dfs);
    // (with the dissipation term the cell's energy gains its zeroth moment)
    out(2, 0, wdu ? (h[0] - dhs) + ws0 : h[0] - dhs);
    {
      const C src0 = (agsg * (C(0) - Gdu)) * G0;
      C s0, e0;
      two_sum(cc, -sge, s0, e0);  // g_eq,0 = s0 + (e0 + clo)
      if (omega_g == C(1)) {
        // tau_g = 1: g_0 becomes g_eq,0 + source
        C hi_new, lo_new;
        fast_two_sum(s0, (e0 + clo) + src0, hi_new, lo_new);
        out(1, 0, hi_new);
        if (g0lo_out) *g0lo_out = lo_new;
        return;
      }
      C dh, de;
      two_sum(s0, -g[0], dh, de);  // g_eq,0 - g_0 = dh + dl
      const C dl = de + ((e0 + clo) - g0lo);
      const C p = omega_g * dh;
      const C pe = fmaf(omega_g, dh, -p);  // rounding error of the product
      C hs, he;
      two_sum(g[0], p, hs, he);
      const C lo = he + pe + g0lo + omega_g * dl + src0;
      C hi_new, lo_new;
      fast_two_sum(hs, lo, hi_new, lo_new);
      out(1, 0, hi_new);
      if (g0lo_out) *g0lo_out = lo_new;
    }
  } else {
    const C H0 = dv(cc - dv((C(1) - WGT<C>(0)) * Gm * d.mu, cs2<C>(), C(3)), WGT<C>(0),
                    C(9) / C(4));
    // the pressure-work / viscous-dissipation term of Eq. aEq7 (wdu: the
    // cell's velocity gradients d_x u_x, d_y u_x, d_x u_y, d_y u_y), per
    // direction -fbar_i (xi_i - u).(xi_i.grad) u with fbar_i the density
    // distribution of the f lattice (f_i = c_s^2 fbar_i + w_i (p - rho
    // c_s^2)), its non-equilibrium part scaled by (1 - omega_f/2); its
    // isotropic part w_i sum_j enters whole (T = sum hbar/(rho c_v) carries
    // no half-step correction), the rest with (1 - omega_T/2)
    C ws[9], ws0 = C(0);
    if (wdu) {
#pragma unroll
      for (int i = 0; i < 9; i++) {
        const C W = WGT<C>(i);
        const C xu = dv(C(EX(i)) * ux + C(EY(i)) * uy, cs2<C>(), C(3));
        const C G = W * (C(1) + xu + C(0.5) * (xu * xu - uu));
        const C fbe = d.rho * G;
        const C fb = (f[i] - W * (pp - rcs2)) / cs2<C>();
        const C fph = fbe + (C(1) - C(0.5) * omega_f) * (fb - fbe);
        const C dx = C(EX(i)) - ux, dy = C(EY(i)) - uy;
        const C q = dx * (C(EX(i)) * wdu[0] + C(EY(i)) * wdu[1]) +
                    dy * (C(EX(i)) * wdu[2] + C(EY(i)) * wdu[3]);
        ws[i] = -fph * q;
        ws0 += ws[i];
      }
    }
#pragma unroll
    for (int i = 0; i < 9; i++) {
      const C W = WGT<C>(i);
      const C xu = dv(C(EX(i)) * ux + C(EY(i)) * uy, cs2<C>(), C(3));
      const C hq = C(0.5) * (xu * xu - uu);
      const C G = W * (C(1) + xu + hq);
      const C q = xu + hq;  // velocity part, without the cancelling w_i
      const C dx = C(EX(i)) - ux, dy = C(EY(i)) - uy;
      // f (Eq. 12 with Eq. 5; with a varying density the source's
      // (xi_i - u).grad(rho c_s^2) (Gamma_i(u) - w_i) term)
      const C feq = W * (pp + rcs2 * q);
      C fs = (Fx * dx + Fy * dy) * G;
      if (vr) fs = fs + (dx * d.dRx + dy * d.dRy) * (G - W);
      out(0, i, f[i] - omega_f * (f[i] - feq) + af * fs);
      // g (Eq. 27 with Eq. 21-22)
      const C geq = W * ((i == 0 ? H0 : Hi) + cc * q);
      const C gs = dv(cc * (dx * Gx + dy * Gy), rcs2, inv_rcs2) * G;
      out(1, i, g[i] - omega_g * (g[i] - geq) + ag * gs);
      // hbar (Eq. aEq12 with Eq. aEq9); deviation form:
      // h_eq - w_i rho c_v T_r = rho c_v (T' Gamma_i + T_r w_i q_i)
      const C heq = rcvT * G;
      // Fbar = grad(rho c_s^2) - grad p + F
      const C Hx = vr ? d.dRx + Gx : Gx, Hy = vr ? d.dRy + Gy : Gy;
      const C hs = dv(Hx * dx + Hy * dy, rcs2, inv_rcs2) * heq;
      const C heqd = dev_h<S>() ? rcvTd * G + rcvTr * (W * q) : heq;
      if (wdu)
        out(2, i, h[i] - omega_T * (h[i] - heqd) + aT * (hs + (ws[i] - W * ws0)) + W * ws0);
      else
        out(2, i, h[i] - omega_T * (h[i] - heqd) + aT * hs);
    }
    if (g0lo_out) *g0lo_out = C(0);
  }
}

// 16-bit forms: g_0 as c minus the stored (16-bit, stochastically rounded)
// moving g_i, gsum (their exact sum: eight 16-bit values), as two floats:
// the stored populations then carry the cell's c exactly, whatever the
// rounding of the g_i, so that sum c is conserved to the two-float precision
// of g_0 (a rounding of the g_i toward zero, as for the tiniest FP16 values,
// would otherwise drain it).  In exact arithmetic this is the relaxed g_0,
// since the collision conserves c and the source has no zeroth moment.
__device__ __forceinline__ void g0_remainder(float cc, float clo, float gsum, float& hi,
                                             float& lo) {
  float s, e;
  two_sum(cc, -gsum, s, e);
  fast_two_sum(s, e + clo, hi, lo);
}

// Store one population of cell x (row base offset rowbase) and its periodic
// ghost copies: element XG + x holds cell x; elements 0..XG-1 repeat cells
// nx-XG..nx-1 and elements nx+XG..nx+2XG-1 repeat cells 0..XG-1.
template <class S>
__device__ __forceinline__ void st_cell(const InstDev& I, char* dst, int k, int i, size_t rowbase,
                                        int x, typename S::C v) {
  S::st(I, dst, k, i, rowbase + XG + x, v);
  if (x < XG) S::st(I, dst, k, i, rowbase + XG + x + I.nx, v);
  if (x >= I.nx - XG) S::st(I, dst, k, i, rowbase + XG + x - I.nx, v);
}

// Store the low part of g_0 of cell x and its periodic ghost copies.
template <class S>
__device__ __forceinline__ void st_cell_g0lo(const InstDev& I, char* dst, size_t rowbase, int x,
                                             float lo) {
  st_g0lo<S>(I, dst, rowbase + XG + x, lo);
  if (x < XG) st_g0lo<S>(I, dst, rowbase + XG + x + I.nx, lo);
  if (x >= I.nx - XG) st_g0lo<S>(I, dst, rowbase + XG + x - I.nx, lo);
}

}  // namespace lbe

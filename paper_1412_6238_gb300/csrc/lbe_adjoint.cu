// Discrete adjoint (vector-Jacobian product) of one FP64 step, and the
// drop-migration observable.  (The adjoint recomputes the forward step with
// reciprocal products where the step divides, so it differentiates the step
// at a state equal to the FP64 one to rounding, not bitwise.)
//
// The step maps the pre-collision state Q_n (27 planes, [27][ny][nx]) to
// Q_{n+1} = Pull(Post(Q_n; theta)); Post is the collision of every cell,
// which reads its own populations and, through the stencils, c at distance
// <= 2 and p, T at distance 1 (with the wall ghost rows).  Given
// a = dL/dQ_{n+1} the adjoint step returns
//   dL/dQ_n = Post'(Q_n)^T Pull^T a + w dl/dQ_n
// and adds a^T dQ_{n+1}/dtheta (+ w dl/dtheta) to the gradient of
// theta = (sigmaT, eta ratio eta2/eta1, conductivity ratio lam2/lam1), where
// l(Q) = sum_x c u_y / sum_x c is the centroid velocity of phase 1 (the
// migration velocity of Sec. IV.C without the c >= 0.5 threshold) and w the
// loss weight of step n.  Passes, all deterministic gathers:
//   M   c, p, T of every cell                      (moments, Eq. 13/28/aEq13)
//   N   n = grad c / |grad c|_eta on cells and the ghost rows -1, ny (Eq. 3)
//   P   b = Pull^T a (the transpose of streaming with bounce-back /
//       anti-bounce-back: a permutation with signs)
//   A   per cell: recompute the forward step (stencils, mu, F, u, the three
//       collisions) and back-propagate b through it; writes the direct
//       population adjoints, the adjoints of the stencil outputs
//       (grad c, lap c, grad T, grad p, kappa) and of the cell's own c, p, T,
//       and per-block theta partials
//   B   kappa-bar -> n-bar (transposed divergence) -> grad-c-bar through the
//       normalisation, on cells and ghost rows
//   CD  per cell: transposed stencils (ghost images folded back: mirror for
//       c and p, sign flip for T) give c-bar, p-bar, T-bar, added to g, f,
//       hbar adjoints.
#include <cstdio>

#include "../../include/lbe.h"
#include "lbe_launch.h"

namespace lbe {
namespace adj {

constexpr int TPB = 256;
constexpr int RBLK = 304;  // blocks of the deterministic reductions
constexpr double CS2 = 1.0 / 3.0;
constexpr double ICS2 = 3.0;  // 1 / c_s^2: products instead of FP64 divisions

struct Geo {
  int nx, ny;
  int64_t N;  // nx * ny
};

__device__ __forceinline__ int wrap(int x, int nx) {
  x %= nx;
  return x < 0 ? x + nx : x;
}

// c with mirrored ghost rows (depth 2), p mirrored (depth 1), T antisymmetric
// about the wall temperature (depth 1)
__device__ __forceinline__ double cget(const double* c, const Geo& G, int x, int y) {
  if (y < 0) y = -1 - y;
  else if (y >= G.ny) y = 2 * G.ny - 1 - y;
  return c[(int64_t)y * G.nx + wrap(x, G.nx)];
}
__device__ __forceinline__ double Tget(const double* T, const Geo& G, const InstDev& I, int x,
                                       int y) {
  x = wrap(x, G.nx);
  if (y < 0) return 2.0 * I.Tbot[x] - T[x];
  if (y >= G.ny) return 2.0 * I.Ttop[x] - T[(int64_t)(G.ny - 1) * G.nx + x];
  return T[(int64_t)y * G.nx + x];
}
// ext arrays hold rows -1..ny (ny + 2 rows)
__device__ __forceinline__ double eget(const double* e, const Geo& G, int x, int y) {
  return e[(int64_t)(y + 1) * G.nx + wrap(x, G.nx)];
}

// isotropic gradient, index order i = 1..8, of a field given by an accessor,
// in the arithmetic type R
template <class R, class Fn>
__device__ __forceinline__ void grad_at(Fn v, int x, int y, R& gx, R& gy) {
  R sx = R(0), sy = R(0);
  for (int i = 1; i < 9; i++) {
    const R a = (R)v(x + EX(i), y + EY(i));
    sx += WGT<R>(i) * R(EX(i)) * a;
    sy += WGT<R>(i) * R(EY(i)) * a;
  }
  gx = sx * R(ICS2);
  gy = sy * R(ICS2);
}
template <class R, class Fn>
__device__ __forceinline__ R lap_at(Fn v, int x, int y) {
  const R v0 = (R)v(x, y);
  R s = R(0);
  for (int i = 1; i < 9; i++) s += WGT<R>(i) * ((R)v(x + EX(i), y + EY(i)) - v0);
  return R(2) * s * R(ICS2);
}

// ---------------------------------------------------------------- M, N, P
__global__ void pass_M(Geo G, const InstDev* __restrict__ d, const double* __restrict__ Q,
                       double* __restrict__ C, double* __restrict__ Pp, double* __restrict__ T) {
  const InstDev& I = *d;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < G.N;
       k += (int64_t)gridDim.x * blockDim.x) {
    double sf = 0, sg = 0, sh = 0;
    for (int i = 0; i < 9; i++) {
      sf += Q[(int64_t)i * G.N + k];
      sg += Q[(int64_t)(9 + i) * G.N + k];
      sh += Q[(int64_t)(18 + i) * G.N + k];
    }
    C[k] = sg;
    Pp[k] = sf;
    T[k] = sh / (I.pd.rho * I.pd.cv);
  }
}

__global__ void pass_N(Geo G, const InstDev* __restrict__ d, const double* __restrict__ C,
                       double* __restrict__ NX, double* __restrict__ NY) {
  const InstDev& I = *d;
  const int64_t NE = (int64_t)(G.ny + 2) * G.nx;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < NE;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(k % G.nx), y = (int)(k / G.nx) - 1;
    double gx, gy;
    grad_at<double>([&](int a, int b) { return cget(C, G, a, b); }, x, y, gx, gy);
    const double inv = 1.0 / sqrt(gx * gx + gy * gy + I.pd.eta_n2);
    NX[k] = gx * inv;
    NY[k] = gy * inv;
  }
}

// b_j(x) = a_j(x + xi_j), or +-a_jbar(x) where x + xi_j is beyond a wall
__global__ void pass_P(Geo G, const double* __restrict__ a, double* __restrict__ b) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < G.N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(k % G.nx), y = (int)(k / G.nx);
    for (int j = 0; j < 9; j++) {
      const int yt = y + EY(j);
      const bool wall = yt < 0 || yt >= G.ny;
      const int64_t kt = wall ? k : (int64_t)yt * G.nx + wrap(x + EX(j), G.nx);
      const int js = wall ? OPP(j) : j;
      for (int l = 0; l < 3; l++) {
        const double v = a[(int64_t)(l * 9 + js) * G.N + kt];
        b[(int64_t)(l * 9 + j) * G.N + k] = (wall && l == 2) ? -v : v;
      }
    }
  }
}

// ---------------------------------------------------------------- A
// Stencil-output adjoint planes written by pass A.
enum { S_GCX = 0, S_GCY, S_LAP, S_GTX, S_GTY, S_GPX, S_GPY, S_KAP, S_C, S_P, S_T, S_NUM };

__device__ __forceinline__ void block_sum(double v[4], double* sh) {
  for (int j = 0; j < 4; j++) sh[j * TPB + threadIdx.x] = v[j];
  __syncthreads();
  for (int s = TPB / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int j = 0; j < 4; j++) sh[j * TPB + threadIdx.x] += sh[j * TPB + threadIdx.x + s];
    __syncthreads();
  }
  for (int j = 0; j < 4; j++) v[j] = sh[j * TPB];
}

// MODE 0: observable partials (sum c u_y, sum c) into part[blk][4].
// MODE 1: adjoint of the step at this state.
// R: the arithmetic type (the planes stay FP64): double for an FP64 handle,
// float for a handle whose forward step is FP32 or 16-bit arithmetic (the
// adjoint is then linearised about an FP32 trajectory anyway; GB300's FP64
// rate is a small fraction of its FP32 rate, and this pass is most of the
// reverse sweep).  The theta partials are summed in FP64.
template <int MODE, class R>
__global__ void __launch_bounds__(TPB, sizeof(R) == 4 ? 2 : 1)
pass_A(Geo G, const InstDev* __restrict__ d, const double* __restrict__ Q,
       const double* __restrict__ C, const double* __restrict__ Pp, const double* __restrict__ T,
       const double* __restrict__ NX, const double* __restrict__ NY, const double* __restrict__ b,
       const double* __restrict__ obs, double wl, double* __restrict__ aout,
       double* __restrict__ S, double* __restrict__ part) {
  __shared__ double sh[4 * TPB];
  const InstDev& I = *d;
  const Phys<R>& P = phys<R>(I);
  const R I3 = R(ICS2), H = R(0.5), ONE = R(1), TWO = R(2);
  double acc[4] = {0, 0, 0, 0};
  for (int64_t k = blockIdx.x * (int64_t)TPB + threadIdx.x; k < G.N;
       k += (int64_t)RBLK * TPB) {
    const int x = (int)(k % G.nx), y = (int)(k / G.nx);
    R f[9], g[9], h[9];
    for (int i = 0; i < 9; i++) {
      f[i] = (R)Q[(int64_t)i * G.N + k];
      g[i] = (R)Q[(int64_t)(9 + i) * G.N + k];
      h[i] = (R)Q[(int64_t)(18 + i) * G.N + k];
    }
    const R cc = (R)C[k], pp = (R)Pp[k], TT = (R)T[k];
    auto cf = [&](int a, int bb) { return cget(C, G, a, bb); };
    auto pf = [&](int a, int bb) { return cget(Pp, G, a, bb); };
    auto Tf = [&](int a, int bb) { return Tget(T, G, I, a, bb); };
    R gcx, gcy, gTx, gTy, gpx, gpy, d1, d2, dum;
    grad_at<R>(cf, x, y, gcx, gcy);
    const R lapc = lap_at<R>(cf, x, y);
    grad_at<R>(Tf, x, y, gTx, gTy);
    grad_at<R>(pf, x, y, gpx, gpy);
    grad_at<R>([&](int a, int bb) { return eget(NX, G, a, bb); }, x, y, d1, dum);
    grad_at<R>([&](int a, int bb) { return eget(NY, G, a, bb); }, x, y, dum, d2);
    const R kappa = d1 + d2;
    // forward (same expressions as the FP64 step)
    const R mu = P.beta2 * cc * (cc - ONE) * (TWO * cc - ONE) - P.eps2 * lapc;
    const R sigma = P.sigma0 - P.sigmaT * (TT - P.Tref);
    const R g2 = gcx * gcx + gcy * gcy;
    const R gabs = sqrt(g2);
    const R cdT = gcx * gTx + gcy * gTy;
    const R ea = P.ea;
    const R cap = -sigma * kappa * ea * gabs;
    const R mar = -P.sigmaT * ea;
    const R Fx = cap * gcx + mar * (g2 * gTx - cdT * gcx) + P.Fbx;
    const R Fy = cap * gcy + mar * (g2 * gTy - cdT * gcy) + P.Fby;
    R jx = f[1] - f[3];
    jx = jx + f[5];
    jx = jx - f[6];
    jx = jx - f[7];
    jx = jx + f[8];
    R jy = f[2] - f[4];
    jy = jy + f[5];
    jy = jy + f[6];
    jy = jy - f[7];
    jy = jy - f[8];
    const R rho = P.rho, rcs2 = P.rcs2;
    // reciprocals once per cell: the FP64 divisions dominated this pass
    const R irc = ONE / rcs2, irho = ONE / rho;
    const R ux = jx * irc + H * Fx * irho;
    const R uy = jy * irc + H * Fy * irho;
    if (MODE == 0) {
      acc[0] += (double)(cc * uy);
      acc[1] += (double)cc;
      continue;
    }
    const R eta = P.eta1 + cc * P.deta;
    const R lam = P.lam1 + cc * P.dlam;
    const R tau_f = eta * irc + H;
    const R omega_f = ONE / tau_f;
    const R ircv = ONE / P.rcvcs2;
    const R tau_h = lam * ircv;
    const R omega_T = TWO / (TWO * tau_h + ONE);
    const R omega_g = P.omega_g;
    const R af = ONE - H * omega_f, ag = ONE - H * omega_g, aT = ONE - H * omega_T;
    const R uu = (ux * ux + uy * uy) * I3;
    const R Gm = P.Gm;
    const R W0 = WGT<R>(0);
    const R Hi = Gm * mu * I3;
    const R H0 = (cc - (ONE - W0) * Gm * mu * I3) * (ONE / W0);
    const R Gx = Fx - gpx, Gy = Fy - gpy;
    const R rcvT = P.rho * P.cv * TT;

    // ---- reverse through the collisions
    R fb[9], gbr[9], hb[9];
    R cb = 0, pb = 0, Tb = 0, uxb = 0, uyb = 0, Fxb = 0, Fyb = 0, Gxb = 0, Gyb = 0;
    R uub = 0, Hib = 0, H0b = 0, rcvTb = 0, wfb = 0, wTb = 0, afb = 0, aTb = 0;
    for (int i = 0; i < 9; i++) {
      const R W = WGT<R>(i);
      const R ex = R(EX(i)), ey = R(EY(i));
      const R xu = (ex * ux + ey * uy) * I3;
      const R hq = H * (xu * xu - uu);
      const R Gam = W * (ONE + xu + hq);
      const R q = xu + hq;
      const R dx = ex - ux, dy = ey - uy;
      const R feq = W * (pp + rcs2 * q);
      const R fsd = Fx * dx + Fy * dy;
      const R fs = fsd * Gam;
      const R Hx = (i == 0 ? H0 : Hi);
      const R geq = W * (Hx + cc * q);
      const R gdot = dx * Gx + dy * Gy;
      const R sgv = cc * gdot * irc;
      const R heq = rcvT * Gam;
      const R shv = (Gx * dx + Gy * dy) * irc;
      const R hs = shv * heq;
      const R bf = (R)b[(int64_t)i * G.N + k], bg = (R)b[(int64_t)(9 + i) * G.N + k],
              bh = (R)b[(int64_t)(18 + i) * G.N + k];
      R Gamb = 0, qb = 0, dxb = 0, dyb = 0, xub = 0, hqb = 0;
      // h: ho = h - wT (h - heq) + aT hs
      hb[i] = bh * (ONE - omega_T);
      wTb += bh * (heq - h[i]);
      R heqb = bh * omega_T;
      const R hsb = bh * aT;
      aTb += bh * hs;
      const R shb = hsb * heq;
      heqb += hsb * shv;
      const R shr = shb * irc;
      Gxb += shr * dx;
      Gyb += shr * dy;
      dxb += shr * Gx;
      dyb += shr * Gy;
      rcvTb += heqb * Gam;
      Gamb += heqb * rcvT;
      // g: go = g - wg (g - geq) + ag gs, gs = (c gdot / rcs2) Gam
      gbr[i] = bg * (ONE - omega_g);
      const R geqb = bg * omega_g;
      const R gsb = bg * ag;
      const R sgb = gsb * Gam;
      Gamb += gsb * sgv;
      const R sgr = sgb * irc, sgc = sgr * cc;
      cb += sgr * gdot;
      Gxb += sgc * dx;
      Gyb += sgc * dy;
      dxb += sgc * Gx;
      dyb += sgc * Gy;
      if (i == 0) H0b += geqb * W; else Hib += geqb * W;
      cb += geqb * W * q;
      qb += geqb * W * cc;
      // f: fo = f - wf (f - feq) + af fs, fs = (F.(xi - u)) Gam
      fb[i] = bf * (ONE - omega_f);
      wfb += bf * (feq - f[i]);
      const R feqb = bf * omega_f;
      const R fsb = bf * af;
      afb += bf * fs;
      Fxb += fsb * Gam * dx;
      Fyb += fsb * Gam * dy;
      dxb += fsb * Gam * Fx;
      dyb += fsb * Gam * Fy;
      Gamb += fsb * fsd;
      pb += feqb * W;
      qb += feqb * W * rcs2;
      // dx = EX - ux
      uxb -= dxb;
      uyb -= dyb;
      // Gam = W (1 + xu + hq), q = xu + hq, hq = (xu^2 - uu)/2
      xub += Gamb * W + qb;
      hqb += Gamb * W + qb;
      xub += hqb * xu;
      uub -= H * hqb;
      uxb += xub * ex * I3;
      uyb += xub * ey * I3;
    }
    Tb += rcvTb * P.rho * P.cv;
    Fxb += Gxb;
    Fyb += Gyb;
    R gpxb = -Gxb, gpyb = -Gyb;
    R mub = Hib * Gm * I3;
    cb += H0b * (ONE / W0);
    mub -= H0b * (ONE - W0) * Gm * (I3 / W0);
    uxb += uub * TWO * ux * I3;
    uyb += uub * TWO * uy * I3;
    wTb -= H * aTb;
    wfb -= H * afb;
    const R tauhb = -wTb * omega_T * omega_T;
    const R lamb = tauhb * ircv;
    const R taufb = -wfb * omega_f * omega_f;
    const R etab = taufb * irc;
    cb += etab * P.deta + lamb * P.dlam;
    R th_eta = etab * cc * P.eta1;  // d eta / d (eta2/eta1) = c eta1
    R th_lam = lamb * cc * P.lam1;
    // the observable at this step: l = A/B, dl/dc = u_y/B - A/B^2, dl/du_y = c/B
    if (wl != 0.0) {
      const R A = (R)obs[0], B = (R)obs[1], wr = (R)wl;
      cb += wr * (uy / B - A / (B * B));
      uyb += wr * cc / B;
    }
    // u = j/(rho cs2) + F/(2 rho)
    const R jxb = uxb * irc, jyb = uyb * irc;
    Fxb += H * uxb * irho;
    Fyb += H * uyb * irho;
    for (int i = 0; i < 9; i++) fb[i] += R(EX(i)) * jxb + R(EY(i)) * jyb;
    // F = cap gc + mar (g2 gT - cdT gc) + rho a
    const R capb = Fxb * gcx + Fyb * gcy;
    const R marb = Fxb * (g2 * gTx - cdT * gcx) + Fyb * (g2 * gTy - cdT * gcy);
    R gcxb = Fxb * cap - Fxb * mar * cdT;
    R gcyb = Fyb * cap - Fyb * mar * cdT;
    R g2b = mar * (Fxb * gTx + Fyb * gTy);
    R gTxb = mar * g2 * Fxb, gTyb = mar * g2 * Fyb;
    const R cdTb = -mar * (Fxb * gcx + Fyb * gcy);
    R th_sig = -marb * ea;
    // cap = -sigma kappa ea gabs
    const R sigb = -capb * kappa * ea * gabs;
    const R kapb = -capb * sigma * ea * gabs;
    const R gabsb = -capb * sigma * kappa * ea;
    gcxb += cdTb * gTx;
    gcyb += cdTb * gTy;
    gTxb += cdTb * gcx;
    gTyb += cdTb * gcy;
    if (gabs > R(0)) g2b += gabsb / (TWO * gabs);
    gcxb += TWO * g2b * gcx;
    gcyb += TWO * g2b * gcy;
    // sigma = sigma0 - sigmaT (T - Tref)
    Tb += -sigb * P.sigmaT;
    th_sig += -sigb * (TT - P.Tref);
    // mu = 2 beta c (c-1)(2c-1) - eps^2 lap c
    cb += mub * P.beta2 * (R(6) * cc * cc - R(6) * cc + ONE);
    const R lapb = -mub * P.eps2;

    for (int i = 0; i < 9; i++) {
      aout[(int64_t)i * G.N + k] = (double)fb[i];
      aout[(int64_t)(9 + i) * G.N + k] = (double)gbr[i];
      aout[(int64_t)(18 + i) * G.N + k] = (double)hb[i];
    }
    S[(int64_t)S_GCX * G.N + k] = (double)gcxb;
    S[(int64_t)S_GCY * G.N + k] = (double)gcyb;
    S[(int64_t)S_LAP * G.N + k] = (double)lapb;
    S[(int64_t)S_GTX * G.N + k] = (double)gTxb;
    S[(int64_t)S_GTY * G.N + k] = (double)gTyb;
    S[(int64_t)S_GPX * G.N + k] = (double)gpxb;
    S[(int64_t)S_GPY * G.N + k] = (double)gpyb;
    S[(int64_t)S_KAP * G.N + k] = (double)kapb;
    S[(int64_t)S_C * G.N + k] = (double)cb;
    S[(int64_t)S_P * G.N + k] = (double)pb;
    S[(int64_t)S_T * G.N + k] = (double)Tb;
    acc[0] += (double)th_sig;
    acc[1] += (double)th_eta;
    acc[2] += (double)th_lam;
  }
  block_sum(acc, sh);
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; j++) part[blockIdx.x * 4 + j] = acc[j];
}

// ---------------------------------------------------------------- B
// kappa(X) = sum_i (w_i/cs2) xi_i . n(X + xi_i)  =>  n-bar(Y) = sum_i
// (w_i/cs2) xi_i kappa-bar(Y - xi_i) over cells Y - xi_i; then through
// n = v / s, s = sqrt(|v|^2 + eta_n^2): v-bar = n-bar/s - v (v.n-bar)/s^3.
// R: the arithmetic type, as for pass A.
template <class R>
__global__ void pass_B(Geo G, const InstDev* __restrict__ d, const double* __restrict__ C,
                       const double* __restrict__ S, double* __restrict__ VX,
                       double* __restrict__ VY) {
  const InstDev& I = *d;
  const int64_t NE = (int64_t)(G.ny + 2) * G.nx;
  const double* kb = S + (int64_t)S_KAP * G.N;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < NE;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(k % G.nx), y = (int)(k / G.nx) - 1;
    R nbx = 0, nby = 0;
    for (int i = 1; i < 9; i++) {
      const int yy = y - EY(i);
      if (yy < 0 || yy >= G.ny) continue;
      const R kv = (R)kb[(int64_t)yy * G.nx + wrap(x - EX(i), G.nx)];
      nbx += WGT<R>(i) * R(EX(i)) / R(CS2) * kv;
      nby += WGT<R>(i) * R(EY(i)) / R(CS2) * kv;
    }
    R vx, vy;
    grad_at<R>([&](int a, int bb) { return cget(C, G, a, bb); }, x, y, vx, vy);
    const R s2 = vx * vx + vy * vy + phys<R>(I).eta_n2;
    const R s = sqrt(s2);
    const R vn = vx * nbx + vy * nby;
    VX[k] = (double)(nbx / s - vx * vn / (s2 * s));
    VY[k] = (double)(nby / s - vy * vn / (s2 * s));
  }
}

// ---------------------------------------------------------------- CD
// R: the arithmetic type, as for pass A.
template <class R>
__global__ void pass_CD(Geo G, const InstDev* __restrict__ d, const double* __restrict__ S,
                        const double* __restrict__ VX, const double* __restrict__ VY,
                        double* __restrict__ aout) {
  const InstDev& I = *d;
  const int ny = G.ny;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < G.N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(k % G.nx), y = (int)(k / G.nx);
    R cb = (R)S[(int64_t)S_C * G.N + k];
    R pb = (R)S[(int64_t)S_P * G.N + k];
    R Tb = (R)S[(int64_t)S_T * G.N + k];
    // Laplacian centre term
    R sw = R(0);
    for (int i = 1; i < 9; i++) sw += WGT<R>(i);
    cb += R(-2) * sw / R(CS2) * (R)S[(int64_t)S_LAP * G.N + k];
    // positions q holding c(x, y): the cell and its ghost images
    int qs[5], nq = 0;
    qs[nq++] = y;
    const int gr[4] = {-2, -1, ny, ny + 1};
    for (int j = 0; j < 4; j++) {
      const int m = gr[j] < 0 ? -1 - gr[j] : 2 * ny - 1 - gr[j];
      if (m == y) qs[nq++] = gr[j];
    }
    for (int jq = 0; jq < nq; jq++) {
      const int qy = qs[jq];
      const bool depth1 = qy >= -1 && qy <= ny;  // p, T ghosts reach one row
      const R tsign = (qy == y) ? R(1) : R(-1);
      for (int i = 1; i < 9; i++) {
        const int X = wrap(x - EX(i), G.nx), Y = qy - EY(i);
        const R wa = WGT<R>(i) / R(CS2);
        const R ex = R(EX(i)), ey = R(EY(i));
        if (Y >= 0 && Y < ny) {
          const int64_t kk = (int64_t)Y * G.nx + X;
          cb += wa * (ex * (R)S[(int64_t)S_GCX * G.N + kk] + ey * (R)S[(int64_t)S_GCY * G.N + kk]);
          cb += R(2) * wa * (R)S[(int64_t)S_LAP * G.N + kk];
          if (depth1) {
            pb += wa * (ex * (R)S[(int64_t)S_GPX * G.N + kk] +
                        ey * (R)S[(int64_t)S_GPY * G.N + kk]);
            Tb += tsign * wa *
                  (ex * (R)S[(int64_t)S_GTX * G.N + kk] + ey * (R)S[(int64_t)S_GTY * G.N + kk]);
          }
        }
        if (Y >= -1 && Y <= ny) {
          const int64_t ke = (int64_t)(Y + 1) * G.nx + X;
          cb += wa * (ex * (R)VX[ke] + ey * (R)VY[ke]);
        }
      }
    }
    const R Tsc = Tb / (phys<R>(I).rho * phys<R>(I).cv);
    for (int i = 0; i < 9; i++) {
      aout[(int64_t)i * G.N + k] += (double)pb;
      aout[(int64_t)(9 + i) * G.N + k] += (double)cb;
      aout[(int64_t)(18 + i) * G.N + k] += (double)Tsc;
    }
  }
}

__global__ void dT0_kernel(Geo G, const InstDev* __restrict__ d, const double* __restrict__ a,
                           double* __restrict__ out) {
  const double rcv = d->pd.rho * d->pd.cv;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < G.N;
       k += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < 9; i++) s += WGT<double>(i) * a[(int64_t)(18 + i) * G.N + k];
    out[k] = rcv * s;
  }
}

// final reduction of the per-block partials: into out[0..3] (overwrite) or
// added to acc[0..3]
__global__ void reduce_parts(const double* __restrict__ part, double* __restrict__ out,
                             int accumulate) {
  __shared__ double sh[4 * TPB];
  double v[4] = {0, 0, 0, 0};
  for (int bb = threadIdx.x; bb < RBLK; bb += TPB)
    for (int j = 0; j < 4; j++) v[j] += part[bb * 4 + j];
  block_sum(v, sh);
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; j++) out[j] = accumulate ? out[j] + v[j] : v[j];
}

}  // namespace adj

// Scratch doubles needed for one instance of nx x ny cells.
int64_t adjoint_scratch_doubles(int nx, int ny) {
  const int64_t N = (int64_t)nx * ny, NE = (int64_t)nx * (ny + 2);
  return 27 * N + 3 * N + 2 * NE + adj::S_NUM * N + 2 * NE + 4 * adj::RBLK + 8;
}

cudaError_t launch_observable(const InstDev* d, int nx, int ny, const double* Q, double* scratch,
                              double* out4, cudaStream_t s) {
  using namespace adj;
  const Geo G{nx, ny, (int64_t)nx * ny};
  const int64_t NE = (int64_t)nx * (ny + 2);
  double* C = scratch + 27 * G.N;
  double* Pp = C + G.N;
  double* T = Pp + G.N;
  double* NX = T + G.N;
  double* NY = NX + NE;
  double* S = NY + NE;
  double* part = S + S_NUM * G.N + 2 * NE;
  const int gN = (int)((G.N + TPB - 1) / TPB < 65535 ? (G.N + TPB - 1) / TPB : 65535);
  const int gE = (int)((NE + TPB - 1) / TPB < 65535 ? (NE + TPB - 1) / TPB : 65535);
  pass_M<<<gN, TPB, 0, s>>>(G, d, Q, C, Pp, T);
  pass_N<<<gE, TPB, 0, s>>>(G, d, C, NX, NY);
  pass_A<0, double><<<RBLK, TPB, 0, s>>>(G, d, Q, C, Pp, T, NX, NY, nullptr, nullptr, 0.0,
                                         nullptr, nullptr, part);
  reduce_parts<<<1, TPB, 0, s>>>(part, out4, 0);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_step(const InstDev* d, int nx, int ny, const double* Q,
                                const double* a_next, double wl, const double* obs,
                                double* a_out, double* theta_acc, double* scratch, bool fp32,
                                cudaStream_t s) {
  using namespace adj;
  const Geo G{nx, ny, (int64_t)nx * ny};
  const int64_t NE = (int64_t)nx * (ny + 2);
  double* b = scratch;
  double* C = b + 27 * G.N;
  double* Pp = C + G.N;
  double* T = Pp + G.N;
  double* NX = T + G.N;
  double* NY = NX + NE;
  double* S = NY + NE;
  double* VX = S + S_NUM * G.N;
  double* VY = VX + NE;
  double* part = VY + NE;
  const int gN = (int)((G.N + TPB - 1) / TPB < 65535 ? (G.N + TPB - 1) / TPB : 65535);
  const int gE = (int)((NE + TPB - 1) / TPB < 65535 ? (NE + TPB - 1) / TPB : 65535);
  pass_M<<<gN, TPB, 0, s>>>(G, d, Q, C, Pp, T);
  pass_N<<<gE, TPB, 0, s>>>(G, d, C, NX, NY);
  if (a_next) {
    pass_P<<<gN, TPB, 0, s>>>(G, a_next, b);
  } else {
    cudaError_t e = cudaMemsetAsync(b, 0, sizeof(double) * 27 * G.N, s);
    if (e != cudaSuccess) return e;
  }
  if (fp32) {
    pass_A<1, float><<<RBLK, TPB, 0, s>>>(G, d, Q, C, Pp, T, NX, NY, b, obs, wl, a_out, S, part);
    reduce_parts<<<1, TPB, 0, s>>>(part, theta_acc, 1);
    pass_B<float><<<gE, TPB, 0, s>>>(G, d, C, S, VX, VY);
    pass_CD<float><<<gN, TPB, 0, s>>>(G, d, S, VX, VY, a_out);
  } else {
    pass_A<1, double><<<RBLK, TPB, 0, s>>>(G, d, Q, C, Pp, T, NX, NY, b, obs, wl, a_out, S,
                                           part);
    reduce_parts<<<1, TPB, 0, s>>>(part, theta_acc, 1);
    pass_B<double><<<gE, TPB, 0, s>>>(G, d, C, S, VX, VY);
    pass_CD<double><<<gN, TPB, 0, s>>>(G, d, S, VX, VY, a_out);
  }
  return cudaGetLastError();
}

cudaError_t launch_adjoint_dT0(const InstDev* d, int nx, int ny, const double* a, double* dT0,
                               cudaStream_t s) {
  using namespace adj;
  const Geo G{nx, ny, (int64_t)nx * ny};
  const int gN = (int)((G.N + TPB - 1) / TPB < 65535 ? (G.N + TPB - 1) / TPB : 65535);
  dT0_kernel<<<gN, TPB, 0, s>>>(G, d, a, dT0);
  return cudaGetLastError();
}

}  // namespace lbe

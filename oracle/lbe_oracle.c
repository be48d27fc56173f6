/*
 * FP64 CPU oracle for one time step of the three coupled D2Q9 lattices of the
 * continuous-surface-force (CSF) lattice Boltzmann method for thermocapillary
 * flow (Zheng, Zheng & Zhai, arXiv:1412.6238).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is compared against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header or
 * table with the CUDA library.
 *
 * Everything is double precision and written as loops over cells, in the order
 * the paper states the scheme:
 *
 *   1. moments      c = sum g_i (Eq. 28), p = sum f_i (Eq. 13, uniform rho),
 *                   rho c_v T = sum hbar_i (Eq. aEq13)
 *   2. ghost rows   mirror for c and p, antisymmetric about the wall value
 *                   for T (the paper names the walls but gives no scheme)
 *   3. stencils     isotropic D2Q9 gradient and Laplacian; n = grad c/|grad c|
 *                   (regularised), kappa = div n (Eq. 3)
 *   4. properties   eta(c), lambda(c) linear in c; tau_f from
 *                   eta = rho c_s^2 (tau_f - 1/2) (Sec. II), omega_T from
 *                   omega = 2/(2 tau_h + 1) and lambda = rho c_v c_s^2 tau_h
 *                   (Eq. aEq12, aEq14 and Appendix A)
 *   5. mu = mu_0 - eps^2 lap c with E_0 = beta c^2 (c-1)^2 (Sec. II, Eq. 16)
 *   6. F = eps*alpha*|grad c|^2 (-sigma kappa n + grad_s sigma) + rho a (Eq. 3,
 *      Eq. aEq3), alpha = 6 sqrt(2)
 *   7. u = sum xi_i f_i / (rho c_s^2) + F/(2 rho)   (Eq. 13, read so that the
 *      half-step force carries the c_s^2 that the first moment of the Eq. 12
 *      source has)
 *   8. collide f (Eq. 12, Eq. 5, Eq. 6), g (Eq. 27, Eq. 21, Eq. 22),
 *      hbar (Eq. aEq12, Eq. aEq9)
 *   9. stream (pull form), periodic in x, halfway bounce-back for f and g and
 *      anti-bounce-back for hbar at walls half a cell outside the first and
 *      last rows.
 *
 * Variants the paper leaves open (orc_params; each off by default): a
 * density varying with c (the grad(rho c_s^2) terms of Eq. 12, Eq. 13 and
 * Fbar); the harmonic property law; the anti-bounce-back's wall temperature
 * taken where the link crosses the wall; wetting walls with a contact angle
 * (Young's law through a cubic wall energy); the pressure-work and
 * viscous-dissipation term of Eq. aEq7 that Eq. aEq8 drops.
 *
 * Population storage: one array of 27 planes [k*9+i][y][x], k = 0 (f), 1 (g),
 * 2 (hbar), x fastest.  Velocity order i: 0 (0,0), 1 (1,0), 2 (0,1), 3 (-1,0),
 * 4 (0,-1), 5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no FMA contraction,
 * so that every product and sum rounds once, as written).
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t nx, ny;
  int32_t periodic_y; /* 0: walls at y=-1/2 and y=ny-1/2; 1: periodic in y */
  int32_t ablate;     /* test hook, 0 normally: bit 0 drops the grad(rho cs2)
                         source of Eq. 12, bit 1 the pressure correction of
                         Eq. 13, bit 2 grad(rho cs2) in Fbar (planted
                         mistakes the density pins must detect) */
  double rho, cv;     /* rho: density of phase c = 0 (see rho2) */
  double eta1, eta2, lam1, lam2; /* phase c=0 and phase c=1 */
  double sigma0, sigmaT, Tref;   /* sigma = sigma0 - sigmaT (T - Tref) */
  double eps, beta, tau_g, mobility;
  double ax, ay;   /* body acceleration */
  double eta_n;    /* regularisation of n = grad c / sqrt(|grad c|^2+eta_n^2) */
  double rho2;     /* density of phase c = 1 (rho2 = rho: uniform density) */
  /* boundary and property variants (0: the scheme as the paper states it) */
  int32_t interp;   /* eta(c), lambda(c): 0 linear, 1 harmonic */
  int32_t wall_mid; /* 1: the anti-bounce-back of a link takes T_w where the
                       link crosses the wall (x - xi_x/2, interpolated) */
  double cos_wet;   /* cos of the contact angle of phase 1 at both walls
                       (0: neutral wetting, the mirror ghost rows) */
  int32_t dissip;   /* 1: keep the -fbar_i q_i term of Eq. aEq7 (pressure
                       work and viscous dissipation) that Eq. aEq8 drops */
  int32_t pad_;
} orc_params;

/* Density of a cell, linear in c like eta and lambda (the paper states no
 * interpolation): rho(c) = rho1 + c (rho2 - rho1).  With rho2 = rho1 every
 * expression below reduces exactly to the uniform-density one. */
static double rho_of(const orc_params* P, double c) {
  return P->rho + c * (P->rho2 - P->rho);
}
static int varying_rho(const orc_params* P) { return P->rho2 != P->rho; }

/* A property of a cell between its phase-0 value a and phase-1 value b.
 * Linear in c (the default; the paper gives no law), or harmonic,
 * 1/((1 - c)/a + c/b), whose series form keeps the flux continuous across
 * a layered interface (conduction, shear). */
static double prop_of(const orc_params* P, double a, double b, double c) {
  if (P->interp == 1) return 1.0 / ((1.0 - c) / a + c / b);
  return a + c * (b - a);
}

/* Wetting walls: the free energy beta c^2 (c-1)^2 + (eps^2/2)|grad c|^2 with
 * the cubic wall energy -sigma cos(theta) (3c^2 - 2c^3), sigma =
 * eps sqrt(2 beta)/6, gives at a wall the condition
 *   dc/dn_out = (sqrt(2 beta)/eps) cos(theta) c (1 - c)
 * (n_out pointing out of the fluid): Young's law with contact angle theta of
 * phase 1.  Ghost row -1-j (or ny+j) of c: its mirror cell j plus
 * (2j+1) times that flux, evaluated at the mirror cell's c (the normal
 * distance between the two is 2j+1). */
static double wet_ghost(const orc_params* P, double cm, int j) {
  const double kw = P->cos_wet * sqrt(2.0 * P->beta) / P->eps;
  return cm + (double)(2 * j + 1) * kw * cm * (1.0 - cm);
}

/* ---- D2Q9 lattice (the paper names D2Q9 weights but does not list them) */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                            1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

void orc_lattice(int32_t ex[9], int32_t ey[9], double w[9], int32_t opp[9],
                 double* cs2) {
  for (int i = 0; i < 9; i++) {
    ex[i] = EX[i];
    ey[i] = EY[i];
    w[i] = W[i];
    opp[i] = OPP[i];
  }
  *cs2 = CS2;
}

/* ---- Eq. 6: Gamma_i(u) = w_i {1 + xi.u/cs2 + [(xi.u/cs2)^2 - u^2/cs2]/2} */
static double gamma_i(int i, double ux, double uy) {
  double xu = (EX[i] * ux + EY[i] * uy) / CS2;
  double uu = (ux * ux + uy * uy) / CS2;
  return W[i] * (1.0 + xu + 0.5 * (xu * xu - uu));
}

/* ---- Eq. 5: f_eq_i = w_i [p + rho cs2 (xi.u/cs2 + ((xi.u/cs2)^2 - u^2/cs2)/2)] */
static double f_equilibrium(int i, double p, double rho, double ux, double uy) {
  double xu = (EX[i] * ux + EY[i] * uy) / CS2;
  double uu = (ux * ux + uy * uy) / CS2;
  return W[i] * (p + rho * CS2 * (xu + 0.5 * (xu * xu - uu)));
}

/* ---- Eq. 21 with Eq. 22: g_eq_i = w_i {H_i + c[xi.u/cs2 + (...)/2]},
 *      H_0 = [c - (1-w_0) Gm mu/cs2]/w_0, H_{i>0} = Gm mu/cs2,
 *      Gm = M/(tau_g - 1/2) (the paper's Gamma, Eq. 16). */
static double g_equilibrium(int i, double c, double mu, double Gm, double ux,
                            double uy) {
  double xu = (EX[i] * ux + EY[i] * uy) / CS2;
  double uu = (ux * ux + uy * uy) / CS2;
  double H;
  if (i == 0)
    H = (c - (1.0 - W[0]) * Gm * mu / CS2) / W[0];
  else
    H = Gm * mu / CS2;
  return W[i] * (H + c * (xu + 0.5 * (xu * xu - uu)));
}

/* ---- Eq. aEq9: h_eq_i = rho c_v T Gamma_i(u) */
static double h_equilibrium(int i, double rho, double cv, double T, double ux,
                            double uy) {
  return rho * cv * T * gamma_i(i, ux, uy);
}

/* ---- Eq. 12 source (without the (1 - omega/2) factor):
 *      F.(xi_i - u) Gamma_i(u) + (xi_i - u).grad(rho cs2) (Gamma_i(u) - Gamma_i(0)),
 *      Gamma_i(0) = w_i; (dRx, dRy) = grad(rho cs2), zero for uniform rho
 *      (then the second term is left out). */
static double f_source(int i, double Fx, double Fy, double ux, double uy, double dRx,
                       double dRy, int with_drho) {
  double G = gamma_i(i, ux, uy);
  double s = (Fx * (EX[i] - ux) + Fy * (EY[i] - uy)) * G;
  if (with_drho) s += ((EX[i] - ux) * dRx + (EY[i] - uy) * dRy) * (G - W[i]);
  return s;
}

/* ---- Eq. 27 source (without the (1 - omega/2) factor):
 *      [c (xi_i - u).(F - grad p) / (rho cs2)] Gamma_i(u) */
static double g_source(int i, double c, double rho, double Fx, double Fy,
                       double gpx, double gpy, double ux, double uy) {
  double G = gamma_i(i, ux, uy);
  return c * ((EX[i] - ux) * (Fx - gpx) + (EY[i] - uy) * (Fy - gpy)) /
         (rho * CS2) * G;
}

/* ---- Eq. aEq12 source (without the (1 - omega/2) factor):
 *      Fbar.(xi_i - u)/(rho cs2) h_eq_i, Fbar = grad(rho cs2) - grad p + F
 *      (after Eq. aEq4); grad(rho cs2) = (dRx, dRy), zero for uniform rho. */
static double h_source(int i, double rho, double cv, double T, double Fx,
                       double Fy, double gpx, double gpy, double ux,
                       double uy, double dRx, double dRy, int with_drho) {
  double Fbx = Fx - gpx, Fby = Fy - gpy;
  if (with_drho) {
    Fbx = dRx + Fbx;
    Fby = dRy + Fby;
  }
  return (Fbx * (EX[i] - ux) + Fby * (EY[i] - uy)) / (rho * CS2) *
         h_equilibrium(i, rho, cv, T, ux, uy);
}

/* The pressure-work / viscous-dissipation term of Eq. aEq7 (kept when the
 * variant `dissip` is on; Eq. aEq8 drops it), per direction:
 *   S_i = -fbar_i q_i,  q_i = (xi_i - u).(d_t u + (xi_i.grad) u).
 * - Sign: h = |xi - u|^2/2 fbar (Eq. aEq6) gives -fbar q on differentiating
 *   (the printed + would make viscous dissipation cool the fluid).
 * - fbar_i, the density distribution, from the f lattice by the change of
 *   variables behind Eq. 5, f_i = c_s^2 fbar_i + w_i (p - rho c_s^2), its
 *   non-equilibrium part scaled by (1 - omega_f/2) to the physical
 *   distribution of the trapezoidal scheme (whose stress is the viscous
 *   stress of eta = rho c_s^2 (tau_f - 1/2)).
 * - The d_t u part is left out: its zeroth moment, (sum_i fbar_i (xi_i - u)).
 *   d_t u, vanishes (sum fbar xi = rho u), so the energy equation does not
 *   see it.
 * Then sum_i S_i = -p_th div u + the viscous dissipation (eta/2)|grad u +
 * grad u^T|^2 with p_th = rho c_s^2.  In the collision the isotropic part
 * w_i sum_j S_j enters whole and the rest with the trapezoidal factor
 * (1 - omega_T/2) of Eq. aEq12: T = sum hbar / (rho c_v) has no half-step
 * correction for a source with a zeroth moment, and through (1 - omega_T/2)
 * alone the fluid would gain only that fraction of the heat.  du =
 * {d_x u_x, d_y u_x, d_x u_y, d_y u_y}. */
static double work_source(int i, double rho, double p, double f, double omega_f, double ux,
                          double uy, const double du[4]) {
  const double fbe = rho * gamma_i(i, ux, uy);
  const double fb = (f - W[i] * (p - rho * CS2)) / CS2;
  const double fph = fbe + (1.0 - 0.5 * omega_f) * (fb - fbe);
  const double dx = EX[i] - ux, dy = EY[i] - uy;
  const double q = dx * (EX[i] * du[0] + EY[i] * du[1]) + dy * (EX[i] * du[2] + EY[i] * du[3]);
  return -fph * q;
}

/* Per-cell terms for the moment pins in the tests: equilibria and sources. */
void orc_cell_terms(const orc_params* P, double c, double p, double T,
                    double mu, double ux, double uy, double Fx, double Fy,
                    double gpx, double gpy, double feq[9], double geq[9],
                    double heq[9], double fsrc[9], double gsrc[9],
                    double hsrc[9]) {
  double Gm = P->mobility / (P->tau_g - 0.5);
  for (int i = 0; i < 9; i++) {
    feq[i] = f_equilibrium(i, p, P->rho, ux, uy);
    geq[i] = g_equilibrium(i, c, mu, Gm, ux, uy);
    heq[i] = h_equilibrium(i, P->rho, P->cv, T, ux, uy);
    fsrc[i] = f_source(i, Fx, Fy, ux, uy, 0.0, 0.0, 0);
    gsrc[i] = g_source(i, c, P->rho, Fx, Fy, gpx, gpy, ux, uy);
    hsrc[i] = h_source(i, P->rho, P->cv, T, Fx, Fy, gpx, gpy, ux, uy, 0.0, 0.0, 0);
  }
}

/* ------------------------------------------------------------------------
 * Scalar fields with ghost rows.  An extended field holds rows
 * -G .. ny-1+G (G ghost rows each side); x is periodic and wrapped on access.
 */
typedef struct {
  int nx, ny, G;
  double* v; /* (ny + 2G) * nx */
} ext_field;

static double* ext_at(ext_field* e, int x, int y) {
  int xx = ((x % e->nx) + e->nx) % e->nx;
  return &e->v[(size_t)(y + e->G) * e->nx + xx];
}
static double ext_get(const ext_field* e, int x, int y) {
  int xx = ((x % e->nx) + e->nx) % e->nx;
  return e->v[(size_t)(y + e->G) * e->nx + xx];
}
static ext_field ext_new(int nx, int ny, int G) {
  ext_field e = {nx, ny, G, NULL};
  e.v = (double*)calloc((size_t)(ny + 2 * G) * nx, sizeof(double));
  return e;
}

/* Isotropic gradient: d_a phi = (1/cs2) sum_{i>=1} w_i xi_ia phi(x + xi_i). */
static void grad_iso(const ext_field* e, int x, int y, double* gx,
                     double* gy) {
  double sx = 0.0, sy = 0.0;
  for (int i = 1; i < 9; i++) {
    double v = ext_get(e, x + EX[i], y + EY[i]);
    sx += W[i] * EX[i] * v;
    sy += W[i] * EY[i] * v;
  }
  *gx = sx / CS2;
  *gy = sy / CS2;
}

/* Isotropic Laplacian: lap phi = (2/cs2) sum_{i>=1} w_i (phi(x+xi_i) - phi(x)). */
static double lap_iso(const ext_field* e, int x, int y) {
  double s = 0.0, v0 = ext_get(e, x, y);
  for (int i = 1; i < 9; i++) s += W[i] * (ext_get(e, x + EX[i], y + EY[i]) - v0);
  return 2.0 * s / CS2;
}

/* Fill ghost rows.  Walls: p (is_T = 0) and c (is_T = 2) mirror about the
 * wall (phi(-1-j) = phi(j)), c with the wetting flux added when the contact
 * angle is not 90 degrees; T (is_T = 1) is antisymmetric about the wall
 * temperature at the same column (T(-1-j) = 2 T_w - T(j)).  Periodic y:
 * wrap. */
static void fill_ghosts(const orc_params* P, ext_field* e, int is_T,
                        const double* Tbot, const double* Ttop) {
  int nx = e->nx, ny = e->ny;
  for (int j = 0; j < e->G; j++) {
    for (int x = 0; x < nx; x++) {
      if (P->periodic_y) {
        *ext_at(e, x, -1 - j) = ext_get(e, x, ny - 1 - j);
        *ext_at(e, x, ny + j) = ext_get(e, x, j);
      } else if (is_T == 1) {
        *ext_at(e, x, -1 - j) = 2.0 * Tbot[x] - ext_get(e, x, j);
        *ext_at(e, x, ny + j) = 2.0 * Ttop[x] - ext_get(e, x, ny - 1 - j);
      } else if (is_T == 3) { /* velocity: zero at the wall (no slip) */
        *ext_at(e, x, -1 - j) = -ext_get(e, x, j);
        *ext_at(e, x, ny + j) = -ext_get(e, x, ny - 1 - j);
      } else if (is_T == 2 && P->cos_wet != 0.0) {
        *ext_at(e, x, -1 - j) = wet_ghost(P, ext_get(e, x, j), j);
        *ext_at(e, x, ny + j) = wet_ghost(P, ext_get(e, x, ny - 1 - j), j);
      } else {
        *ext_at(e, x, -1 - j) = ext_get(e, x, j);
        *ext_at(e, x, ny + j) = ext_get(e, x, ny - 1 - j);
      }
    }
  }
}

/* Outputs of the scalar stage at every cell (arrays of nx*ny). */
typedef struct {
  double *gcx, *gcy, *lapc, *kappa, *gTx, *gTy, *gpx, *gpy, *mu, *Fx, *Fy;
} scalar_out;

/* Steps 2-6 from cell values of c, p, T. */
static void scalar_stage(const orc_params* P, const double* Tbot,
                         const double* Ttop, const double* c, const double* p,
                         const double* T, scalar_out* o) {
  const int nx = P->nx, ny = P->ny;
  ext_field cE = ext_new(nx, ny, 2), pE = ext_new(nx, ny, 1),
            TE = ext_new(nx, ny, 1);
  ext_field nxE = ext_new(nx, ny, 1), nyE = ext_new(nx, ny, 1);
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      *ext_at(&cE, x, y) = c[(size_t)y * nx + x];
      *ext_at(&pE, x, y) = p[(size_t)y * nx + x];
      *ext_at(&TE, x, y) = T[(size_t)y * nx + x];
    }
  fill_ghosts(P, &cE, 2, Tbot, Ttop);
  fill_ghosts(P, &pE, 0, Tbot, Ttop);
  fill_ghosts(P, &TE, 1, Tbot, Ttop);

  /* unit normal n on cells and on one ghost row each side (Eq. 3) */
  const double en2 = P->eta_n * P->eta_n;
#pragma omp parallel for schedule(static)
  for (int y = -1; y <= ny; y++)
    for (int x = 0; x < nx; x++) {
      double gx, gy;
      grad_iso(&cE, x, y, &gx, &gy);
      double inv = 1.0 / sqrt(gx * gx + gy * gy + en2);
      *ext_at(&nxE, x, y) = gx * inv;
      *ext_at(&nyE, x, y) = gy * inv;
    }

  const double alpha = 6.0 * sqrt(2.0); /* delta normalisation, Sec. II */
  const double ea = P->eps * alpha;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      size_t k = (size_t)y * nx + x;
      double gcx, gcy, gTx, gTy, gpx, gpy, d1, d2, dummy;
      grad_iso(&cE, x, y, &gcx, &gcy);
      double lapc = lap_iso(&cE, x, y);
      grad_iso(&TE, x, y, &gTx, &gTy);
      grad_iso(&pE, x, y, &gpx, &gpy);
      /* kappa = div n with the same isotropic stencil */
      grad_iso(&nxE, x, y, &d1, &dummy);
      grad_iso(&nyE, x, y, &dummy, &d2);
      double kappa = d1 + d2;

      double cc = c[k];
      double mu = 2.0 * P->beta * cc * (cc - 1.0) * (2.0 * cc - 1.0) -
                  P->eps * P->eps * lapc;

      double sigma = P->sigma0 - P->sigmaT * (T[k] - P->Tref);
      double g2 = gcx * gcx + gcy * gcy;
      double gabs = sqrt(g2);
      double cdT = gcx * gTx + gcy * gTy;
      /* -sigma kappa delta n with delta n = eps alpha |grad c| grad c */
      double Fx = -sigma * kappa * ea * gabs * gcx;
      double Fy = -sigma * kappa * ea * gabs * gcy;
      /* delta grad_s sigma with grad sigma = -sigmaT grad T and
         delta (I - n n) grad T = eps alpha (|grad c|^2 grad T - (grad c.grad T) grad c) */
      Fx += -P->sigmaT * ea * (g2 * gTx - cdT * gcx);
      Fy += -P->sigmaT * ea * (g2 * gTy - cdT * gcy);
      /* body force, part of the total F of Eq. 1 */
      Fx += rho_of(P, cc) * P->ax;
      Fy += rho_of(P, cc) * P->ay;

      o->gcx[k] = gcx;
      o->gcy[k] = gcy;
      o->lapc[k] = lapc;
      o->kappa[k] = kappa;
      o->gTx[k] = gTx;
      o->gTy[k] = gTy;
      o->gpx[k] = gpx;
      o->gpy[k] = gpy;
      o->mu[k] = mu;
      o->Fx[k] = Fx;
      o->Fy[k] = Fy;
    }
  free(cE.v);
  free(pE.v);
  free(TE.v);
  free(nxE.v);
  free(nyE.v);
}

static scalar_out scalar_out_new(size_t n) {
  scalar_out o;
  o.gcx = calloc(n, sizeof(double));
  o.gcy = calloc(n, sizeof(double));
  o.lapc = calloc(n, sizeof(double));
  o.kappa = calloc(n, sizeof(double));
  o.gTx = calloc(n, sizeof(double));
  o.gTy = calloc(n, sizeof(double));
  o.gpx = calloc(n, sizeof(double));
  o.gpy = calloc(n, sizeof(double));
  o.mu = calloc(n, sizeof(double));
  o.Fx = calloc(n, sizeof(double));
  o.Fy = calloc(n, sizeof(double));
  return o;
}
static void scalar_out_free(scalar_out* o) {
  free(o->gcx); free(o->gcy); free(o->lapc); free(o->kappa); free(o->gTx);
  free(o->gTy); free(o->gpx); free(o->gpy); free(o->mu); free(o->Fx);
  free(o->Fy);
}

/* Exposed scalar stage, for the stencil, curvature and force pins. */
void orc_scalar_ops(const orc_params* P, const double* Tbot, const double* Ttop,
                    const double* c, const double* p, const double* T,
                    double* gcx, double* gcy, double* lapc, double* kappa,
                    double* gTx, double* gTy, double* gpx, double* gpy,
                    double* mu, double* Fx, double* Fy) {
  scalar_out o = {gcx, gcy, lapc, kappa, gTx, gTy, gpx, gpy, mu, Fx, Fy};
  scalar_stage(P, Tbot, Ttop, c, p, T, &o);
}

/* Step 1: moments of the (pre-collision) populations. */
static void moments(const orc_params* P, const double* pop, double* c,
                    double* p, double* T, double* jx, double* jy) {
  const size_t N = (size_t)P->nx * P->ny;
#pragma omp parallel for schedule(static)
  for (long long kk = 0; kk < (long long)N; kk++) {
    size_t k = (size_t)kk;
    double sf = 0, sg = 0, sh = 0, sx = 0, sy = 0;
    for (int i = 0; i < 9; i++) {
      double f = pop[(size_t)i * N + k];
      sf += f;
      sx += EX[i] * f;
      sy += EY[i] * f;
      sg += pop[(size_t)(9 + i) * N + k];
      sh += pop[(size_t)(18 + i) * N + k];
    }
    c[k] = sg;           /* Eq. 28 */
    p[k] = sf;           /* Eq. 13 without (dt/2) u.grad(rho cs2): see p_correct */
    T[k] = sh / (rho_of(P, sg) * P->cv); /* Eq. aEq13 */
    jx[k] = sx;
    jy[k] = sy;
  }
}

/* Eq. 13 with a varying density: p = sum f_i + (dt/2) u.grad(rho cs2), with
 * grad(rho cs2) = cs2 (rho2 - rho1) grad c (the isotropic gradient of the
 * interpolated density: the stencil is linear).  p is corrected in place. */
static void p_correct(const orc_params* P, const double* c, const double* ux,
                      const double* uy, const scalar_out* o, double* p) {
  const size_t N = (size_t)P->nx * P->ny;
  const double dr = CS2 * (P->rho2 - P->rho);
  (void)c;
  for (size_t k = 0; k < N; k++)
    p[k] = p[k] + 0.5 * (ux[k] * (dr * o->gcx[k]) + uy[k] * (dr * o->gcy[k]));
}

/* The isotropic gradient of a cell field whose ghost rows mirror (as p's). */
static void grad_mirrored(const orc_params* P, const double* Tbot, const double* Ttop,
                          const double* v, double* gx, double* gy) {
  const int nx = P->nx, ny = P->ny;
  ext_field e = ext_new(nx, ny, 1);
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) *ext_at(&e, x, y) = v[(size_t)y * nx + x];
  fill_ghosts(P, &e, 0, Tbot, Ttop);
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      size_t k = (size_t)y * nx + x;
      grad_iso(&e, x, y, &gx[k], &gy[k]);
    }
  free(e.v);
}

/* Macroscopic fields (c, p, u, T) of a population state. */
void orc_fields(const orc_params* P, const double* Tbot, const double* Ttop,
                const double* pop, double* c, double* p, double* ux,
                double* uy, double* T) {
  const size_t N = (size_t)P->nx * P->ny;
  double* jx = calloc(N, sizeof(double));
  double* jy = calloc(N, sizeof(double));
  moments(P, pop, c, p, T, jx, jy);
  scalar_out o = scalar_out_new(N);
  scalar_stage(P, Tbot, Ttop, c, p, T, &o);
  for (size_t k = 0; k < N; k++) {
    const double rho = rho_of(P, c[k]);
    ux[k] = jx[k] / (rho * CS2) + 0.5 * o.Fx[k] / rho;
    uy[k] = jy[k] / (rho * CS2) + 0.5 * o.Fy[k] / rho;
  }
  if (varying_rho(P) && !(P->ablate & 2)) p_correct(P, c, ux, uy, &o, p);
  scalar_out_free(&o);
  free(jx);
  free(jy);
}

/* One time step: in (pre-collision state at t) -> out (pre-collision at t+1). */
static void step_once(const orc_params* P, const double* Tbot,
                      const double* Ttop, const double* in, double* out,
                      double* post, double* c, double* p, double* T,
                      double* jx, double* jy, scalar_out* o) {
  const int nx = P->nx, ny = P->ny;
  const size_t N = (size_t)nx * ny;
  const double cv = P->cv;
  const int vrho = varying_rho(P);
  const double dr = CS2 * (P->rho2 - P->rho); /* grad(rho cs2) = dr grad c */

  moments(P, in, c, p, T, jx, jy);
  scalar_stage(P, Tbot, Ttop, c, p, T, o);
  if (vrho && !(P->ablate & 2)) {
    /* Eq. 13: p needs u, u needs F, F needs no p; grad p is then taken of
       the corrected p */
    double* ux = malloc(N * sizeof(double));
    double* uy = malloc(N * sizeof(double));
    for (size_t k = 0; k < N; k++) {
      const double rho = rho_of(P, c[k]);
      ux[k] = jx[k] / (rho * CS2) + 0.5 * o->Fx[k] / rho;
      uy[k] = jy[k] / (rho * CS2) + 0.5 * o->Fy[k] / rho;
    }
    p_correct(P, c, ux, uy, o, p);
    grad_mirrored(P, Tbot, Ttop, p, o->gpx, o->gpy);
    free(ux);
    free(uy);
  }

  /* velocity gradients of every cell for the dissipation term (the same u
     as the collision's; ghost rows antisymmetric: no slip at the walls) */
  double* du = NULL;
  if (P->dissip) {
    du = malloc(4 * N * sizeof(double));
    ext_field uxE = ext_new(nx, ny, 1), uyE = ext_new(nx, ny, 1);
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        const size_t k = (size_t)y * nx + x;
        const double rho = rho_of(P, c[k]);
        *ext_at(&uxE, x, y) = jx[k] / (rho * CS2) + 0.5 * o->Fx[k] / rho;
        *ext_at(&uyE, x, y) = jy[k] / (rho * CS2) + 0.5 * o->Fy[k] / rho;
      }
    fill_ghosts(P, &uxE, 3, Tbot, Ttop);
    fill_ghosts(P, &uyE, 3, Tbot, Ttop);
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        const size_t k = (size_t)y * nx + x;
        grad_iso(&uxE, x, y, &du[k], &du[N + k]);
        grad_iso(&uyE, x, y, &du[2 * N + k], &du[3 * N + k]);
      }
    free(uxE.v);
    free(uyE.v);
  }

  const double omega_g = 1.0 / P->tau_g;             /* Eq. 27 */
  const double Gm = P->mobility / (P->tau_g - 0.5);  /* M = Gamma (tau_g - 1/2), Eq. 16 */

#pragma omp parallel for schedule(static)
  for (long long kk = 0; kk < (long long)N; kk++) {
    size_t k = (size_t)kk;
    double cc = c[k], TT = T[k];
    const double rho = rho_of(P, cc);
    /* properties, linear in c */
    double eta = prop_of(P, P->eta1, P->eta2, cc);
    double lam = prop_of(P, P->lam1, P->lam2, cc);
    double tau_f = eta / (rho * CS2) + 0.5;
    double omega_f = 1.0 / tau_f;
    double tau_h = lam / (rho * cv * CS2);
    double omega_T = 2.0 / (2.0 * tau_h + 1.0);

    double Fx = o->Fx[k], Fy = o->Fy[k];
    double ux = jx[k] / (rho * CS2) + 0.5 * Fx / rho;
    double uy = jy[k] / (rho * CS2) + 0.5 * Fy / rho;
    const double dRx = dr * o->gcx[k], dRy = dr * o->gcy[k];
    /* the work / dissipation term of Eq. aEq7 per direction, and its sum */
    double ws[9], ws0 = 0.0;
    if (du) {
      const double dk[4] = {du[k], du[N + k], du[2 * N + k], du[3 * N + k]};
      for (int i = 0; i < 9; i++) {
        ws[i] = work_source(i, rho, p[k], in[(size_t)i * N + k], omega_f, ux, uy, dk);
        ws0 += ws[i];
      }
    }
    for (int i = 0; i < 9; i++) {
      double f = in[(size_t)i * N + k];
      double feq = f_equilibrium(i, p[k], rho, ux, uy);
      post[(size_t)i * N + k] =
          f - omega_f * (f - feq) +
          (1.0 - 0.5 * omega_f) *
              f_source(i, Fx, Fy, ux, uy, dRx, dRy, vrho && !(P->ablate & 1));

      double g = in[(size_t)(9 + i) * N + k];
      double geq = g_equilibrium(i, cc, o->mu[k], Gm, ux, uy);
      post[(size_t)(9 + i) * N + k] =
          g - omega_g * (g - geq) +
          (1.0 - 0.5 * omega_g) *
              g_source(i, cc, rho, Fx, Fy, o->gpx[k], o->gpy[k], ux, uy);

      double h = in[(size_t)(18 + i) * N + k];
      double heq = h_equilibrium(i, rho, cv, TT, ux, uy);
      double hs = h_source(i, rho, cv, TT, Fx, Fy, o->gpx[k], o->gpy[k], ux, uy, dRx, dRy,
                           vrho && !(P->ablate & 4));
      if (du) {
        post[(size_t)(18 + i) * N + k] = h - omega_T * (h - heq) +
                                         (1.0 - 0.5 * omega_T) * (hs + (ws[i] - W[i] * ws0)) +
                                         W[i] * ws0;
      } else {
        post[(size_t)(18 + i) * N + k] = h - omega_T * (h - heq) + (1.0 - 0.5 * omega_T) * hs;
      }
    }
  }

  free(du);

  /* streaming, pull form: P_i(x, t+1) = P*_i(x - xi_i, t); f and g first,
     then hbar, whose anti-bounce-back at a wall takes rho of the cell's new
     c (the c the next step's moments see; with a varying density this is
     the density the wall term needs at the time the pull applies it) */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      size_t k = (size_t)y * nx + x;
      for (int pass = 0; pass < 2; pass++)
      for (int i = 0; i < 9; i++) {
        int xs = ((x - EX[i]) % nx + nx) % nx;
        int ys = y - EY[i];
        int wall = 0;
        if (P->periodic_y)
          ys = ((ys % ny) + ny) % ny;
        else if (ys < 0 || ys >= ny)
          wall = 1;
        if (!wall) {
          size_t ks = (size_t)ys * nx + xs;
          if (pass == 0) {
            out[(size_t)i * N + k] = post[(size_t)i * N + ks];
            out[(size_t)(9 + i) * N + k] = post[(size_t)(9 + i) * N + ks];
          } else {
            out[(size_t)(18 + i) * N + k] = post[(size_t)(18 + i) * N + ks];
          }
        } else {
          /* halfway bounce-back: the population that left this cell towards
             the wall returns reversed one step later */
          int o_ = OPP[i];
          const double* Twall = (ys < 0) ? Tbot : Ttop;
          double Tw = Twall[x];
          if (P->wall_mid && EX[i] != 0) /* the link crosses the wall at x - xi_x/2 */
            Tw = 0.5 * (Twall[x] + Twall[((x - EX[i]) % nx + nx) % nx]);
          if (pass == 0) {
            out[(size_t)i * N + k] = post[(size_t)o_ * N + k];
            out[(size_t)(9 + i) * N + k] = post[(size_t)(9 + o_) * N + k];
          } else {
            /* anti-bounce-back fixes T = T_w at the wall (u = 0 there) */
            double cn = 0.0;
            for (int j = 0; j < 9; j++) cn += out[(size_t)(9 + j) * N + k];
            out[(size_t)(18 + i) * N + k] =
                -post[(size_t)(18 + o_) * N + k] + 2.0 * W[i] * rho_of(P, cn) * cv * Tw;
          }
        }
      }
    }
}

/* Run nsteps from pop_in; the result is written to pop_out (may alias). */
int orc_run(const orc_params* P, const double* Tbot, const double* Ttop,
            const double* pop_in, double* pop_out, int64_t nsteps) {
  if (P->nx < 1 || P->ny < 2 || nsteps < 0) return -1;
  const size_t N = (size_t)P->nx * P->ny;
  double* a = malloc(27 * N * sizeof(double));
  double* b = malloc(27 * N * sizeof(double));
  double* post = malloc(27 * N * sizeof(double));
  double *c = malloc(N * sizeof(double)), *p = malloc(N * sizeof(double)),
         *T = malloc(N * sizeof(double)), *jx = malloc(N * sizeof(double)),
         *jy = malloc(N * sizeof(double));
  if (!a || !b || !post || !c || !p || !T || !jx || !jy) return -2;
  scalar_out o = scalar_out_new(N);
  memcpy(a, pop_in, 27 * N * sizeof(double));
  for (int64_t n = 0; n < nsteps; n++) {
    step_once(P, Tbot, Ttop, a, b, post, c, p, T, jx, jy, &o);
    double* t = a;
    a = b;
    b = t;
  }
  memcpy(pop_out, a, 27 * N * sizeof(double));
  scalar_out_free(&o);
  free(a); free(b); free(post); free(c); free(p); free(T); free(jx); free(jy);
  return 0;
}

/* Initial state: u = 0, p = 0, c = c0, T = T0.
 * f_i = f_eq(p=0, u=0) = 0; g_i = g_eq(c0, mu(c0), u=0) with the discrete
 * Laplacian of c0; hbar_i = h_eq(T0, u=0) = w_i rho c_v T0. */
int orc_init(const orc_params* P, const double* c0, const double* T0,
             const double* Tbot, const double* Ttop, double* pop) {
  if (P->nx < 1 || P->ny < 2) return -1;
  const size_t N = (size_t)P->nx * P->ny;
  double* zero = calloc(N, sizeof(double));
  scalar_out o = scalar_out_new(N);
  scalar_stage(P, Tbot, Ttop, c0, zero, T0, &o);
  const double Gm = P->mobility / (P->tau_g - 0.5);
  for (size_t k = 0; k < N; k++) {
    for (int i = 0; i < 9; i++) {
      pop[(size_t)i * N + k] = f_equilibrium(i, 0.0, P->rho, 0.0, 0.0);
      pop[(size_t)(9 + i) * N + k] = g_equilibrium(i, c0[k], o.mu[k], Gm, 0.0, 0.0);
      pop[(size_t)(18 + i) * N + k] =
          h_equilibrium(i, rho_of(P, c0[k]), P->cv, T0[k], 0.0, 0.0);
    }
  }
  scalar_out_free(&o);
  free(zero);
  return 0;
}

/* Threads the OpenMP runtime will use (reported beside CPU timings). */
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads for the following calls (n <= 0: one per processor), for the
 * one-thread and all-core timings of the CPU baseline.  The arithmetic and
 * its result do not depend on it. */
void orc_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
  (void)n;
#endif
}

"""Seeded synthetic workloads: parameters, initial and wall fields.

This module builds the *inputs* of a run and nothing else: lattice-unit
parameters derived from the dimensionless groups of each problem, the initial
order parameter (a tanh profile of width W), the initial temperature and the
wall temperature tables.  It holds none of the method's arithmetic
(equilibria, stencils, collision, streaming), so the CUDA path and the CPU
oracle can both take their inputs from it.

Conventions (lattice units, dx = dt = 1):

* cells x = 0..nx-1 (periodic), y = 0..ny-1; walls lie half a cell outside,
  at y = -1/2 and y = ny - 1/2;
* phase c = 0 has (eta1, lam1), phase c = 1 has (eta2, lam2); a drop is the
  phase c = 1; ratios are drop / matrix;
* sigma = sigma0 - sigmaT (T - Tref) with sigmaT > 0 (the paper's d sigma/dT
  is -sigmaT, Eq. aEq3);
* the planar equilibrium profile of Sec. II, c = (1 + tanh(d / (2 sqrt 2 eps)))/2
  with d the signed distance into phase 1, is written with the width
  W = 4 sqrt(2) eps, i.e. c = (1 + tanh(2 d / W)) / 2.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    params: dict          # lattice parameters incl. nx, ny (see PARAM_KEYS)
    c0: np.ndarray        # (ny, nx) float64
    T0: np.ndarray        # (ny, nx) float64
    Tbot: np.ndarray      # (nx,) float64, wall temperature at y = -1/2
    Ttop: np.ndarray      # (nx,) float64, wall temperature at y = ny - 1/2
    steps: int            # step count of the problem as stated
    info: dict = dataclasses.field(default_factory=dict)

    @property
    def nx(self) -> int:
        return int(self.params["nx"])

    @property
    def ny(self) -> int:
        return int(self.params["ny"])

    @property
    def cells(self) -> int:
        return self.nx * self.ny


PARAM_KEYS = ("rho", "cv", "eta1", "eta2", "lam1", "lam2", "sigma0", "sigmaT",
              "Tref", "eps", "beta", "tau_g", "mobility", "ax", "ay", "eta_n")


def base_params(nx: int, ny: int, **kw) -> dict:
    p = dict(nx=int(nx), ny=int(ny), rho=1.0, cv=1.0, eta1=0.1, eta2=0.1,
             lam1=0.1, lam2=0.1, sigma0=0.0, sigmaT=0.0, Tref=0.0,
             eps=4.0 / (4.0 * math.sqrt(2.0)), beta=0.25, tau_g=1.0,
             mobility=0.1, ax=0.0, ay=0.0, eta_n=1e-12)
    p.update(kw)
    return p


def eps_from_width(W: float) -> float:
    return W / (4.0 * math.sqrt(2.0))


# The transcendental functions of the input fields are evaluated with IEEE
# basic operations only (+, -, *, /, rounding to an integer and exact scaling
# by powers of two), each correctly rounded on every platform, so that the
# inputs -- and the hashes of stored FP64 end states -- are bitwise the same
# on every machine.  (numpy's own tanh and cos differ in the last bits
# between its x86 SIMD and Arm builds.)
_INV_LN2 = 1.0 / math.log(2.0)
_LN2_HI = 6.93147180369123816490e-01  # ln 2 with its low 32 mantissa bits zero
_LN2_LO = 1.90821492927058770002e-10  # ln 2 - _LN2_HI
_EXP_C = [1.0 / math.factorial(n) for n in range(14)]
_COS_C = [(-1.0) ** n / math.factorial(2 * n) for n in range(10)]
_SIN_C = [(-1.0) ** n / math.factorial(2 * n + 1) for n in range(9)]


def det_exp(x) -> np.ndarray:
    """exp(x): x = k ln 2 + r with |r| <= ln2/2 (Cody-Waite split of ln 2,
    k ln2_hi exact for |k| < 2^21), Taylor polynomial of degree 13 in r
    (truncation below 1e-17 relative), times 2^k (overflow to inf, underflow
    through the subnormals to 0)."""
    # beyond +-1100 the result is inf or 0 either way
    x = np.clip(np.asarray(x, dtype=np.float64), -1100.0, 1100.0)
    k = np.round(x * _INV_LN2)
    r = (x - k * _LN2_HI) - k * _LN2_LO
    p = np.full_like(r, _EXP_C[13])
    for n in range(12, -1, -1):
        p = p * r + _EXP_C[n]
    with np.errstate(over="ignore", under="ignore"):
        return np.ldexp(p, k.astype(np.int64))


def det_cos2pi(q) -> np.ndarray:
    """cos(2 pi q): q reduced to [-1/2, 1/2] and to the first octant by exact
    differences, then the Taylor polynomial of cos or sin (degree 18 / 17,
    |argument| <= pi/4, truncation below 1e-17)."""
    q = np.asarray(q, dtype=np.float64)
    a = np.abs(q - np.round(q))
    two_pi = 2.0 * math.pi

    def cos_p(t):
        s = t * t
        p = np.full_like(t, _COS_C[9])
        for n in range(8, -1, -1):
            p = p * s + _COS_C[n]
        return p

    def sin_p(t):
        s = t * t
        p = np.full_like(t, _SIN_C[8])
        for n in range(7, -1, -1):
            p = p * s + _SIN_C[n]
        return t * p

    out = np.empty_like(a)
    m1 = a <= 0.125
    m3 = a > 0.375
    m2 = ~(m1 | m3)
    out[m1] = cos_p(two_pi * a[m1])
    out[m2] = sin_p(two_pi * (0.25 - a[m2]))
    out[m3] = -cos_p(two_pi * (0.5 - a[m3]))
    return out


def tanh_profile(d: np.ndarray, W: float) -> np.ndarray:
    """(1 + tanh(2 d / W)) / 2, evaluated as 1 / (1 + exp(-4 d / W))."""
    return 1.0 / (1.0 + det_exp(-4.0 * np.asarray(d, dtype=np.float64) / W))


def linear_T(nx: int, ny: int, Tbot, Ttop) -> np.ndarray:
    """Conduction profile between the walls at y = -1/2 and y = ny - 1/2."""
    Tb = np.broadcast_to(np.asarray(Tbot, dtype=np.float64), (nx,))
    Tt = np.broadcast_to(np.asarray(Ttop, dtype=np.float64), (nx,))
    s = (np.arange(ny, dtype=np.float64) + 0.5)[:, None] / ny
    return np.ascontiguousarray(Tb[None, :] + (Tt - Tb)[None, :] * s)


def _drop_distance(nx, ny, R, xc, yc):
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    dx = x - xc
    dx = dx - nx * np.round(dx / nx)  # nearest periodic image in x
    return R - np.sqrt(dx * dx + (y - yc) ** 2)


# ---------------------------------------------------------------- problems

def layered_poiseuille(nx: int = 4, ny: int = 101, eta1=0.1, eta2=0.2,
                       lam1=0.1, lam2=0.2, T_bottom=1.0, T_top=0.0,
                       umax=1e-3, W=4.0, sigma0=1e-3, sigmaT=1e-4,
                       mobility=0.1, steps=20000) -> Workload:
    """Two-layer thermal Poiseuille flow (Sec. IV.A): phase 0 in the lower
    half, phase 1 in the upper half, interface on row (ny-1)/2, body force
    a_x set so that the Eq. 32 profile peaks at ``umax``."""
    yi = (ny - 1) / 2.0
    h = H = ny / 2.0
    # max of Eq. 32 on a fine grid for a_x = 1, then scale
    yy = np.linspace(-h, H, 20001)
    e1, e2 = eta1, eta2
    lo = h * h / (2 * e1) * (-(yy / h) ** 2 + ((H * H / (h * h) * e1 - e2) / (H / h * e1 + e2)) * (yy / h)
                             + (1 + H / h) * H * e1 / (e1 * H + e2 * h))
    up = H * H / (2 * e2) * (-(yy / H) ** 2 + ((e1 - h * h / (H * H) * e2) / (e1 + h / H * e2)) * (yy / H)
                             + (1 + h / H) * h * e2 / (e1 * H + e2 * h))
    u1 = np.where(yy <= 0, lo, up).max()
    ax = umax / u1
    p = base_params(nx, ny, eta1=eta1, eta2=eta2, lam1=lam1, lam2=lam2,
                    sigma0=sigma0, sigmaT=sigmaT, Tref=0.0, eps=eps_from_width(W),
                    mobility=mobility, ax=ax)
    d = (np.arange(ny, dtype=np.float64) - yi)[:, None] * np.ones((1, nx))
    c0 = np.ascontiguousarray(tanh_profile(d, W))
    Tb = np.full(nx, float(T_bottom))
    Tt = np.full(nx, float(T_top))
    return Workload("layered_poiseuille_%dx%d" % (nx, ny), p, c0,
                    linear_T(nx, ny, Tb, Tt), Tb, Tt, steps,
                    dict(h=h, H=H, y_interface=yi, umax=umax))


def planar_marangoni(nx: int = 512, ny: int = 256, eta=0.2, lam_upper=0.2,
                     lam_lower=0.2, eta_upper=None, Th=20.0, Tc=10.0, Tr=4.0,
                     sigma0=2.5e-2, sigmaT=5e-4, eps=1.0, mobility=5e-2,
                     steps=100000) -> Workload:
    """Two superimposed planar fluids heated by a sinusoidal bottom wall
    (Sec. IV.B): T(-h, x) = Th + Tr cos(2 pi x / nx), T(H) = Tc, interface
    midway between rows ny/2-1 and ny/2, phase 1 above."""
    eta_upper = eta if eta_upper is None else eta_upper
    yi = ny / 2.0 - 0.5
    W = 4.0 * math.sqrt(2.0) * eps
    p = base_params(nx, ny, eta1=eta, eta2=eta_upper, lam1=lam_lower,
                    lam2=lam_upper, sigma0=sigma0, sigmaT=sigmaT, Tref=Tc,
                    eps=eps, mobility=mobility)
    d = (np.arange(ny, dtype=np.float64) - yi)[:, None] * np.ones((1, nx))
    c0 = np.ascontiguousarray(tanh_profile(d, W))
    x = np.arange(nx, dtype=np.float64)
    Tb = Th + Tr * det_cos2pi(x / nx)
    Tt = np.full(nx, float(Tc))
    return Workload("planar_marangoni_%dx%d" % (nx, ny), p, c0,
                    linear_T(nx, ny, Tb, Tt), Tb, Tt, steps,
                    dict(h=ny / 2.0, H=ny / 2.0, y_interface=yi, L=nx, Th=Th,
                         Tc=Tc, Tr=Tr))


def droplet(nx: int, ny: int, R: float, xc: float, yc: float, Re: float,
            Ma: float, Ca: float, eta_m: float, eta_r: float, lam_r: float,
            gradT: float = 1e-3, W: float = 4.0, mobility: float = 0.1,
            steps: int = 0, dT0: np.ndarray | None = None,
            name: str | None = None, sigmaT: float | None = None) -> Workload:
    """Thermocapillary migration of one 2D drop (Sec. IV.C): drop (phase 1)
    of radius R at (xc, yc); walls at T = 0 (bottom) and T = gradT (ny-1)
    (top), linear conduction profile at t = 0 (plus an optional perturbation
    dT0).  Lattice parameters from the dimensionless groups with the velocity
    scale U of Eq. 43:

      U = eta_m Re / (rho R)      (Re = rho U R / eta_m)
      sigmaT = U eta_m / (gradT R)
      sigma0 = U eta_m / Ca       (Ca = U eta_m / sigma0)
      lam_m = U R / Ma            (Ma = U R rho c_v / lam_m)

    If ``sigmaT`` is given, U follows from it instead of from Re."""
    if sigmaT is None:
        U = eta_m * Re / R
        sigmaT = U * eta_m / (gradT * R)
    else:
        U = sigmaT * gradT * R / eta_m
    sigma0 = U * eta_m / Ca
    lam_m = U * R / Ma
    Ttop = gradT * (ny - 1)
    Tref = Ttop * (yc + 0.5) / ny
    p = base_params(nx, ny, eta1=eta_m, eta2=eta_r * eta_m, lam1=lam_m,
                    lam2=lam_r * lam_m, sigma0=sigma0, sigmaT=sigmaT, Tref=Tref,
                    eps=eps_from_width(W), mobility=mobility)
    c0 = np.ascontiguousarray(tanh_profile(_drop_distance(nx, ny, R, xc, yc), W))
    Tb = np.zeros(nx)
    Tt = np.full(nx, Ttop)
    T0 = linear_T(nx, ny, Tb, Tt)
    if dT0 is not None:
        T0 = np.ascontiguousarray(T0 + dT0)
    info = dict(R=R, xc=xc, yc=yc, U=U, Re=U * R / eta_m, Ma=Ma, Ca=Ca,
                gradT=gradT, eta_r=eta_r, lam_r=lam_r)
    return Workload(name or "droplet_%dx%d" % (nx, ny), p, c0, T0, Tb, Tt, steps,
                    info)


def droplet_512x1024(steps: int = 40000) -> Workload:
    """Drop of radius 32 at (256, 256) in 512 x 1024, ratios 0.5, Re = 1,
    Ma = 10, Ca = 0.05, eta_m = 0.2, |grad T| = 1e-3, W = 4."""
    return droplet(512, 1024, 32.0, 256.0, 256.0, Re=1.0, Ma=10.0, Ca=0.05,
                   eta_m=0.2, eta_r=0.5, lam_r=0.5, steps=steps)


def droplet_scaled(nx: int, ny: int, steps: int = 200) -> Workload:
    """The 512 x 1024 drop scaled to a larger grid: R = nx/16, centre
    (nx/2, ny/4), same Re, Ma, Ca and ratios."""
    return droplet(nx, ny, nx / 16.0, nx / 2.0, ny / 4.0, Re=1.0, Ma=10.0,
                   Ca=0.05, eta_m=0.2, eta_r=0.5, lam_r=0.5, steps=steps)


BATCH_GRIDS = ((128, 256), (256, 512), (512, 1024), (768, 1536))


def batch_sweep(n: int = 64, seed: int = 0, steps: int = 10000,
                grids=BATCH_GRIDS) -> list:
    """Parameter sweep of ``n`` drops: per instance, in this order, a grid
    drawn uniformly from ``grids``, Ma ~ U[1, 50], Ca ~ U[0.01, 0.2],
    sigmaT ~ U[1e-5, 1e-3], eta_r ~ U[0.25, 4], lam_r ~ U[0.25, 4]
    (numpy default_rng(seed)); R = nx/8 at (nx/2, ny/4); |grad T| = 1e-3,
    eta_m = 0.1."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(n):
        gi = int(rng.integers(0, len(grids)))
        Ma = float(rng.uniform(1.0, 50.0))
        Ca = float(rng.uniform(0.01, 0.2))
        sT = float(rng.uniform(1e-5, 1e-3))
        er = float(rng.uniform(0.25, 4.0))
        lr = float(rng.uniform(0.25, 4.0))
        nx, ny = grids[gi]
        out.append(droplet(nx, ny, nx / 8.0, nx / 2.0, ny / 4.0, Re=0.0, Ma=Ma,
                           Ca=Ca, eta_m=0.1, eta_r=er, lam_r=lr, sigmaT=sT,
                           steps=steps, name="sweep%02d_%dx%d" % (j, nx, ny)))
    return out


def migration_256x512(steps: int = 2000, seed: int = 1, amp: float = 1e-4,
                      nx: int = 256, ny: int = 512, R: float = 24.0,
                      xc: float = 128.0, yc: float = 128.0) -> Workload:
    """Drop for the differentiable-migration problem: R = 24 at (128, 128) in
    256 x 512, Re = 1, Ma = 10, Ca = 0.05, eta_m = 0.2, ratios 1, plus an
    i.i.d. Gaussian initial temperature perturbation of standard deviation
    ``amp`` drawn by default_rng(seed) in [ny][nx] order."""
    rng = np.random.default_rng(seed)
    dT0 = rng.normal(0.0, amp, size=(ny, nx))
    return droplet(nx, ny, R, xc, yc, Re=1.0, Ma=10.0, Ca=0.05, eta_m=0.2,
                   eta_r=1.0, lam_r=1.0, steps=steps, dT0=dT0,
                   name="migration_%dx%d" % (nx, ny))


def migration_tiny(steps: int = 2000, seed: int = 1, amp: float = 1e-4) -> Workload:
    """32 x 64 version of the migration problem (R = 8 at (16, 16))."""
    return migration_256x512(steps=steps, seed=seed, amp=amp, nx=32, ny=64,
                             R=8.0, xc=16.0, yc=16.0)

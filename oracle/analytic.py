"""Closed-form solutions the paper uses to validate the scheme (Sec. IV).

TEST INFRASTRUCTURE ONLY (part of the oracle package).

* Two-layer thermal Poiseuille flow: steady u_x(y), Eq. 32, and T(y), Eq. 33;
  the same flow with layers of unequal density under a body force rho a.
* Two superimposed planar fluids with a sinusoidal wall temperature (Pendse and
  Esmaeeli, as restated in Sec. IV.B), with three misprints read as follows:
  "cost(kx)" is cos(kx); the first of the two printed C^h_2 is C^h_1; C^h_3 is
  the mirror image of C^H_3, (sinh 2b - 2b) / (2 [sinh^2 b - b^2]), which is
  the only reading that satisfies no-slip at y = -h (checked in the tests).
* Young-Goldstein-Block migration velocity, Eq. 42 and Eq. 43.

Sign convention: ``sigma_T_paper`` is the paper's d sigma / d T (negative for
the usual fluids, Eq. aEq3).
"""
from __future__ import annotations

import numpy as np


def poiseuille_u(y, h, H, eta_lower, eta_upper, rho, ax):
    """Eq. 32: steady u_x of two layers -h <= y <= 0 (viscosity eta_lower) and
    0 <= y <= H (eta_upper), no slip at y = -h and y = H, body force rho*ax."""
    y = np.asarray(y, dtype=np.float64)
    e1, e2 = eta_lower, eta_upper
    lo = rho * ax * h * h / (2 * e1) * (
        -(y / h) ** 2
        + ((H * H / (h * h) * e1 - e2) / (H / h * e1 + e2)) * (y / h)
        + (1 + H / h) * H * e1 / (e1 * H + e2 * h))
    up = rho * ax * H * H / (2 * e2) * (
        -(y / H) ** 2
        + ((e1 - h * h / (H * H) * e2) / (e1 + h / H * e2)) * (y / H)
        + (1 + h / H) * h * e2 / (e1 * H + e2 * h))
    return np.where(y <= 0, lo, up)


def poiseuille_u_rho(y, h, H, eta_lower, eta_upper, rho_lower, rho_upper, ax):
    """Steady u_x of two layers of unequal density under the body force
    rho_k ax of each: eta_k u'' = -rho_k ax in each layer, no slip at y = -h
    and y = H, u and eta u' continuous at y = 0.  With rho_lower = rho_upper
    this is Eq. 32.  u_k = -rho_k ax y^2 / (2 eta_k) + A_k y + B with
    eta_lower A_lower = eta_upper A_upper and B from the wall conditions."""
    y = np.asarray(y, dtype=np.float64)
    e1, e2, r1, r2 = eta_lower, eta_upper, rho_lower, rho_upper
    A1 = (r2 * ax * H * H / (2 * e2) - r1 * ax * h * h / (2 * e1)) / (h + e1 * H / e2)
    A2 = e1 * A1 / e2
    B = r1 * ax * h * h / (2 * e1) + A1 * h
    lo = -r1 * ax * y * y / (2 * e1) + A1 * y + B
    up = -r2 * ax * y * y / (2 * e2) + A2 * y + B
    return np.where(y <= 0, lo, up)


def poiseuille_T(y, h, H, lam_lower, lam_upper, T_bottom, T_top):
    """Eq. 33 with the wall temperatures named by position: T(-h) = T_bottom,
    T(H) = T_top (the paper's T_c is at the bottom and T_h at the top)."""
    y = np.asarray(y, dtype=np.float64)
    l1, l2 = lam_lower, lam_upper
    D = l1 * H + l2 * h
    Ti = (l1 * H * T_bottom + l2 * h * T_top) / D
    lo = l2 * (T_top - T_bottom) / D * y + Ti
    up = l1 * (T_top - T_bottom) / D * y + Ti
    return np.where(y <= 0, lo, up)


def pendse_constants(L, h, H, eta_upper, eta_lower, lam_upper, lam_lower,
                     Tr, sigma_T_paper):
    k = 2 * np.pi / L
    a, b = H * k, h * k
    eta_r = eta_upper / eta_lower
    lam_r = lam_upper / lam_lower
    Da = np.sinh(a) ** 2 - a * a
    Db = np.sinh(b) ** 2 - b * b
    f = 1.0 / (lam_r * np.cosh(a) * np.sinh(b) + np.sinh(a) * np.cosh(b))
    g = np.sinh(a) * f
    hfun = Da * Db / (eta_r * Db * (np.sinh(2 * a) - 2 * a) + Da * (np.sinh(2 * b) - 2 * b))
    Umax = -Tr * sigma_T_paper / eta_lower * g * hfun
    CH = (np.sinh(a) ** 2 / Da, -H * a / Da, (2 * a - np.sinh(2 * a)) / (2 * Da))
    Ch = (np.sinh(b) ** 2 / Db, -h * b / Db, (np.sinh(2 * b) - 2 * b) / (2 * Db))
    return dict(k=k, alpha=a, beta=b, eta_r=eta_r, lam_r=lam_r, f=f, g=g,
                hfun=hfun, Umax=Umax, CH=CH, Ch=Ch)


def pendse(x, y, L, h, H, eta_upper, eta_lower, lam_upper, lam_lower, Tc, Th,
           Tr, sigma_T_paper):
    """Velocity (ux, uy) and temperature T of two planar layers, fluid 1 above
    (0 <= y <= H), fluid 2 below (-h <= y <= 0), T(H) = Tc,
    T(-h) = Th + Tr cos(kx), k = 2 pi / L (Sec. IV.B)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    K = pendse_constants(L, h, H, eta_upper, eta_lower, lam_upper, lam_lower, Tr,
                         sigma_T_paper)
    k, U, f, a, lr = K["k"], K["Umax"], K["f"], K["alpha"], K["lam_r"]

    def vel(C):
        C1, C2, C3 = C
        ux = U * ((C1 + k * (C2 + C3 * y)) * np.cosh(k * y)
                  + (C3 + k * C1 * y) * np.sinh(k * y)) * np.sin(k * x)
        uy = -k * U * (C1 * y * np.cosh(k * y)
                       + (C2 + C3 * y) * np.sinh(k * y)) * np.cos(k * x)
        return ux, uy

    uxu, uyu = vel(K["CH"])
    uxl, uyl = vel(K["Ch"])
    Tu = ((Tc - Th) * y + lr * Tc * h + Th * H) / (H + lr * h) \
        + Tr * f * np.sinh(a - k * y) * np.cos(k * x)
    Tl = (lr * (Tc - Th) * y + lr * Tc * h + Th * H) / (H + lr * h) \
        + Tr * f * (np.sinh(a) * np.cosh(k * y) - lr * np.sinh(k * y) * np.cosh(a)) * np.cos(k * x)
    up = y >= 0
    return (np.where(up, uxu, uxl), np.where(up, uyu, uyl), np.where(up, Tu, Tl))


def ygb_velocity(sigma_T_paper, gradT, R, eta_matrix, eta_r, lam_r):
    """Eq. 42 with Eq. 43: U_YGB = 2U / ((2 + lam_r)(2 + 3 eta_r)),
    U = -sigma_T |grad T| R / eta_matrix."""
    U = -sigma_T_paper * gradT * R / eta_matrix
    return 2 * U / ((2 + lam_r) * (2 + 3 * eta_r))

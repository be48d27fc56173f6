"""The oracle against the paper's validation problems (Sec. IV.A, IV.B):
the analytic steady profiles of the two-layer thermal Poiseuille flow
(Eq. 32, Eq. 33) and the Pendse-Esmaeeli planar Marangoni solution.

These agree to the diffuse-interface error only (the analytic solutions have
a sharp interface), so the bounds are the errors expected from an interface
of width W ~ 4-6 cells in a channel of 24-50 cells per layer.  CPU only.
"""
import numpy as np

from oracle import analytic as an
from paper_1412_6238_gb300 import workloads as wl


def _run_to_steady(orc, w, chunk, tol, max_steps):
    pop = orc.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop)
    prev = None
    n = 0
    while n < max_steps:
        pop = orc.run(w.params, pop, w.Tbot, w.Ttop, chunk)
        n += chunk
        F = orc.fields(w.params, pop, w.Tbot, w.Ttop)
        if prev is not None:
            r_u = np.linalg.norm(F["ux"] - prev["ux"]) / np.linalg.norm(F["ux"]) / chunk
            r_T = np.linalg.norm(F["T"] - prev["T"]) / np.linalg.norm(F["T"]) / chunk
            if r_u < tol and r_T < tol:
                return F, n
        prev = F
    raise AssertionError("not steady after %d steps" % n)


def test_layered_poiseuille_matches_eq32_eq33(orc):
    """4 x 101 channel, eta2/eta1 = 2, lam2/lam1 = 2, T = 1 at the bottom wall
    and 0 at the top, u_max = 1e-3: at a per-step residual below 1e-10 the
    velocity matches Eq. 32 and the temperature Eq. 33 (walls half a cell
    outside the first and last rows, h = H = 50.5)."""
    w = wl.layered_poiseuille()
    F, n = _run_to_steady(orc, w, 5000, 1e-10, 300000)
    p = w.params
    y = np.arange(w.ny) - w.info["y_interface"]
    ue = an.poiseuille_u(y, w.info["h"], w.info["H"], p["eta1"], p["eta2"], p["rho"], p["ax"])
    Te = an.poiseuille_T(y, w.info["h"], w.info["H"], p["lam1"], p["lam2"],
                         w.Tbot[0], w.Ttop[0])
    u = F["ux"][:, 0]
    T = F["T"][:, 0]
    assert np.linalg.norm(u - ue) / np.linalg.norm(ue) < 3e-3
    assert np.abs(u - ue).max() < 5e-3 * ue.max()
    assert np.linalg.norm(T - Te) / np.linalg.norm(Te) < 5e-3
    assert np.abs(F["uy"]).max() < 1e-12
    # every column identical (no x dependence)
    assert np.abs(F["ux"] - F["ux"][:, :1]).max() < 1e-15


def test_planar_marangoni_matches_pendse(orc):
    """96 x 48 version of the Sec. IV.B problem (H = h = 24, eps = 1,
    T_h = 20, T_r = 4, T_c = 10, sigma_T = -5e-4 in the paper's sign): the
    steady velocity and temperature follow the closed form; the velocity
    to the O(W/H) diffuse-interface error (about 10 % here), the
    temperature to 1e-3."""
    w = wl.planar_marangoni(96, 48)
    pop = orc.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop)
    pop = orc.run(w.params, pop, w.Tbot, w.Ttop, 20000)
    F = orc.fields(w.params, pop, w.Tbot, w.Ttop)
    p = w.params
    x = np.arange(w.nx)[None, :] * np.ones((w.ny, 1))
    y = (np.arange(w.ny) - w.info["y_interface"])[:, None] * np.ones((1, w.nx))
    ux, uy, T = an.pendse(x, y, w.nx, w.info["h"], w.info["H"], p["eta2"], p["eta1"],
                          p["lam2"], p["lam1"], w.info["Tc"], w.info["Th"], w.info["Tr"],
                          -p["sigmaT"])
    num = np.sqrt(((F["ux"] - ux) ** 2 + (F["uy"] - uy) ** 2).sum())
    assert num / np.sqrt((ux ** 2 + uy ** 2).sum()) < 0.12
    corr = (F["ux"] * ux + F["uy"] * uy).sum() / np.sqrt(
        (F["ux"] ** 2 + F["uy"] ** 2).sum() * (ux ** 2 + uy ** 2).sum())
    assert corr > 0.99
    assert np.linalg.norm(F["T"] - T) / np.linalg.norm(T) < 1e-3

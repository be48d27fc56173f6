"""Differentiable drop migration through the library's discrete adjoint.

``LBEMigration.apply(sigmaT, eta_ratio, lam_ratio, dT0, problem)`` returns the
migration loss of a thermocapillary drop (Sec. IV.C): the mean over the last
``window`` of ``steps`` states of the phase-1 centroid velocity
sum(c u_y) / sum(c).  Its backward gives the gradient with respect to the
surface-tension temperature coefficient sigmaT (Eq. aEq3), the viscosity and
conductivity ratios eta2/eta1 and lam2/lam1 (eta1, lam1 held fixed) and the
per-cell initial temperature perturbation dT0 (T(x, 0) = T0(x) + dT0(x)).

The forward and the reverse sweep both run inside ``lbe_adjoint``: the
forward stores a raw checkpoint every ``ckpt_every`` steps, the reverse
sweep recomputes each segment from its checkpoint and back-propagates
through it in FP64.  The gradient is computed during the forward call (one
library call for both) and scaled by the incoming gradient in backward.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import lbe as _lbe


@dataclasses.dataclass
class MigrationProblem:
    workload: object          # workloads.Workload: params, c0, T0 (unperturbed), walls
    steps: int = 2000
    window: int = 200
    ckpt_every: int = 100
    storage: str = "f32"


def _scalar(t) -> float:
    return float(t.detach().cpu().item()) if torch.is_tensor(t) else float(t)


def migration_handle(problem: MigrationProblem, sigmaT: float, eta_ratio: float,
                     lam_ratio: float, dT0: np.ndarray):
    """Handle of the migration problem at the given parameters."""
    w = problem.workload
    p = dict(w.params)
    p["sigmaT"] = float(sigmaT)
    p["eta2"] = float(eta_ratio) * p["eta1"]
    p["lam2"] = float(lam_ratio) * p["lam1"]
    T0 = np.ascontiguousarray(np.asarray(w.T0, dtype=np.float64) + dT0)
    wp = dataclasses.replace(w, params=p, T0=T0)
    return _lbe.LBE(wp, storage=problem.storage)


class LBEMigration(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigmaT, eta_ratio, lam_ratio, dT0, problem: MigrationProblem):
        d = dT0.detach().to("cpu", torch.float64).numpy()
        sim = migration_handle(problem, _scalar(sigmaT), _scalar(eta_ratio),
                               _scalar(lam_ratio), d)
        try:
            r = sim.adjoint(problem.steps, problem.window, problem.ckpt_every, want_dT0=True)
        finally:
            sim.close()
        dev = dT0.device
        g = torch.tensor(r["grad"], dtype=torch.float64, device=dev)
        ctx.save_for_backward(g, r["dT0"].to(dev))
        ctx.dtypes = tuple(t.dtype if torch.is_tensor(t) else torch.float64
                           for t in (sigmaT, eta_ratio, lam_ratio, dT0))
        return torch.tensor(r["loss"], dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, gout):
        g, gT = ctx.saved_tensors
        ds, de, dl = (gout * g[j] for j in range(3))
        dt = ctx.dtypes
        return (ds.to(dt[0]), de.to(dt[1]), dl.to(dt[2]), (gout * gT).to(dt[3]), None)


def migration_loss(sigmaT, eta_ratio, lam_ratio, dT0, problem: MigrationProblem):
    """Functional form of ``LBEMigration.apply``."""
    return LBEMigration.apply(sigmaT, eta_ratio, lam_ratio, dT0, problem)

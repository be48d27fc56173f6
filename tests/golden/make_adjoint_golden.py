"""Writes adjoint_32x64.json: the reference gradient of the drop-migration
loss on the 32 x 64 problem, by central finite differences of the FP64
oracle only (no CUDA code is involved).

Problem: the 32 x 64 migration drop (R = 8 at (16, 16), Re = 1, Ma = 10,
Ca = 0.05, initial temperature perturbation N(0, 1e-4^2) per cell from
default_rng(1)), loss = mean centroid velocity sum(c u_y)/sum(c) over the
states 301..400 of a 400-step run (Sec. IV.C observable).

Stored: dL/dT0 at every cell (one central difference per cell, step H_T),
and dL/dsigmaT, dL/d(eta2/eta1), dL/d(lam2/lam1) (relative step H_REL).

Usage: python tests/golden/make_adjoint_golden.py [processes]
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

STEPS, WINDOW = 400, 100
H_T = 1e-6      # absolute step on T0 at one cell
H_REL = 1e-5    # relative step on sigmaT and the two ratios
OUT = os.path.join(HERE, "adjoint_32x64.json")


def problem():
    from paper_1412_6238_gb300 import workloads as W
    return W.migration_tiny(steps=STEPS)


def loss(params, T0):
    import oracle
    w = problem()
    return oracle.migration_loss(params, w.c0, T0, w.Tbot, w.Ttop, STEPS, WINDOW)


def cell_fd(k):
    w = problem()
    T0 = w.T0.copy().reshape(-1)
    Tp, Tm = T0.copy(), T0.copy()
    Tp[k] += H_T
    Tm[k] -= H_T
    shape = w.T0.shape
    return (loss(w.params, Tp.reshape(shape)) - loss(w.params, Tm.reshape(shape))) / (2 * H_T)


def param_fd(name):
    w = problem()
    p = dict(w.params)
    if name == "sigmaT":
        x0 = p["sigmaT"]
        h = H_REL * x0
        setp = lambda q, x: q.__setitem__("sigmaT", x)  # noqa: E731
    else:
        base, other = ("eta1", "eta2") if name == "eta_ratio" else ("lam1", "lam2")
        x0 = p[other] / p[base]
        h = H_REL * x0
        setp = lambda q, x: q.__setitem__(other, x * q[base])  # noqa: E731
    qp, qm = dict(p), dict(p)
    setp(qp, x0 + h)
    setp(qm, x0 - h)
    return (loss(qp, w.T0) - loss(qm, w.T0)) / (2 * h)


def _init():
    os.environ["OMP_NUM_THREADS"] = "1"


def main():
    nproc = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    os.environ["OMP_NUM_THREADS"] = "1"
    import oracle
    oracle.build()
    w = problem()
    ny, nx = w.T0.shape
    t0 = time.time()
    L0 = loss(w.params, w.T0)
    ctx = mp.get_context("spawn")
    with ctx.Pool(nproc, initializer=_init) as pool:
        grads = pool.map(param_fd, ["sigmaT", "eta_ratio", "lam_ratio"])
        dT0 = pool.map(cell_fd, range(nx * ny), chunksize=16)
    out = dict(
        problem="migration drop 32x64, R=8 at (16,16), Re=1, Ma=10, Ca=0.05, "
                "dT0 ~ N(0, 1e-4^2) from default_rng(1)",
        loss="mean of sum(c u_y)/sum(c) over states %d..%d" % (STEPS - WINDOW + 1, STEPS),
        steps=STEPS, window=WINDOW, h_T=H_T, h_rel=H_REL, nx=nx, ny=ny,
        loss_value=L0,
        dsigmaT=grads[0], deta_ratio=grads[1], dlam_ratio=grads[2],
        dT0=[float("%.17g" % v) for v in dT0],
        seconds=round(time.time() - t0, 1),
    )
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
    print("wrote %s in %.0f s (L = %.6e)" % (OUT, time.time() - t0, L0))


if __name__ == "__main__":
    main()

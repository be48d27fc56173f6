"""Shared helpers of the test suite: running a workload through the CUDA
library and through the oracle on the same seeded inputs, and the error
norms used by the parity tests (relative L2 over the domain; velocity as a
vector)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.sqrt((b * b).sum())
    return float(np.sqrt(((a - b) ** 2).sum()) / den) if den > 0 else float(np.sqrt((a * a).sum()))


def field_errors(F, G):
    """Relative L2 errors of c, T, p and u (vector) of F against G."""
    ua = np.stack([F["ux"], F["uy"]])
    ub = np.stack([G["ux"], G["uy"]])
    return dict(c=rel_l2(F["c"], G["c"]), T=rel_l2(F["T"], G["T"]), p=rel_l2(F["p"], G["p"]),
                u=rel_l2(ua, ub))


def gpu_fields(sim, instance=0):
    F = sim.fields(instance, device="cpu")
    return {k: v.numpy() for k, v in F.items()}


def oracle_fields(orc, w, pop):
    return orc.fields(w.params, pop, w.Tbot, w.Ttop)

"""Writes longrun_<case>.json: the FP64 oracle's state after the full step
count of a benchmark problem, for the full-length parity tests.  Only the
oracle and the seeded input generators are used.

Per case the file holds
  - input_sha256: hash of the inputs (c0, T0, Tbot, Ttop as float64 bytes),
    so a test can tell whether its inputs are bit-identical to these;
  - state_sha256: hash of the final [27][ny][nx] float64 population state
    (a bitwise-exact FP64 path must reproduce it);
  - fields c, p, ux, uy, T sampled every `stride` rows and columns (starting
    at stride/2), 17 significant digits;
  - full-domain figures: L2 norms of each field, sum c, the phase-1
    centroid height and velocity.

Cases (``python tests/golden/make_longrun_golden.py <case> ...``):
  planar    two superimposed fluids with Marangoni convection, 512 x 256,
            100 000 steps (Sec. IV.B)
  drop      drop migration, 512 x 1024, R = 32, 40 000 steps (Sec. IV.C)
  sweep00   first 128 x 256 instance of the 64-drop parameter sweep, 10 000 steps
  sweep01   first 256 x 512 instance of the sweep, 10 000 steps
  sweep02   first 512 x 1024 instance of the sweep, 10 000 steps
  sweep03   first 768 x 1536 instance of the sweep, 10 000 steps
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _sweep_instance(grid):
    from paper_1412_6238_gb300 import workloads as W
    ws = W.batch_sweep(64, seed=0, steps=10000)
    for j, w in enumerate(ws):
        if (w.nx, w.ny) == grid:
            return j, w
    raise RuntimeError("no sweep instance on grid %s" % (grid,))


def case(name):
    """(workload, steps, stride, description) of a case."""
    from paper_1412_6238_gb300 import workloads as W
    if name == "planar":
        return W.planar_marangoni(), 100000, 8, "planar_marangoni() 512x256"
    if name == "drop":
        return W.droplet_512x1024(), 40000, 16, "droplet_512x1024()"
    if name == "sweep00":
        j, w = _sweep_instance((128, 256))
        return w, 10000, 8, "batch_sweep(64, seed=0)[%d] 128x256" % j
    if name == "sweep01":
        j, w = _sweep_instance((256, 512))
        return w, 10000, 8, "batch_sweep(64, seed=0)[%d] 256x512" % j
    if name == "sweep02":
        j, w = _sweep_instance((512, 1024))
        return w, 10000, 16, "batch_sweep(64, seed=0)[%d] 512x1024" % j
    if name == "sweep03":
        j, w = _sweep_instance((768, 1536))
        return w, 10000, 24, "batch_sweep(64, seed=0)[%d] 768x1536" % j
    raise ValueError(name)


def input_sha(w) -> str:
    h = hashlib.sha256()
    for a in (w.c0, w.T0, w.Tbot, w.Ttop):
        h.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    return h.hexdigest()


def summarize(F, stride):
    """Sampled fields and full-domain figures of a field dict (ny, nx)."""
    s0 = stride // 2
    out = {"stride": stride, "offset": s0, "samples": {}, "norms": {}}
    for k in ("c", "p", "ux", "uy", "T"):
        a = np.asarray(F[k], dtype=np.float64)
        out["samples"][k] = [[float("%.17g" % v) for v in row] for row in a[s0::stride, s0::stride]]
        out["norms"][k] = float(np.sqrt((a * a).sum()))
    c = np.asarray(F["c"])
    y = np.arange(c.shape[0], dtype=np.float64)[:, None]
    out["sum_c"] = float(c.sum())
    out["centroid_y"] = float((c * y).sum() / c.sum())
    out["centroid_vy"] = float((c * F["uy"]).sum() / c.sum())
    return out


def main():
    import oracle
    oracle.build()
    for name in sys.argv[1:]:
        w, steps, stride, desc = case(name)
        t0 = time.time()
        pop = oracle.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop)
        pop = oracle.run(w.params, pop, w.Tbot, w.Ttop, steps)
        F = oracle.fields(w.params, pop, w.Tbot, w.Ttop)
        rec = {"case": name, "problem": desc, "nx": w.nx, "ny": w.ny, "steps": steps,
               "params": w.params, "input_sha256": input_sha(w),
               "state_sha256": hashlib.sha256(np.ascontiguousarray(pop).tobytes()).hexdigest(),
               "oracle_threads": oracle.num_threads(), "seconds": round(time.time() - t0, 1)}
        rec.update(summarize(F, stride))
        path = os.path.join(HERE, "longrun_%s.json" % name)
        with open(path, "w") as f:
            json.dump(rec, f, indent=0)
        print("wrote %s (%d steps, %.0f s)" % (path, steps, time.time() - t0), flush=True)


if __name__ == "__main__":
    main()

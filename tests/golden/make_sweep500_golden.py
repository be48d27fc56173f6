"""Writes sweep500.json: the FP64 oracle's state after 500 steps of every
instance of the 64-drop parameter sweep (batch_sweep(64, seed=0)), for the
batch parity test.  Only the oracle and the seeded input generators are used.

Per instance the file holds the grid, input_sha256 (c0, T0, Tbot, Ttop as
float64 bytes), state_sha256 (the final [27][ny][nx] float64 population
state, which the bitwise-exact FP64 path must reproduce), and full-domain
figures of the fields: sum c, the L2 norms of c, u (as a vector) and T.

    python tests/golden/make_sweep500_golden.py
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

STEPS = 500


def input_sha(w) -> str:
    h = hashlib.sha256()
    for a in (w.c0, w.T0, w.Tbot, w.Ttop):
        h.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    return h.hexdigest()


def main():
    import oracle
    from paper_1412_6238_gb300 import workloads as W
    oracle.build()
    ws = W.batch_sweep(64, seed=0)
    t0 = time.time()
    recs = []
    for j, w in enumerate(ws):
        pop = oracle.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop)
        pop = oracle.run(w.params, pop, w.Tbot, w.Ttop, STEPS)
        F = oracle.fields(w.params, pop, w.Tbot, w.Ttop)
        u = np.sqrt(np.sum(np.asarray(F["ux"]) ** 2 + np.asarray(F["uy"]) ** 2))
        recs.append({"index": j, "nx": w.nx, "ny": w.ny, "input_sha256": input_sha(w),
                     "state_sha256": hashlib.sha256(np.ascontiguousarray(pop).tobytes()).hexdigest(),
                     "sum_c": float(np.sum(F["c"])),
                     "norm_c": float(np.sqrt(np.sum(np.asarray(F["c"]) ** 2))),
                     "norm_u": float(u),
                     "norm_T": float(np.sqrt(np.sum(np.asarray(F["T"]) ** 2)))})
        print("instance %d (%d x %d) done at %.0f s" % (j, w.nx, w.ny, time.time() - t0),
              flush=True)
    rec = {"problem": "batch_sweep(64, seed=0)", "steps": STEPS, "instances": recs,
           "oracle_threads": oracle.num_threads(), "seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, "sweep500.json"), "w") as f:
        json.dump(rec, f, indent=0)
    print("wrote sweep500.json (%.0f s)" % (time.time() - t0))


if __name__ == "__main__":
    main()

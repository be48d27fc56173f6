"""Full-length runs of the benchmark problems against the FP64 oracle's
stored end states (tests/golden/longrun_*.json, written by
make_longrun_golden.py from the oracle alone):

  planar   two planar fluids with Marangoni convection, 512 x 256, 100 000 steps
  drop     drop migration, 512 x 1024, 40 000 steps
  sweep00..sweep03   one instance of each grid size of the 64-drop parameter
           sweep, 10 000 steps, run inside the whole 64-instance batch (one
           launch per step)

FP64: the end state is bitwise the oracle's: the inputs are generated
bitwise alike on every platform (workloads.py builds them from IEEE basic
operations), so their hash must equal the one the golden was made from, and
the state hash is compared every time.  FP32 and the 16-bit storages: the
relative L2 errors of u (as a vector) and T over the sampled points against
the stated bounds (1e-5 in FP32, 1e-3 with 16-bit storage), printed.
"""
import hashlib
import json
import os

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HERE = os.path.dirname(__file__)


def _golden(name):
    path = os.path.join(HERE, "golden", "longrun_%s.json" % name)
    if not os.path.exists(path):
        pytest.skip("golden %s missing" % name)
    return json.load(open(path))


def _case(name):
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_longrun_golden", os.path.join(HERE, "golden", "make_longrun_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.case(name), mod.input_sha


def _sampled(F, G):
    s, o = G["stride"], G["offset"]
    return {k: np.asarray(F[k])[o::s, o::s] for k in ("c", "p", "ux", "uy", "T")}


def _errors(F, G):
    A = _sampled(F, G)
    B = {k: np.asarray(v) for k, v in G["samples"].items()}
    ua = np.stack([A["ux"], A["uy"]])
    ub = np.stack([B["ux"], B["uy"]])
    rel = lambda a, b: float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))  # noqa: E731
    return dict(u=rel(ua, ub), T=rel(A["T"], B["T"]), c=rel(A["c"], B["c"]))


def _run(w, steps, storage):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_6238_gb300.lbe import LBE
    sim = LBE(w, storage=storage)
    sim.step(steps)
    return sim


# (case, storage) -> bounds on (u, T) relative L2 at the stated step count:
# FP32 1e-5, 16-bit storage 1e-3
BOUNDS = {
    ("planar", "f32"): (1e-5, 1e-5), ("drop", "f32"): (1e-5, 1e-5),
    ("drop", "f16mix"): (1e-3, 1e-3), ("drop", "f16dev"): (1e-3, 1e-3),
}
# sum c drift over the run, relative: FP32 conserves it to ~1e-9 (two-float
# g_0); the 16-bit forms round the moving g_i stochastically
MASS = {"f32": 1e-6, "f16dev": 1e-5, "f16mix": 1e-5}


@pytest.mark.parametrize("name", ["planar", "drop"])
def test_fp64_end_state_is_the_oracles(name):
    G = _golden(name)
    (w, steps, stride, desc), input_sha = _case(name)
    assert steps == G["steps"]
    assert input_sha(w) == G["input_sha256"], "inputs differ from the golden's"
    sim = _run(w, steps, "f64")
    state = sim.get_state().numpy()
    assert hashlib.sha256(np.ascontiguousarray(state).tobytes()).hexdigest() == \
        G["state_sha256"]
    print(name, "f64: end-state hash equal to the oracle's")
    F = {k: v.numpy() for k, v in sim.fields(device="cpu").items()}
    e = _errors(F, G)
    print(name, "f64", e)
    assert max(e.values()) < 1e-10


@pytest.mark.parametrize("name,storage", sorted(BOUNDS))
def test_storage_end_state_error(name, storage):
    G = _golden(name)
    (w, steps, stride, desc), input_sha = _case(name)
    assert input_sha(w) == G["input_sha256"], "inputs differ from the golden's"
    sim = _run(w, steps, storage)
    F = {k: v.numpy() for k, v in sim.fields(device="cpu").items()}
    e = _errors(F, G)
    print(name, storage, steps, "steps:", e)
    bu, bT = BOUNDS[(name, storage)]
    assert e["u"] < bu and e["T"] < bT, e
    assert abs(float(F["c"].sum()) - G["sum_c"]) < MASS[storage] * abs(G["sum_c"])


@pytest.mark.parametrize("storage,bu,bT", [("f64", 1e-10, 1e-10), ("f32", 1e-5, 1e-5),
                                           ("f16mix", 1e-3, 1e-3)])
def test_sweep_instances_inside_the_batch(storage, bu, bT):
    """The 64-instance sweep advanced 10 000 steps in one launch per step;
    the instances with stored oracle end states compared.  (The sweep's
    16-bit storage is F16MIX, FP16 deviations of g and hbar with f in FP32;
    FP16DEV, which also stores f in 16 bits, cannot resolve its slow flows.)
    FP64 arithmetic is slow on this part, so the FP64 batch holds the
    instances with stored end states and the smallest (128 x 256) ones in
    between, not all 64."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_6238_gb300 import workloads as W
    from paper_1412_6238_gb300.lbe import LBE
    ws = W.batch_sweep(64, seed=0, steps=10000)
    goldens = {}
    for name in ("sweep00", "sweep01", "sweep02", "sweep03"):
        path = os.path.join(HERE, "golden", "longrun_%s.json" % name)
        if os.path.exists(path):
            G = json.load(open(path))
            (w, steps, stride, desc), input_sha = _case(name)
            assert input_sha(w) == G["input_sha256"], "inputs differ from the golden's"
            j = int(desc.split("[")[1].split("]")[0])
            goldens[j] = G
    if not goldens:
        pytest.skip("sweep goldens missing")
    keep = list(range(len(ws)))
    if storage == "f64":
        keep = sorted(set(goldens) | {j for j, w in enumerate(ws) if w.nx * w.ny <= 128 * 256})
    slot = {j: k for k, j in enumerate(keep)}
    sim = LBE([ws[j] for j in keep], storage=storage)
    sim.step(10000)
    for j, G in goldens.items():
        if storage == "f64":
            st = np.ascontiguousarray(sim.get_state(slot[j]).numpy())
            assert hashlib.sha256(st.tobytes()).hexdigest() == G["state_sha256"], j
            print("sweep instance", j, "f64: end-state hash equal to the oracle's")
        F = {k: v.numpy() for k, v in sim.fields(slot[j], device="cpu").items()}
        e = _errors(F, G)
        print("sweep instance", j, storage, e)
        assert e["u"] < bu and e["T"] < bT, (j, e)

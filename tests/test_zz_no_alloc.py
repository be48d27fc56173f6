"""The allocation-free sums entry point (lbe_sums_fields_noalloc) against the
handle-based lbe_sums, through the C ABI.

lbe_sums_fields_noalloc exists for callers that cannot let the library
allocate device memory (a framework whose caching allocator owns the GPU's
memory, a monitoring loop where cudaMalloc/cudaFree would synchronize the
device); its scratch is a static array inside the library.  This file is
collected last so that a run stopping at the first failure has run every
other test first.
"""
import ctypes

import numpy as np
import pytest

from paper_1412_6238_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _fn():
    from paper_1412_6238_gb300 import lbe
    L = lbe.library()
    f = L.lbe_sums_fields_noalloc
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                  ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return L, f


def _ptrs(F):
    arr = (ctypes.c_void_p * 5)()
    for k, name in enumerate(("c", "p", "ux", "uy", "T")):
        arr[k] = F[name].data_ptr()
    return arr


def test_noalloc_sums_match_lbe_sums_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_6238_gb300.lbe import LBE
    L, fn = _fn()
    w = wl.droplet(150, 77, 12.0, 70.3, 33.2, Re=1.0, Ma=10.0, Ca=0.05, eta_m=0.2, eta_r=0.5,
                   lam_r=2.0)
    sim = LBE(w, storage="f64")
    rho_cv = w.params["rho"] * w.params["cv"]
    n = w.cells
    # the sentinel is written on the stream the entry point's kernels run on
    with torch.cuda.stream(sim.stream):
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    for steps in (30, 17):  # two calls in a row, different states
        sim.step(steps - 1)
        prev = sim.fields(device="cuda")
        sim.step(1)
        cur = sim.fields(device="cuda")
        ref = sim.sums()
        st = fn(_ptrs(cur), _ptrs(prev), n, rho_cv, ctypes.c_void_p(out.data_ptr()),
                ctypes.c_void_p(sim.stream.cuda_stream))
        assert st == 0, L.lbe_last_error(None).decode()
        sim.stream.synchronize()
        got = out.cpu().numpy()
        expect = np.array([ref["sum_c"], ref["sum_p"], ref["sum_h"], ref["residual"],
                           ref["nonfinite"]])
        assert got[4] == expect[4] == 0
        for k in range(4):
            assert got[k] == pytest.approx(expect[k], rel=1e-12, abs=1e-14), (k, got, expect)
        assert expect[3] > 0
    # without a previous state the residual is 0
    st = fn(_ptrs(cur), None, n, rho_cv, ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(sim.stream.cuda_stream))
    assert st == 0
    sim.stream.synchronize()
    assert out[3].item() == 0.0 and out[0].item() == pytest.approx(ref["sum_c"], rel=1e-12)
    # sizes beyond the static scratch are rejected with a message
    st = fn(_ptrs(cur), None, 33554432 + 1, rho_cv, ctypes.c_void_p(out.data_ptr()), None)
    assert st == -1 and "maximum" in L.lbe_last_error(None).decode()


@pytest.mark.parametrize("n", [3_000_001, 33_554_432])
def test_noalloc_sums_large_n_against_torch(n):
    """Many blocks (733 and the 8192-block maximum, so the second pass loops
    over the partials), a partial last block, and a planted NaN counted."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L, fn = _fn()
    g = torch.Generator(device="cuda").manual_seed(7)
    cur = {k: torch.rand(n, dtype=torch.float64, device="cuda", generator=g) + 0.25
           for k in ("c", "p", "ux", "uy", "T")}
    prev = {k: v + 1e-3 * torch.rand(n, dtype=torch.float64, device="cuda", generator=g)
            for k, v in cur.items()}
    rho_cv = 1.5
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    for rep in range(2):
        st = fn(_ptrs(cur), _ptrs(prev), n, rho_cv, ctypes.c_void_p(out.data_ptr()),
                ctypes.c_void_p(s.cuda_stream))
        assert st == 0, L.lbe_last_error(None).decode()
        s.synchronize()
        got = out.cpu().numpy()
        du2 = ((cur["ux"] - prev["ux"]) ** 2 + (cur["uy"] - prev["uy"]) ** 2).sum()
        u2 = (cur["ux"] ** 2 + cur["uy"] ** 2).sum()
        expect = [cur["c"].sum().item(), cur["p"].sum().item(),
                  rho_cv * cur["T"].sum().item(), (du2.sqrt() / u2.sqrt()).item()]
        for k in range(4):
            assert got[k] == pytest.approx(expect[k], rel=1e-12), (rep, k, got, expect)
        assert got[4] == 0
    cur["uy"][n - 3] = float("nan")
    s.wait_stream(torch.cuda.current_stream())
    st = fn(_ptrs(cur), _ptrs(prev), n, rho_cv, ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(s.cuda_stream))
    assert st == 0
    s.synchronize()
    got = out.cpu().numpy()
    # counted; the sums of the other fields are unaffected (the residual, like
    # lbe_sums', is reported as 0 when |u|^2 is not a positive number)
    assert got[4] == 1 and got[0] == pytest.approx(expect[0], rel=1e-12)
    assert got[2] == pytest.approx(expect[2], rel=1e-12) and got[3] == 0.0

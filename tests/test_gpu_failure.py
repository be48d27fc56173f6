"""Failure detection without a GPU fault: the bounded waits of the library
run out on purpose and report their status codes.

  - device: the strip kernel's copy waits are bounded.  LBE_FAULT=withhold:<row>
    makes the first step of a handle stage nothing for one row (the slot's
    barrier still expects the bytes) and give up a wait after 2^12 polls;
    the CTAs that need that row stop, the host reads the device error word
    and reports LBE_ECUDA, the handle refuses to step (LBE_ESTATE) and
    lbe_set_state brings it back.
  - host: every host wait is bounded by LBE_TIMEOUT_MS; a limit of 1 ms
    around a long lbe_step with check_every returns LBE_ETIMEOUT, and the
    work left on the stream completes normally afterwards.
"""
import os
import time

import numpy as np
import pytest

from paper_1412_6238_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbe_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_6238_gb300 import lbe
    return lbe


def _drop(nx=200, ny=160):
    return wl.droplet(nx, ny, 20.0, nx / 2.0, ny / 2.0, Re=1.0, Ma=10.0, Ca=0.05, eta_m=0.2,
                      eta_r=0.5, lam_r=2.0)


class _env:
    def __init__(self, **kv):
        self.kv = kv

    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kv}
        os.environ.update(self.kv)

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("storage", ["f32", "f16mix"])
def test_copy_wait_runs_out_reports_ecuda_and_recovers(lbe_mod, storage):
    w = _drop()
    ref = lbe_mod.LBE(w, storage=storage)
    start = ref.get_state()
    ref.step(7)
    want = ref.fields(device="cpu")
    with _env(LBE_FAULT="withhold:57"):
        sim = lbe_mod.LBE(w, storage=storage)
    assert sim.get_tile()["kernel"] in (7, 8)  # the strip kernel
    t0 = time.time()
    sim.step(3)
    with pytest.raises(lbe_mod.LBEError) as ei:
        sim.synchronize()
    dt = time.time() - t0
    assert ei.value.status == -3, ei.value
    assert "ran out of its poll limit" in str(ei.value)
    print("withheld row: LBE_ECUDA after %.3f s: %s" % (dt, ei.value))
    # every later wait reports it, and the handle refuses to step
    with pytest.raises(lbe_mod.LBEError) as e2:
        sim.fields(device="cpu")
    assert e2.value.status == -3
    with pytest.raises(lbe_mod.LBEError) as e3:
        sim.step(1)
    assert e3.value.status == -6
    # a new state clears the condition; the hook applied to one launch only,
    # so the handle then follows a fresh one: in FP32 to the rounding of the
    # state's round trip through FP64 (measured 1.4e-7 of the maximum of u);
    # with 16-bit storage to its stochastic rounding, whose random bits
    # follow the handle's step count (3 steps ahead of the fresh handle's)
    sim.set_state(start)
    sim.step(7)
    sim.synchronize()
    got = sim.fields(device="cpu")
    tol = 1e-6 if storage == "f32" else 1e-2
    for k in ("c", "ux", "uy", "T"):
        a, b = got[k].numpy(), want[k].numpy()
        assert np.abs(a - b).max() <= tol * np.abs(b).max(), (k, np.abs(a - b).max())


def test_host_wait_limit_returns_etimeout(lbe_mod):
    # few, long steps (0.7 ms each at 4096^2), so that the host has enqueued
    # them all long before the GPU is done and the check's wait starts early
    w = wl.droplet_scaled(4096, 4096)
    sim = lbe_mod.LBE(w, storage="f32", check_every=40)
    sim.step(1)
    sim.sums()  # the scratch of the check is allocated here, not inside the timed call
    sim.synchronize()
    with _env(LBE_TIMEOUT_MS="1"):
        with pytest.raises(lbe_mod.LBEError) as ei:
            sim.step(80)  # ~27 ms of GPU work before the first check waits
    assert ei.value.status == -5, ei.value
    assert "not done after 1 ms" in str(ei.value)
    # the work stays enqueued; with the default limit it completes
    sim.synchronize()
    s = sim.sums()
    assert s["nonfinite"] == 0
    assert sim.steps_done == 40  # the call returned at its first check

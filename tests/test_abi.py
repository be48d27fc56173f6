"""The C-ABI library builds, loads and exports every symbol that
include/lbe.h declares, and rejects bad arguments before touching the GPU.
CPU only (no kernel runs)."""
import ctypes
import os
import re

import pytest

from paper_1412_6238_gb300 import lbe, workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbe_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    L = lbe.library()
    decl = _declared()
    assert {"lbe_init", "lbe_step", "lbe_fields", "lbe_destroy"} <= decl
    for name in sorted(decl):
        assert hasattr(L, name), name
    assert set(lbe.EXPORTS) <= decl
    assert L.lbe_abi_version() == 2


def test_tile_table():
    shapes = lbe.tile_shapes()
    assert len(shapes) >= 1 and shapes[0] == (32, 8)
    for tx, ty in shapes:
        # tile kernel: TX multiple of a warp; strip kernels: TX output
        # columns per CTA (the retired ones had 4 halo threads besides)
        assert (tx % 32 == 0 and ty > 0) or (ty == 0 and tx % 32 in (0, 28))
    # the stash strip kernel, one thread per output column: 7 with the ghost
    # columns refreshed by a second kernel, 8 writing them in the step
    assert shapes[7] == (128, 0) and shapes[8] == (128, 0)


def _init(params, storage="f32"):
    L = lbe.library()
    w = wl.droplet(16, 32, 4.0, 8.0, 8.0, Re=1.0, Ma=10.0, Ca=0.05, eta_m=0.2, eta_r=1.0,
                   lam_r=1.0)
    w.params.update(params)
    p = lbe.make_params(w.params, storage)
    arrs = [w.c0, w.T0, w.Tbot, w.Ttop]
    dp = ctypes.POINTER(ctypes.c_double)
    init = lbe.InitFields(*[a.ctypes.data_as(dp) for a in arrs])
    h = ctypes.c_void_p()
    st = L.lbe_init(ctypes.byref(p), ctypes.byref(init), None, ctypes.byref(h))
    return st, L.lbe_last_error(None).decode(), h


@pytest.mark.parametrize("bad,msg", [
    (dict(ny=1), "ny"), (dict(nx=0), "nx"), (dict(tau_g=0.5), "tau_g"),
    (dict(eta1=0.0), "eta1"), (dict(eps=-1.0), "eps"), (dict(eta_n=0.0), "eta_n"),
    (dict(lam2=-1e-3), "lam"), (dict(rho=0.0), "rho"), (dict(sigmaT=float("nan")), "non-finite"),
    (dict(nx=65536, ny=65537), "2^31"),
    (dict(rho2=-1.0), "rho2"), (dict(rho2=float("inf")), "rho2"),
    (dict(rho2=3.0), "FP64"),  # a density ratio with FP32 storage
    (dict(interp=2), "interp"), (dict(interp=1, lam1=0.0), "harmonic"),
    (dict(wall_mid=3), "wall_mid"), (dict(cos_wet=1.5), "cos_wet"),
    (dict(cos_wet=float("nan")), "cos_wet"),
    (dict(dissip=2), "dissip"),
])
def test_invalid_parameters_rejected(bad, msg):
    st, err, h = _init(bad)
    assert st == -1 and msg in err and not h.value


def test_dissipation_needs_fp64_or_fp32():
    st, err, h = _init(dict(dissip=1), storage="f16mix")
    assert st == -1 and "FP64 or FP32" in err and not h.value


def test_invalid_storage_rejected():
    for bad in (7, -1, 5):
        st, err, h = _init({}, storage=bad)
        assert st == -1 and "storage" in err, bad
    # every named storage passes validation (no GPU here: it fails later, at
    # the device, not as an unknown storage)
    for name in lbe.STORAGE:
        st, err, h = _init({}, storage=name)
        if h.value:
            lbe.library().lbe_destroy(h)
        assert st == 0 or "storage" not in err, (name, err)


def test_alloc_failure_injected_on_host(monkeypatch):
    monkeypatch.setenv("LBE_FAULT", "alloc")
    st, err, h = _init({})
    assert st == -2 and "alloc" in err and not h.value


def test_null_handle_calls():
    L = lbe.library()
    assert L.lbe_step(None, 1) == -1
    assert L.lbe_steps_done(None) == -1
    assert L.lbe_num_instances(None) == 0
    L.lbe_destroy(None)
    assert L.lbe_set_tile(None, 0, 0, 0) == -1


def test_storage_names_match_the_header_enum():
    """The binding's storage names carry the values of lbe_storage."""
    src = open(os.path.join(ROOT, "include", "lbe.h")).read()
    body = re.search(r"typedef enum \{(.*?)\} lbe_storage;", src, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    enum = {k: int(v) for k, v in re.findall(r"(LBE_\w+)\s*=\s*(\d+)", body)}
    names = {"f64": "LBE_F64", "f32": "LBE_F32", "f16dev": "LBE_F16DEV",
             "bf16dev": "LBE_BF16DEV", "f16mix": "LBE_F16MIX"}
    assert set(lbe.STORAGE) == set(names)
    for k, c in names.items():
        assert lbe.STORAGE[k] == enum[c], k

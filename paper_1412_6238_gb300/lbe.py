"""ctypes binding of the C ABI in include/lbe.h (argument marshalling only).

Every step of the method runs in the CUDA kernels of ``liblbe.so``; this
module converts arguments, owns the handle, and hands torch tensors to the
library as output buffers.  There is no CPU fallback: if the library cannot
be built or loaded, or CUDA is unavailable, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

STORAGE = {"f64": 0, "f32": 1, "f16dev": 2, "bf16dev": 3, "f16mix": 4}
FIELD_NAMES = ("c", "p", "ux", "uy", "T")
STATUS = {0: "LBE_OK", -1: "LBE_EINVAL", -2: "LBE_ENOMEM", -3: "LBE_ECUDA", -4: "LBE_ENAN",
          -5: "LBE_ETIMEOUT", -6: "LBE_ESTATE"}
PARAM_KEYS = ("rho", "cv", "eta1", "eta2", "lam1", "lam2", "sigma0", "sigmaT", "Tref", "eps",
              "beta", "tau_g", "mobility", "ax", "ay", "eta_n")

# Symbols declared in include/lbe.h (checked by the tests against the header).
EXPORTS = ("lbe_abi_version", "lbe_init", "lbe_init_batch", "lbe_step", "lbe_synchronize",
           "lbe_fields", "lbe_sums", "lbe_get_state", "lbe_set_state", "lbe_save", "lbe_load",
           "lbe_num_tiles", "lbe_tile_shape", "lbe_set_tile", "lbe_get_tile", "lbe_steps_done", "lbe_stream",
           "lbe_num_instances", "lbe_state_bytes", "lbe_destroy", "lbe_last_error",
           "lbe_adjoint", "lbe_adjoint_step", "lbe_observable")


class LBEError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status, message))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("check_every", ctypes.c_int32)] + [(k, ctypes.c_double) for k in PARAM_KEYS] + \
               [("rho2", ctypes.c_double), ("interp", ctypes.c_int32),
                ("wall_mid", ctypes.c_int32), ("cos_wet", ctypes.c_double),
                ("dissip", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class InitFields(ctypes.Structure):
    _fields_ = [("c0", ctypes.POINTER(ctypes.c_double)), ("T0", ctypes.POINTER(ctypes.c_double)),
                ("Tbot", ctypes.POINTER(ctypes.c_double)),
                ("Ttop", ctypes.POINTER(ctypes.c_double))]


class AdjointSpec(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("window", ctypes.c_int64),
                ("ckpt_every", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def library(build: bool = True) -> ctypes.CDLL:
    """Load liblbe.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError("liblbe.so is missing (%s)" % path)
            L = ctypes.CDLL(path)
            H = ctypes.c_void_p
            st = ctypes.c_int
            dp = ctypes.POINTER(ctypes.c_double)
            sig = {
                "lbe_abi_version": ([], ctypes.c_int32),
                "lbe_init": ([ctypes.POINTER(Params), ctypes.POINTER(InitFields), ctypes.c_void_p,
                              ctypes.POINTER(H)], st),
                "lbe_init_batch": ([ctypes.c_int32, ctypes.POINTER(Params),
                                    ctypes.POINTER(InitFields), ctypes.c_void_p,
                                    ctypes.POINTER(H)], st),
                "lbe_step": ([H, ctypes.c_int64], st),
                "lbe_synchronize": ([H], st),
                "lbe_fields": ([H, ctypes.c_int32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p),
                                ctypes.c_int32, ctypes.c_int32], st),
                "lbe_sums": ([H, ctypes.c_int32, dp], st),
                "lbe_get_state": ([H, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32], st),
                "lbe_set_state": ([H, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32], st),
                "lbe_save": ([H, ctypes.c_char_p], st),
                "lbe_load": ([H, ctypes.c_char_p], st),
                "lbe_num_tiles": ([], ctypes.c_int32),
                "lbe_tile_shape": ([ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32)], st),
                "lbe_set_tile": ([H, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], st),
                "lbe_get_tile": ([H, ctypes.POINTER(ctypes.c_int32)], st),
                "lbe_steps_done": ([H], ctypes.c_int64),
                "lbe_stream": ([H], ctypes.c_void_p),
                "lbe_num_instances": ([H], ctypes.c_int32),
                "lbe_state_bytes": ([H], ctypes.c_int64),
                "lbe_destroy": ([H], None),
                "lbe_last_error": ([H], ctypes.c_char_p),
                "lbe_adjoint": ([H, ctypes.POINTER(AdjointSpec), dp, dp, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_int32], st),
                "lbe_adjoint_step": ([H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                      ctypes.c_void_p, dp], st),
                "lbe_observable": ([H, ctypes.c_void_p, dp], st),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def tile_shapes():
    L = library()
    out = []
    for t in range(L.lbe_num_tiles()):
        tx, ty = ctypes.c_int32(), ctypes.c_int32()
        L.lbe_tile_shape(t, ctypes.byref(tx), ctypes.byref(ty))
        out.append((tx.value, ty.value))
    return out


def _f64(a, shape):
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), shape))
    return a


def make_params(params: dict, storage: str | int, check_every: int = 0) -> Params:
    p = Params()
    p.nx, p.ny = int(params["nx"]), int(params["ny"])
    p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    p.check_every = int(check_every)
    for k in PARAM_KEYS:
        setattr(p, k, float(params[k]))
    p.rho2 = float(params.get("rho2", 0.0))  # 0: uniform density
    # variants (0: off): harmonic property law, wall temperature at the
    # link's wall crossing, contact angle of phase 1 (cos)
    p.interp = int(params.get("interp", 0))
    p.wall_mid = int(params.get("wall_mid", 0))
    p.cos_wet = float(params.get("cos_wet", 0.0))
    p.dissip = int(params.get("dissip", 0))  # the dissipation term of Eq. aEq7 (FP64)
    return p


class LBE:
    """One handle of the library: one instance, or a batch advanced together.

    ``problems``: a workload (object with ``params``, ``c0``, ``T0``,
    ``Tbot``, ``Ttop``) or a list of them.  ``storage``: how the populations
    are held between steps (arithmetic is FP64 for "f64", FP32 otherwise):
    "f64" (bitwise the FP64 oracle), "f32", "f16mix" (FP32 f, FP16 g and
    hbar deviations), "f16dev" / "bf16dev" (16-bit deviations, FP32 g_0).
    ``stream``: a torch CUDA stream (default: a new non-default stream, so
    that steps can be graph-captured).
    """

    def __init__(self, problems, storage: str = "f32", stream=None, check_every: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA is not available: the LBE step runs only on the GPU")
        self._L = library()
        probs = list(problems) if isinstance(problems, (list, tuple)) else [problems]
        self.n = len(probs)
        self.shapes = [(int(w.params["ny"]), int(w.params["nx"])) for w in probs]
        self.storage = storage
        self.stream = stream if stream is not None else torch.cuda.Stream()
        params = (Params * self.n)()
        inits = (InitFields * self.n)()
        keep = []
        for j, w in enumerate(probs):
            ny, nx = self.shapes[j]
            params[j] = make_params(w.params, storage, check_every)
            arrs = [_f64(w.c0, (ny, nx)), _f64(w.T0, (ny, nx)), _f64(w.Tbot, (nx,)),
                    _f64(w.Ttop, (nx,))]
            keep.append(arrs)
            dp = ctypes.POINTER(ctypes.c_double)
            inits[j] = InitFields(*[a.ctypes.data_as(dp) for a in arrs])
        h = ctypes.c_void_p()
        with torch.cuda.device(self.stream.device):
            st = self._L.lbe_init_batch(self.n, params, inits,
                                        ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise LBEError(st, self._L.lbe_last_error(None).decode())
        self._h = h

    # ------------------------------------------------------------------ helpers
    def _check(self, st):
        if st != 0:
            raise LBEError(st, self._L.lbe_last_error(self._h).decode())

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            self._L.lbe_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- the API
    def step(self, n: int = 1):
        self._check(self._L.lbe_step(self._h, int(n)))

    def synchronize(self):
        self._check(self._L.lbe_synchronize(self._h))

    @property
    def steps_done(self) -> int:
        return int(self._L.lbe_steps_done(self._h))

    @property
    def state_bytes(self) -> int:
        return int(self._L.lbe_state_bytes(self._h))

    def set_tile(self, tile: int, grid_ctas: int = 0, seg_rows: int = 0):
        """Choose the step kernel (see lbe_set_tile in include/lbe.h)."""
        self._check(self._L.lbe_set_tile(self._h, int(tile), int(grid_ctas), int(seg_rows)))

    def get_tile(self) -> dict:
        out = (ctypes.c_int32 * 4)()
        self._check(self._L.lbe_get_tile(self._h, out))
        return dict(kernel=out[0], grid=out[1], seg_rows=out[2], items=out[3])

    def fields(self, instance: int = 0, names=FIELD_NAMES, dtype=None, device="cuda", out=None):
        """Dict of torch tensors (ny, nx) for the requested fields.

        out: optional dict of preallocated contiguous (ny, nx) tensors (float64
        or float32, all of one dtype and all on the host or all on the GPU;
        pinned host memory makes the copy a direct DMA), written in place and
        returned; its keys are the fields to export."""
        import torch
        ny, nx = self.shapes[instance]
        ptrs = (ctypes.c_void_p * 5)()
        mask = 0
        if out is not None:
            ts = list(out.values())
            if not ts or any(k not in FIELD_NAMES for k in out):
                raise ValueError("out: a dict of fields among %s" % (FIELD_NAMES,))
            dtype = ts[0].dtype
            on_dev = ts[0].is_cuda
            for t in ts:
                if (tuple(t.shape) != (ny, nx) or t.dtype != dtype or t.is_cuda != on_dev
                        or not t.is_contiguous() or dtype not in (torch.float64, torch.float32)):
                    raise ValueError("out: contiguous (%d, %d) float64 or float32 tensors of "
                                     "one dtype and one device kind" % (ny, nx))
            for k, name in enumerate(FIELD_NAMES):
                if name in out:
                    ptrs[k] = out[name].data_ptr()
                    mask |= 1 << k
        else:
            dtype = torch.float64 if dtype is None else dtype
            dev = torch.device(device)
            on_dev = dev.type == "cuda"
            out = {}
            for k, name in enumerate(FIELD_NAMES):
                if name in names:
                    t = torch.empty((ny, nx), dtype=dtype, device=dev)
                    out[name] = t
                    ptrs[k] = t.data_ptr()
                    mask |= 1 << k
        self._check(self._L.lbe_fields(self._h, int(instance), mask, ptrs, int(on_dev),
                                       0 if dtype == torch.float64 else 1))
        return out

    def sums(self, instance: int = 0) -> dict:
        out = (ctypes.c_double * 5)()
        self._check(self._L.lbe_sums(self._h, int(instance), out))
        return dict(sum_c=out[0], sum_p=out[1], sum_h=out[2], residual=out[3],
                    nonfinite=int(out[4]))

    def get_state(self, instance: int = 0, device="cpu"):
        import torch
        ny, nx = self.shapes[instance]
        t = torch.empty((27, ny, nx), dtype=torch.float64, device=device)
        self._check(self._L.lbe_get_state(self._h, int(instance), ctypes.c_void_p(t.data_ptr()),
                                          int(t.is_cuda)))
        return t

    def set_state(self, state, instance: int = 0):
        import torch
        ny, nx = self.shapes[instance]
        if not torch.is_tensor(state):
            state = torch.from_numpy(np.ascontiguousarray(np.asarray(state, dtype=np.float64)))
        state = state.to(torch.float64).contiguous()
        if tuple(state.shape) != (27, ny, nx):
            raise ValueError("state must have shape (27, %d, %d)" % (ny, nx))
        if state.is_cuda:
            self._order_after_torch()
        self._check(self._L.lbe_set_state(self._h, int(instance),
                                          ctypes.c_void_p(state.data_ptr()),
                                          int(state.is_cuda)))

    def save(self, path: str):
        self._check(self._L.lbe_save(self._h, os.fsencode(path)))

    def load(self, path: str):
        self._check(self._L.lbe_load(self._h, os.fsencode(path)))

    # ---- discrete adjoint (single-instance handles)
    def adjoint(self, steps: int, window: int, ckpt_every: int = 100, want_dT0: bool = True,
                want_dQ0: bool = False) -> dict:
        """Run ``steps`` steps from the current state and the reverse sweep.
        Returns {loss, grad (sigmaT, eta ratio, lam ratio), dT0, dQ0} with the
        field gradients as float64 CUDA tensors (None when not requested)."""
        import torch
        ny, nx = self.shapes[0]
        dev = self.stream.device
        dT0 = torch.empty((ny, nx), dtype=torch.float64, device=dev) if want_dT0 else None
        dQ0 = torch.empty((27, ny, nx), dtype=torch.float64, device=dev) if want_dQ0 else None
        spec = AdjointSpec(int(steps), int(window), int(ckpt_every))
        loss = ctypes.c_double()
        grad = (ctypes.c_double * 3)()
        ptr = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else 0)  # noqa: E731
        self._check(self._L.lbe_adjoint(self._h, ctypes.byref(spec), ctypes.byref(loss), grad,
                                        ptr(dT0), ptr(dQ0), 1))
        return dict(loss=loss.value, grad=tuple(grad), dT0=dT0, dQ0=dQ0)

    def adjoint_step(self, Q, a_next=None, wl: float = 0.0):
        """(a_out, grad[3]) of one adjoint step at the state Q (CUDA float64
        tensor [27, ny, nx]); a_next = dL/dQ_{n+1} or None (zero)."""
        import torch
        ny, nx = self.shapes[0]
        Q = self._dev_state(Q)
        an = self._dev_state(a_next) if a_next is not None else None
        out = torch.empty_like(Q)
        grad = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
        self._check(self._L.lbe_adjoint_step(
            self._h, ctypes.c_void_p(Q.data_ptr()),
            ctypes.c_void_p(an.data_ptr() if an is not None else 0), float(wl),
            ctypes.c_void_p(out.data_ptr()), grad))
        return out, tuple(grad)

    def observable(self, Q) -> float:
        """Phase-1 centroid velocity sum(c u_y) / sum(c) of the state Q."""
        Q = self._dev_state(Q)
        out = ctypes.c_double()
        self._check(self._L.lbe_observable(self._h, ctypes.c_void_p(Q.data_ptr()),
                                           ctypes.byref(out)))
        return out.value

    def _dev_state(self, t):
        import torch
        ny, nx = self.shapes[0]
        if not torch.is_tensor(t):
            t = torch.from_numpy(np.ascontiguousarray(np.asarray(t, dtype=np.float64)))
        t = t.to(device=self.stream.device, dtype=torch.float64).contiguous()
        if tuple(t.shape) != (27, ny, nx):
            raise ValueError("state must have shape (27, %d, %d)" % (ny, nx))
        self._order_after_torch()
        return t

    def _order_after_torch(self):
        """Make the handle's stream wait for work torch queued on its current
        stream (copies that produced an input tensor)."""
        import torch
        self.stream.wait_stream(torch.cuda.current_stream(self.stream.device))

#!/usr/bin/env python
"""Throughput of the fused coupled-LBE step on GB300, in coupled MLUPS
(cell updates of all three lattices per second) and as a fraction of the
HBM roofline.

Workload: the thermocapillary drop problem (Re = 1, Ma = 10, Ca = 0.05,
viscosity and conductivity ratios 0.5, |grad T| = 1e-3, W = 4) on a
4096 x 4096 grid (R = 256 at (2048, 1024)), FP32 population storage.  One
step = one launch of the fused step kernel over all cells.  The state
(2 x 1.81 GB) is far larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) each rank runs an independent replica (the method
needs no exchange between independent problems), timing is max over ranks
and the value is the whole-job aggregate.  ``--impl reference`` times the
FP64 CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled-LBE MLUPS & % HBM roofline; mixed/batched vs plain FP32 at stated error"
UNIT = "MLUPS"
NX = NY = 4096
# algorithmic bytes per cell update: the 27 populations read once and written
# once in the storage's element size (FP64: 27 x 8; FP32: 27 x 4; 16-bit
# deviation forms: 26 x 2 + the FP32 g_0; F16MIX: 9 FP32 f + 8 FP16 g + the
# FP32 g_0 + 9 FP16 hbar), both directions
BYTES_PER_CELL = {"f64": 432, "f32": 216, "f16dev": 112, "bf16dev": 112, "f16mix": 148}
# bytes the storage moves beyond the populations: the FP16 low part of g_0
# (read and written) in every form but FP64
OVERHEAD_BYTES_PER_CELL = {"f64": 0, "f32": 4, "f16dev": 4, "bf16dev": 4, "f16mix": 4}
PROFILE = os.path.join(ROOT, "profiles", "lbe_step_f32_droplet_4096x4096.md")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=NX)
    ap.add_argument("--ny", type=int, default=NY)
    ap.add_argument("--storage", default="f32", choices=list(BYTES_PER_CELL))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the 16-bit storage and batched-sweep measurements")
    ap.add_argument("--batch-steps", type=int, default=50)
    ap.add_argument("--kernel", type=int, default=-1,
                    help="step kernel id (lbe_set_tile); default: the library's choice")
    ap.add_argument("--seg", type=int, default=0, help="rows per strip work item (0 = auto; < 0: balanced ranges in pieces of at most -seg rows)")
    return ap.parse_args()


# ------------------------------------------------------------ distributed
def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = os.environ.get("BENCH_DIST_BACKEND") or (
            "nccl" if torch.cuda.is_available() else "gloo")
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(ws, ms: float, cells: int, steps: int):
    """(max-over-ranks time in ms, whole-job MLUPS): every rank advances its
    own replica of the problem, so the job updates ws * cells * steps cells
    in the slowest rank's time."""
    ms_max = allmax(ws, ms)
    return ms_max, cells * steps * ws / (ms_max / 1e3) / 1e6


# ------------------------------------------------------------ measurement aids
class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def hbm_peak():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_sha() -> str:
    """Hash of the sources and flags that make the FP32 step kernel (the
    traffic figure of the committed ncu summary is valid while it matches);
    comments and blank space are left out, so that only code changes count."""
    import re
    from paper_1412_6238_gb300 import build as _b
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1412_6238_gb300", "csrc")
    for f in ("lbe_common.cuh", "lbe_cell.cuh", "lbe_tile.cuh", "lbe_stash.cuh",
              "lbe_step_inst.cuh", "lbe_step_f32.cu"):
        src = open(os.path.join(d, f), encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    h.update(repr(_b.UNITS["lbe_step_f32.cu"]).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_id=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    try:
        kv = {}
        for line in open(PROFILE):
            if ":" in line and line.lstrip().startswith("- "):
                k, v = line.lstrip()[2:].split(":", 1)
                kv[k.strip()] = v.strip().strip("`")
        if kv.get("source_sha") != kernel_source_sha():
            return None
        if kernel_id is not None and int(kv.get("kernel_id", -1)) != kernel_id:
            return None
        return float(kv["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


# ------------------------------------------------------------ CPU oracle leg
def band_workload():
    """Bounded CPU sample of the benchmark problem: the same drop problem on
    a 4096 x 256 band (R = 96)."""
    from paper_1412_6238_gb300 import workloads as wl
    return wl.droplet(4096, 256, 96.0, 2048.0, 128.0, Re=1.0, Ma=10.0, Ca=0.05, eta_m=0.2,
                      eta_r=0.5, lam_r=0.5)


def oracle_sample(target_s: float = 12.0, steps: int | None = None, warmup: int = 1):
    """The FP64 oracle as it stands, on the host cores, on the band sample;
    ``steps`` timed steps (or as many as fill ``target_s``)."""
    import oracle
    w = band_workload()
    pop = oracle.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop)
    t = time.perf_counter()
    pop = oracle.run(w.params, pop, w.Tbot, w.Ttop, max(1, warmup))
    one = (time.perf_counter() - t) / max(1, warmup)
    n = steps if steps else max(1, min(200, int(target_s / max(one, 1e-3))))
    t = time.perf_counter()
    oracle.run(w.params, pop, w.Tbot, w.Ttop, n)
    dt = time.perf_counter() - t
    return {"value": w.cells * n / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "FP64 oracle, %d steps of the drop problem on a 4096 x 256 band "
                      "(%.1f s)" % (n, dt)}


def oracle_configs():
    """The oracle-timing workloads: the five-problem set's grids that the
    oracle runs (thermal two-layer Poiseuille 4 x 101, planar Marangoni
    512 x 256, drop 512 x 1024, the first instance of the 64-drop sweep)."""
    from paper_1412_6238_gb300 import workloads as wl
    s0 = wl.batch_sweep(64, seed=0)[0]
    return [("layered_poiseuille_4x101", wl.layered_poiseuille()),
            ("planar_marangoni_512x256", wl.planar_marangoni()),
            ("droplet_512x1024", wl.droplet_512x1024()),
            ("sweep_instance0_%dx%d" % (s0.nx, s0.ny), s0)]


def oracle_timings(target_s: float = 1.5):
    """Oracle MLUPS at one thread and at all host cores on each workload of
    oracle_configs(), each a bounded run of about target_s seconds."""
    import oracle
    out = []
    for name, w in oracle_configs():
        pop0 = oracle.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop)
        for threads in (1, 0):
            oracle.set_threads(threads)
            t = time.perf_counter()
            pop = oracle.run(w.params, pop0, w.Tbot, w.Ttop, 1)
            one = time.perf_counter() - t
            n = max(1, min(200000, int(target_s / max(one, 1e-6))))
            t = time.perf_counter()
            oracle.run(w.params, pop, w.Tbot, w.Ttop, n)
            dt = time.perf_counter() - t
            out.append({"workload": name, "cells": w.cells, "threads": oracle.num_threads(),
                        "steps": n, "seconds": round(dt, 3),
                        "MLUPS": w.cells * n / dt / 1e6})
    oracle.set_threads(0)
    return out


def run_reference(args, ws, rank):
    if rank != 0:
        return
    # each timed step is one oracle step of the band sample; K bounds the run
    cb = oracle_sample(steps=max(1, min(args.steps, 400)), warmup=max(1, min(args.warmup, 5)))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "droplet_4096x4096 (sampled: 4096 x 256 band)",
                       "storage": "f64 CPU oracle"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ GPU leg
def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_1412_6238_gb300 import workloads as wl
    from paper_1412_6238_gb300.lbe import LBE

    torch.cuda.set_device(local)
    w = wl.droplet_scaled(args.nx, args.ny)
    cells = w.cells
    sim = LBE(w, storage=args.storage)
    if args.kernel >= 0 or args.seg != 0:
        sim.set_tile(args.kernel if args.kernel >= 0 else sim.get_tile()["kernel"], 0, args.seg)
    kernel = sim.get_tile()
    stream = sim.stream
    sim.step(args.warmup)
    sim.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clk = Clocks(torch.cuda.current_device())
    time.sleep(0.3)
    t0.record(stream)
    sim.step(args.steps)
    t1.record(stream)
    t1.synchronize()
    torch.cuda.synchronize()
    clocks = clk.stop()
    barrier(ws)
    ms = t0.elapsed_time(t1)
    ms_max, value = aggregate(ws, ms, cells, args.steps)
    launch_ms = ms / args.steps
    algo_bytes = cells * BYTES_PER_CELL[args.storage]
    achieved = algo_bytes / (launch_ms / 1e3) / 1e9
    peak, peak_kind = hbm_peak()
    traffic = (profiled_traffic(kernel["kernel"])
               if (args.storage == "f32" and args.nx == NX and args.ny == NY) else None)
    fin = sim.sums()
    ref_fields = sim.fields(device="cuda") if not args.no_variants else None
    del sim
    torch.cuda.empty_cache()

    variants = None
    if not args.no_variants and ws == 1:
        variants = measure_variants(args, w, ref_fields)
        del ref_fields
        torch.cuda.empty_cache()

    # end to end through the public API, host buffers in and out
    e2e = None
    if not args.no_e2e:
        c0 = torch.from_numpy(w.c0).pin_memory()
        T0 = torch.from_numpy(w.T0).pin_memory()
        outs = {k: torch.empty((w.ny, w.nx), dtype=torch.float64).pin_memory()
                for k in ("c", "p", "ux", "uy", "T")}
        w2 = wl.Workload(w.name, w.params, c0.numpy(), T0.numpy(), w.Tbot, w.Ttop, w.steps)
        # one untimed pass of the same calls first (module and allocator
        # warm-up, like the warm-up steps of the device-timed line)
        for timed in (False, True):
            barrier(ws)
            torch.cuda.synchronize()
            ts = time.perf_counter()
            s2 = LBE(w2, storage=args.storage)
            s2.step(args.steps)
            s2.fields(out=outs)  # device -> pinned host buffers
            te = time.perf_counter() - ts
            del s2
            if not timed:
                torch.cuda.empty_cache()
        te = allmax(ws, te)
        h2d = (2 * cells + 2 * w.nx) * 8
        d2h = 5 * cells * 8
        e2e = {"value": cells * args.steps * ws / te / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "note": "lbe_init from host c0/T0/walls + %d steps + lbe_fields to host, "
                       "wall clock of the second of two identical passes" % args.steps}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample()
        cpu["per_workload"] = oracle_timings()
        cpu["host_cores"] = len(os.sched_getaffinity(0))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.storage != "f64" else "f64", "data": "synthetic",
                "config": {"workload": "droplet_%dx%d" % (args.nx, args.ny),
                           "problem": "thermocapillary drop, R=%g at (%g, %g), Re=1, Ma=10, "
                                      "Ca=0.05, ratios 0.5, |grad T|=1e-3, W=4"
                                      % (w.info["R"], w.info["xc"], w.info["yc"]),
                           "storage": args.storage, "cells": cells,
                           "l2": "state 2 x %.2f GB >> L2 (no flush needed)"
                                 % (algo_bytes / 2 / 1e9),
                           "parallelism": "replicas x%d" % ws,
                           "kernel": kernel},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                             "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                             "peak_kind": peak_kind,
                             "algorithmic_bytes_per_launch": algo_bytes,
                             "algorithmic_bytes_per_cell": BYTES_PER_CELL[args.storage],
                             "overhead_bytes_per_cell": OVERHEAD_BYTES_PER_CELL[args.storage],
                             "frac_with_overhead": cells * (BYTES_PER_CELL[args.storage] +
                                                            OVERHEAD_BYTES_PER_CELL[args.storage])
                                                   / (launch_ms / 1e3) / 1e9 / peak},
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "variants": variants,
                # the stash kernel's step is two launches (the step, then the
                # ghost columns and step counter (7) or the step counter (8))
                "gpu_launches": args.steps * (2 if kernel["kernel"] in (7, 8) else 1),
                "check": {"sum_c": fin["sum_c"], "nonfinite": fin["nonfinite"]}}
        print(json.dumps(line), flush=True)


def _timed(sim, steps):
    import torch
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    sim.synchronize()
    t0.record(sim.stream)
    sim.step(steps)
    t1.record(sim.stream)
    t1.synchronize()
    return t0.elapsed_time(t1)


GOLDEN_DROP = os.path.join(ROOT, "tests", "golden", "longrun_drop.json")


def error_vs_oracle(storage: str):
    """Relative L2 error of u (as a vector) and T against the FP64 oracle's
    stored end state of the 512 x 1024 drop after its stated 40 000 steps
    (tests/golden/longrun_drop.json, written from the oracle alone), over the
    golden's sampled points; None if the golden is missing or was made from
    other inputs."""
    import hashlib

    import numpy as np

    from paper_1412_6238_gb300 import workloads as wl
    from paper_1412_6238_gb300.lbe import LBE
    try:
        G = json.load(open(GOLDEN_DROP))
    except (OSError, ValueError):
        return None
    w = wl.droplet_512x1024()
    h = hashlib.sha256()
    for a in (w.c0, w.T0, w.Tbot, w.Ttop):
        h.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    if h.hexdigest() != G["input_sha256"]:
        return None
    sim = LBE(w, storage=storage)
    sim.step(G["steps"])
    F = {k: v.numpy() for k, v in sim.fields(device="cpu").items()}
    del sim
    s, o = G["stride"], G["offset"]
    A = {k: F[k][o::s, o::s] for k in ("ux", "uy", "T")}
    B = {k: np.asarray(G["samples"][k]) for k in ("ux", "uy", "T")}
    ua, ub = np.stack([A["ux"], A["uy"]]), np.stack([B["ux"], B["uy"]])
    rel = lambda a, b: float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))  # noqa: E731
    return {"u": rel(ua, ub), "T": rel(A["T"], B["T"]), "steps": G["steps"],
            "problem": "drop 512 x 1024, R = 32, Re = 1, Ma = 10, Ca = 0.05, ratios 0.5"}


def measure_extensions(args, w):
    """Throughput of the scheme's extensions on the benchmark drop (4096^2)
    beside the default scheme on the same kernel: the boundary and property
    variants (harmonic law, link-crossing wall temperature, wetting walls)
    on the FP32 strip kernel built with them; the density ratio rho2/rho1 =
    4 (FP64 tile kernel plus its corrected-p pre-pass); the dissipation term
    (FP64 and FP32 tile kernel plus the u pre-pass).  Fraction of the
    measured HBM peak on the 27 populations read and written per cell
    (pre-passes not counted as traffic: they are part of the step's time)."""
    import numpy as np

    from paper_1412_6238_gb300.lbe import LBE
    peak, _ = hbm_peak()
    x = np.arange(w.nx, dtype=float)
    Tb = w.Tbot + 1e-3 * np.cos(2 * np.pi * x / w.nx)

    def run(storage, extra, steps, kernel=None, tb=None):
        p = dict(w.params, **extra)
        w2 = type(w)(w.name, p, w.c0, w.T0, w.Tbot if tb is None else tb, w.Ttop, w.steps)
        sim = LBE(w2, storage=storage)
        if kernel is not None:
            sim.set_tile(kernel)
        sim.step(3)
        ms = _timed(sim, steps)
        tile = sim.get_tile()["kernel"]
        del sim
        ms_step = ms / steps
        mlups = w.cells * steps / (ms / 1e3) / 1e6
        return {"value": mlups, "unit": UNIT, "ms_per_step": ms_step, "kernel": tile,
                "hbm_frac": w.cells * BYTES_PER_CELL[storage] / (ms_step / 1e3) / 1e9 / peak}

    n32, n64 = max(20, args.steps // 4), 10
    var = dict(interp=1, wall_mid=1, cos_wet=0.3)
    return {
        "f32_strip_default": run("f32", {}, n32),
        "f32_strip_N2_variants": run("f32", var, n32, tb=Tb),
        "f32_tile_default": run("f32", {}, n32, kernel=0),
        "f32_tile_N3_dissipation": run("f32", dict(dissip=1), n32),
        "f64_tile_default": run("f64", {}, n64),
        "f64_tile_N1_density_ratio_4": run("f64", dict(rho2=4.0), n64),
        "f64_tile_N3_dissipation": run("f64", dict(dissip=1), n64),
        "f64_tile_N1_N2_N3": run("f64", dict(var, rho2=4.0, dissip=1), n64, tb=Tb),
        "problem": "drop 4096 x 4096 (the benchmark workload); rho2 = 4 rho, cos_wet = 0.3",
    }


def measure_variants(args, w, ref_fields):
    """The same workload with 16-bit deviation storage (timed like the main
    line), each storage's error against the FP64 oracle on the 512 x 1024
    drop after its 40 000 steps, and the batched parameter sweep of 64 drops
    of uneven size in one persistent launch per step (launch shape chosen by
    the autotuner) against 64 sequential FP32 runs."""
    import numpy as np
    import torch

    from paper_1412_6238_gb300 import workloads as wl
    from paper_1412_6238_gb300.lbe import LBE
    out = {}
    peak, _ = hbm_peak()

    def rel(F, G, keys):
        a = torch.stack([F[k] for k in keys])
        b = torch.stack([G[k] for k in keys])
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))

    for st in ("f16mix", "f16dev", "bf16dev"):
        sim = LBE(w, storage=st)
        sim.step(args.warmup)
        ms = _timed(sim, args.steps)
        F = sim.fields(device="cuda")
        del sim
        launch_ms = ms / args.steps
        mlups = w.cells * args.steps / (ms / 1e3) / 1e6
        bytes_launch = w.cells * BYTES_PER_CELL[st]
        out[st] = {"value": mlups, "unit": UNIT, "ms_per_step": launch_ms,
                   "hbm_frac": bytes_launch / (launch_ms / 1e3) / 1e9 / peak,
                   "bytes_per_cell": BYTES_PER_CELL[st],
                   "rel_l2_vs_f32": {"u": rel(F, ref_fields, ("ux", "uy")),
                                     "T": rel(F, ref_fields, ("T",)),
                                     "c": rel(F, ref_fields, ("c",))},
                   "steps_compared": args.warmup + args.steps}
        del F
        torch.cuda.empty_cache()
    # every storage's error against the oracle at the stated step count
    out["error_vs_oracle"] = {st: error_vs_oracle(st)
                              for st in ("f32", "f16mix", "f16dev", "bf16dev")}
    torch.cuda.empty_cache()
    out["extensions"] = measure_extensions(args, w)
    torch.cuda.empty_cache()

    # batched sweep (64 drops, grids 128x256 .. 768x1536, seed 0)
    sweep = wl.batch_sweep(64, seed=0)
    cells = sum(x.cells for x in sweep)
    K = args.batch_steps
    res = {"instances": len(sweep), "cells": cells, "steps": K}
    from paper_1412_6238_gb300 import autotune
    tuned = {}
    with tempfile.TemporaryDirectory() as td:
        os.environ["LBE_AUTOTUNE_CACHE"] = os.path.join(td, "tune.json")
        for st in ("f16mix", "f16dev", "f32"):
            sim = LBE(sweep, storage=st)
            sim.step(3)
            best = autotune.tune(sim, steps=5, warmup=2)
            tuned[st] = {k: best[k] for k in ("kernel", "grid", "seg_rows")}
            ms = _timed(sim, K)
            res["batched_" + st] = cells * K / (ms / 1e3) / 1e6
            del sim
            torch.cuda.empty_cache()
        os.environ.pop("LBE_AUTOTUNE_CACHE", None)
    res["autotuned"] = tuned
    seq_ms = 0.0
    for x in sweep:
        sim = LBE(x, storage="f32")
        sim.step(3)
        seq_ms += _timed(sim, K)
        del sim
    res["sequential_f32"] = cells * K / (seq_ms / 1e3) / 1e6
    res["speedup_batched_f16mix_vs_sequential_f32"] = res["batched_f16mix"] / res["sequential_f32"]
    res["speedup_batched_f16dev_vs_sequential_f32"] = res["batched_f16dev"] / res["sequential_f32"]
    res["unit"] = UNIT
    out["batch64"] = res

    # differentiable migration (256 x 512 drop, 2000 FP32 steps, checkpoints
    # every 100, loss over the last 200 states): forward + reverse sweep
    from paper_1412_6238_gb300 import workloads as wl
    mw = wl.migration_256x512(steps=2000)
    sim = LBE(mw, storage="f32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = sim.adjoint(2000, 200, 100, want_dT0=True)
    ta = time.perf_counter() - t0
    del sim
    torch.cuda.empty_cache()
    out["adjoint_migration_256x512"] = {
        "seconds": ta, "loss": r["loss"], "grad_sigmaT": r["grad"][0],
        "grad_eta_ratio": r["grad"][1], "grad_lam_ratio": r["grad"][2],
        "forward_plus_reverse_MLUPS": mw.cells * 2000 / ta / 1e6,
        "note": "FP32 forward (stash kernel), reverse sweep over recomputed segments with FP32 "
                "per-cell products and FP64 adjoint vectors; wall clock of one lbe_adjoint call"}
    return out


def main():
    args = parse_args()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

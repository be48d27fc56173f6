"""Launch-shape autotuner for the step kernel.

For a handle (one instance or a batch) it times every candidate launch —
kernel id (tile shapes and strip widths), persistent-grid size and, for the
strip kernel, rows per work item — for a few steps each and selects the
fastest.  Results are cached in a JSON file keyed by GPU name, storage and the
instance shapes, so a later handle of the same layout is configured without
timing.  Timing advances the state, so the handle is checkpointed (raw
storage bytes and step counter) before the search and restored after it.
"""
from __future__ import annotations

import json
import os
import tempfile
import threading

_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("LBE_AUTOTUNE_CACHE")
    if p:
        return p
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "lbe_gb300_autotune.json")


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def _store(path: str, d: dict) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def cache_key(device_name: str, storage: str, shapes) -> str:
    """Key of a layout: GPU, storage and the (ny, nx) of every instance."""
    dims = ",".join("%dx%d" % (nx, ny) for ny, nx in shapes)
    return "%s|%s|%s" % (device_name, storage, dims)


def candidates(storage: str, shapes, num_tiles: int, tile_shape):
    """(kernel id, grid, seg rows) triples to try for a layout."""
    min_nx = min(nx for _, nx in shapes)
    max_ny = max(ny for ny, _ in shapes)
    out = []
    for k in range(num_tiles):
        tx, ty = tile_shape(k)
        if storage == "f64" and k != 0:
            continue
        if ty == 0:  # strip kernel
            if storage == "f64" or min_nx < 4:
                continue
            # 0 automatic, -max_ny balanced row ranges (uncut), > 0 items of
            # that many rows
            for seg in (0, -max_ny, 72, 96, max(8, max_ny // 8), max(8, max_ny // 4)):
                out.append((k, 0, seg))
        else:
            out.append((k, 0, 0))
            out.append((k, -1, 0))
    # drop duplicates, keep order
    seen, uniq = set(), []
    for c in out:
        if c not in seen:
            seen.add(c)
            uniq.append(c)
    return uniq


def tune(sim, steps: int = 10, warmup: int = 2, use_cache: bool = True) -> dict:
    """Time every candidate launch of ``sim`` (an lbe.LBE), configure the
    fastest and return {kernel, grid, seg_rows, ms_per_step, tried}."""
    import torch

    from . import lbe as _lbe

    L = _lbe.library()
    dev = torch.cuda.get_device_name(sim.stream.device)
    key = cache_key(dev, sim.storage, sim.shapes)
    path = cache_path()
    if use_cache:
        with _lock:
            hit = _load(path).get(key)
        if hit:
            sim.set_tile(hit["kernel"], hit["grid"], hit["seg_rows"])
            return dict(hit, cached=True)

    shapes_fn = lambda k: _lbe.tile_shapes()[k]  # noqa: E731
    cands = candidates(sim.storage, sim.shapes, L.lbe_num_tiles(), shapes_fn)
    fd, ckpt = tempfile.mkstemp(suffix=".lbeckpt")
    os.close(fd)
    sim.save(ckpt)
    steps0 = sim.steps_done
    results = []
    for k, grid, seg in cands:
        try:
            sim.set_tile(k, grid, seg)
        except _lbe.LBEError:
            continue
        sim.step(warmup)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sim.synchronize()
        e0.record(sim.stream)
        sim.step(steps)
        e1.record(sim.stream)
        e1.synchronize()
        results.append((e0.elapsed_time(e1) / steps, k, grid, seg))
    try:
        sim.load(ckpt)
    finally:
        os.unlink(ckpt)
    if not results:
        raise RuntimeError("no launch candidate could be configured")
    ms, k, grid, seg = min(results)
    sim.set_tile(k, grid, seg)
    best = dict(kernel=k, grid=grid, seg_rows=seg, ms_per_step=ms, steps_before=steps0,
                tried=[dict(kernel=a, grid=b, seg_rows=c, ms_per_step=t)
                       for t, a, b, c in sorted(results)])
    if use_cache:
        with _lock:
            d = _load(path)
            d[key] = {k_: v for k_, v in best.items() if k_ != "tried"}
            _store(path, d)
    return dict(best, cached=False)

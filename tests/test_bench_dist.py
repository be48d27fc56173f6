"""The multi-process path of bench.py on CPU (gloo, world size 2): the
barrier, the max-over-ranks time and the whole-job rate of N replicas, and
the reference arm's rank > 0 exit."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), BENCH_DIST_BACKEND="gloo")
    import torch.distributed as dist

    import bench
    ws_, rank_, _ = bench.dist_init()
    bench.barrier(ws_)
    ms = 10.0 * (rank_ + 1)
    q.put((rank_, ws_) + bench.aggregate(ws_, ms, 1000, 5))
    bench.barrier(ws_)
    dist.destroy_process_group()


def test_two_replicas_max_time_and_aggregate_rate():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, ms_max, value in res:
        assert ws == 2
        assert ms_max == 20.0                      # the slower rank's time
        assert value == pytest.approx(2 * 1000 * 5 / 0.020 / 1e6)


def test_single_process_aggregate():
    import bench
    ms_max, value = bench.aggregate(1, 4.0, 2_000_000, 10)
    assert ms_max == 4.0 and value == pytest.approx(5000.0)


def test_reference_arm_other_ranks_print_nothing(capsys):
    import argparse

    import bench
    args = argparse.Namespace(steps=3, warmup=3, gpus=2)
    bench.run_reference(args, 2, 1)
    assert capsys.readouterr().out == ""


def test_reference_arm_line(capsys):
    """Rank 0 of the reference arm prints one JSON line with the keys of the
    benchmark contract; its value is the FP64 oracle timed on the host."""
    import argparse
    import json

    import bench
    args = argparse.Namespace(steps=1, warmup=1, gpus=1)
    bench.run_reference(args, 1, 0)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0

"""Launch autotuner: candidate list and JSON cache (CPU), and on the GPU a
tuning pass that leaves the state untouched and a cached second call."""
import numpy as np
import pytest

from paper_1412_6238_gb300 import autotune, workloads as wl


def test_candidates_and_cache_roundtrip(tmp_path, monkeypatch):
    shapes = [(256, 128), (512, 256)]
    tile = lambda k: [(32, 8), (64, 4), (32, 16), (64, 8), (128, 4), (124, 0), (60, 0)][k]
    c32 = autotune.candidates("f32", shapes, 7, tile)
    assert (5, 0, 0) in c32 and (0, -1, 0) in c32 and len(set(c32)) == len(c32)
    assert all(k == 0 for k, _, _ in autotune.candidates("f64", shapes, 7, tile))
    assert all(tile(k)[1] > 0 for k, _, _ in autotune.candidates("f32", [(8, 3)], 7, tile))
    monkeypatch.setenv("LBE_AUTOTUNE_CACHE", str(tmp_path / "c.json"))
    p = autotune.cache_path()
    autotune._store(p, {"k": {"kernel": 5}})
    assert autotune._load(p) == {"k": {"kernel": 5}}
    assert autotune.cache_key("GB300", "f32", shapes) == "GB300|f32|128x256,256x512"


def test_candidates_from_the_library_table():
    """With the library's own kernel table the autotuner tries both strip
    kernels (7: ghost columns by a second kernel, 8: by the step) with the
    same row counts, and only tile kernel 0 for FP64."""
    from paper_1412_6238_gb300 import lbe
    shapes_tbl = lbe.tile_shapes()
    shapes = [(256, 128), (1536, 768)]
    c = autotune.candidates("f32", shapes, len(shapes_tbl), lambda k: shapes_tbl[k])
    segs = lambda k: sorted(s for kk, _, s in c if kk == k)  # noqa: E731
    assert segs(7) and segs(7) == segs(8)
    assert 0 in segs(8) and -1536 in segs(8)
    assert [k for k, _, _ in autotune.candidates("f64", shapes, len(shapes_tbl),
                                                lambda k: shapes_tbl[k])] == [0, 0]


@pytest.mark.gpu
def test_tune_restores_state_and_caches(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_6238_gb300.lbe import LBE
    monkeypatch.setenv("LBE_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    ws = wl.batch_sweep(n=3, seed=5, grids=((64, 128), (128, 256)))
    sim = LBE(ws, storage="f16dev")
    sim.step(4)
    before = [sim.get_state(j).numpy() for j in range(3)]
    best = autotune.tune(sim, steps=3, warmup=1)
    assert not best["cached"] and best["tried"]
    for j in range(3):
        assert np.array_equal(sim.get_state(j).numpy(), before[j])
    assert sim.steps_done == 4
    assert sim.get_tile()["kernel"] == best["kernel"]
    again = autotune.tune(LBE(ws, storage="f16dev"), steps=3)
    assert again["cached"] and again["kernel"] == best["kernel"]

"""Host logic of the schedule autotuner (no GPU): candidate choice, the
cache file, and the tile shapes the library reports."""
import json

import pytest

from paper_2209_01983_gb300 import autotune


def test_choose_takes_smallest_median():
    times = {"a": [5.0, 1.0, 5.0], "b": [2.0, 2.0, 2.0], "c": [9.0, 9.0, 0.5]}
    calls = {k: iter(v) for k, v in times.items()}
    best, med = autotune.choose(["a", "b", "c"], lambda c: next(calls[c]), repeats=3)
    assert best == "b"
    assert med == {"a": 5.0, "b": 2.0, "c": 9.0}


def test_choose_ties_go_to_the_first_candidate():
    best, _ = autotune.choose([3, 1, 2], lambda c: 1.0, repeats=1)
    assert best == 3


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    assert autotune.load_cache(p) == {}
    autotune.store_cache(p, "k1", {"shape": 2})
    autotune.store_cache(p, "k2", {"shape": 1, "order": 1})
    assert autotune.load_cache(p) == {"k1": {"shape": 2}, "k2": {"shape": 1, "order": 1}}
    with open(p, "w") as f:
        f.write("not json")
    assert autotune.load_cache(p) == {}
    json.dumps(autotune.load_cache(p))


def test_cache_path_follows_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("SALE_TUNE_CACHE", str(tmp_path / "x.json"))
    assert autotune.cache_path() == str(tmp_path / "x.json")
    monkeypatch.delenv("SALE_TUNE_CACHE")
    assert autotune.cache_path() == autotune.DEFAULT_CACHE


@pytest.fixture(scope="module")
def sale():
    from paper_2209_01983_gb300 import build
    build.build()
    from paper_2209_01983_gb300 import sale as s
    return s


def test_tile_shapes_from_library(sale):
    shapes = autotune.tile_shapes()
    assert [s for s, _, _ in shapes] == list(range(len(shapes)))
    assert shapes[0][1:] == (32, 8)
    assert len(shapes) >= 2
    for _, tx, ty in shapes:
        assert tx % 16 == 0 and (tx * ty) % 32 == 0 and tx * ty <= 1024  # whole warps, a legal block
    assert sale.sale_tile_shape(len(shapes), None, None) == sale.SALE_EINVAL
    assert sale.sale_tile_shape(-1, None, None) == sale.SALE_EINVAL


def test_tiling_calls_check_arguments(sale):
    assert sale.sale_set_tiling(None, 0) == sale.SALE_EINVAL
    assert sale.sale_batch_set_schedule(None, 0, 0) == sale.SALE_EINVAL

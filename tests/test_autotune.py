"""Host logic of the rasteriser autotuner (no GPU: the timing function is
injected): the coordinate-descent search, and the cache keyed by GPU,
workload, mode and library digest."""
import pytest

from paper_2606_11390_gb300 import autotune, scenes


def _fake_measure(table, calls):
    def measure(c):
        calls.append(autotune.name(c))
        t = {(8, 8): 9.0, (16, 16): 5.0, (32, 16): 4.0, (32, 32): 6.0}[c["tile"]]
        t += 0.5 if c["ppt"] == 2 else 0.0
        t += table.get(("f", c["batch_fwd"]), 0.0) + table.get(("b", c["batch_bwd"]), 0.0)
        return t
    return measure


def test_search_walks_each_dimension_once():
    calls = []
    best, times = autotune.search(_fake_measure({("f", 256): -0.3, ("b", 64): -0.2, ("b", 128): -0.1}, calls))
    assert best == {"tile": (32, 16), "ppt": 4, "batch_fwd": 256, "batch_bwd": 64}
    # 7 tile / pixel choices + 4 forward + 4 backward batches
    assert len(calls) == len(set(calls)) == 15
    assert set(times) == set(calls)
    assert min(times, key=times.get) == autotune.name(best)


def test_512_backward_batch_on_large_tiles():
    """A 512-splat backward batch is tried on 256-thread tiles too (its 49 KB
    of staging is opted in) and can win there; the shared-memory rule admits
    every batch size on every tile."""
    calls = []

    def measure(c):
        calls.append(c)
        return (1.0 if c["tile"] == (32, 32) and c["ppt"] == 4 else 9.0) - (0.5 if c["batch_bwd"] == 512 else 0.0)

    best, _ = autotune.search(measure)
    assert best == {"tile": (32, 32), "ppt": 4, "batch_fwd": 0, "batch_bwd": 512}
    assert any(c["batch_bwd"] == 512 for c in calls)
    for tile in autotune.TILES:
        for ppt in (2, 4):
            for b in autotune.BATCHES:
                for dim in ("batch_fwd", "batch_bwd"):
                    assert autotune.batch_supported({"tile": tile, "ppt": ppt}, dim, b)


def test_defaults_win_when_nothing_is_faster():
    best, _ = autotune.search(_fake_measure({}, []))
    assert best["batch_fwd"] == 0 and best["batch_bwd"] == 0


def test_tile_candidates_cover_the_kernel_variants():
    c = autotune.tile_candidates()
    assert {(x["tile"], x["ppt"]) for x in c} == {((8, 8), 2), ((16, 16), 2), ((16, 16), 4), ((32, 16), 2),
                                                  ((32, 16), 4), ((32, 32), 2), ((32, 32), 4)}


def test_cache_is_keyed_by_library_digest(tmp_path, monkeypatch):
    monkeypatch.setenv("GS_AUTOTUNE_CACHE", str(tmp_path / "t.json"))
    s = scenes.random_small(1, N=10)
    calls = []
    m = _fake_measure({("b", 128): -1.0}, calls)
    b1, t1 = autotune.best_config(s, measure=m, gpu="GPU", digest="aaaa")
    n = len(calls)
    b2, t2 = autotune.best_config(s, measure=m, gpu="GPU", digest="aaaa")
    assert (b2, t2) == (b1, t1) and len(calls) == n  # served from the cache
    autotune.best_config(s, measure=m, gpu="GPU", digest="bbbb")
    assert len(calls) == 2 * n  # a new library build is tuned afresh
    autotune.best_config(s, measure=m, gpu="other GPU", digest="aaaa")
    assert len(calls) == 3 * n
    autotune.best_config(scenes.random_small(1, N=11), measure=m, gpu="GPU", digest="aaaa")
    assert len(calls) == 4 * n  # another workload


def test_step_kwargs():
    kw = autotune.step_kwargs({"tile": (32, 16), "ppt": 2, "batch_fwd": 64, "batch_bwd": 0})
    assert kw == {"tile": (32, 16), "raster_px": 2, "raster_batch": (64, 0)}


def test_library_digest_is_stable():
    pytest.importorskip("hashlib")
    assert autotune.library_digest() == autotune.library_digest()


def test_names_round_trip():
    for c in autotune.tile_candidates():
        c = dict(c, batch_fwd=128, batch_bwd=256)
        assert autotune.parse_name(autotune.name(c)) == c
    with pytest.raises(ValueError):
        autotune.parse_name("32x16/4/f128/b256")

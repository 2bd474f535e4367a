"""Autotuner bookkeeping on the host: size buckets, cache before shipped
defaults, nearest-bucket fallback and shapes that always fit (no GPU: tile
shapes are checked with the library's host-side query)."""
import json

import pytest


@pytest.fixture()
def tune(monkeypatch, tmp_path):
    from paper_1803_01516_gb300 import build
    build.build()
    from paper_1803_01516_gb300 import autotune
    monkeypatch.setenv("GAZECUT_TUNE_CACHE", str(tmp_path / "cache.json"))
    return autotune


def test_buckets(tune):
    from paper_1803_01516_gb300 import gazecut as gc
    p = gc.Params(w=384, h=288, D=16, tau=30, lam=10)
    assert tune.bucket(p) == "D16-n21"          # 354*288*15 = 1.53 M nodes
    assert tune.bucket(gc.Params(w=640, h=480, D=64, tau=30, lam=10)) == "D64-n24"
    assert tune.bucket(gc.Params(w=100, h=50, D=13, tau=30, lam=10)).startswith("D16-")


def test_cache_overrides_shipped_defaults(tune):
    from paper_1803_01516_gb300 import gazecut as gc
    p = gc.Params(w=384, h=288, D=16, tau=30, lam=10)
    shipped = tune.tuned_opts(p)
    assert (shipped.tile_w, shipped.tile_h) != (0, 0)
    with open(tune.cache_path(), "w") as f:
        json.dump({tune.bucket(p): {"best": [8, 16, 4, 8, 8], "ms": 1.0}}, f)
    o = tune.tuned_opts(p)
    assert (o.sweeps_per_relabel, o.local_iters, o.relabel_passes, o.tile_w, o.tile_h) == \
        (8, 16, 4, 8, 8)


def test_nearest_bucket_and_fit(tune):
    from paper_1803_01516_gb300 import gazecut as gc
    # no entry for 128 depth numbers: the nearest bucket's schedule, a shape
    # that fits (the borrowed one is too large for 127 layers)
    p = gc.Params(w=1920, h=1080, D=128, tau=30, lam=10)
    o = tune.tuned_opts(p)
    info = gc.gs_tile_info(p, o)
    assert info["smem_bytes"] <= 180 * 1024
    assert o.sweeps_per_relabel >= 1 and o.local_iters >= 1


def test_unparseable_keys_are_ignored(tune):
    from paper_1803_01516_gb300 import gazecut as gc
    table = {"junk": {"best": [1, 1, 1]}, "D16-n20": {"best": [32, 4, 8, 16, 8]}}
    p = gc.Params(w=384, h=288, D=16, tau=30, lam=10)
    assert tune._nearest(table, p)["best"] == [32, 4, 8, 16, 8]


def test_block_size_entry(tune):
    """A seventh entry element sets the threads per block; the library's own
    shape for 256-thread blocks keeps two tiles within an SM's shared memory."""
    from paper_1803_01516_gb300 import gazecut as gc
    p = gc.Params(w=384, h=288, D=16, tau=30, lam=10)
    with open(tune.cache_path(), "w") as f:
        json.dump({tune.bucket(p): {"best": [16, 8, 16, 8, 8, 16, 256], "ms": 1.0}}, f)
    o = tune.tuned_opts(p)
    assert o.cta_threads == 256 and (o.tile_w, o.tile_h, o.tail_iters) == (8, 8, 16)
    info = gc.gs_tile_info(p, gc.SolveOpts(cta_threads=256))
    assert (info["tile_w"], info["tile_h"]) == (8, 8)
    assert 2 * (info["smem_bytes"] + 26 * 1024) <= 228 * 1024
    # 512 threads (the default) take the larger tile
    info = gc.gs_tile_info(p, gc.SolveOpts())
    assert info["tile_w"] * info["tile_h"] > 64


def test_tune_on_callers_pairs(tune, monkeypatch):
    """tune() measures on the caller's own pairs when given (shapes checked),
    keeps the fastest configuration of both stages and caches it under the
    size bucket.  The timer is replaced by a host-side cost model here."""
    import torch
    from paper_1803_01516_gb300 import gazecut as gc
    p = gc.Params(w=100, h=40, D=8, tau=30, lam=10)
    mine = [(torch.zeros(40, 100, dtype=torch.uint8), torch.zeros(40, 100, dtype=torch.uint8))]
    seen = []

    def fake_time(pp, pairs, cfg, reps=2):
        seen.append(pairs)
        spr, li, rp, tw, th = cfg[:5]
        ti = cfg[5] if len(cfg) > 5 else 0
        bt = cfg[6] if len(cfg) > 6 else 0
        # fastest: 8x4 tiles on 256 threads, then 32 sweeps per relabel, 4
        # local iterations, 8 passes, tail 8
        return (abs(tw - 8) + abs(th - 4) + (bt != 256) + abs(spr - 32) / 8 + abs(li - 4)
                + abs(rp - 8) / 4 + abs(ti - 8) / 4)

    monkeypatch.setattr(tune, "_time_config", fake_time)
    e = tune.tune(p, pairs=mine)
    assert e["best"] == [32, 4, 8, 8, 4, 8, 256]
    assert all(s == mine for s in seen) and len(seen) > 10
    o = tune.tuned_opts(p)
    assert (o.sweeps_per_relabel, o.local_iters, o.relabel_passes, o.tile_w, o.tile_h,
            o.tail_iters, o.cta_threads) == (32, 4, 8, 8, 4, 8, 256)
    with pytest.raises(ValueError):
        tune.tune(p, pairs=[(torch.zeros(40, 99, dtype=torch.uint8),) * 2])
    with pytest.raises(ValueError):
        tune.tune(p, pairs=[])


def test_block_size_shapes_fit_every_depth_range(tune):
    """With 256-thread blocks the library's own tile fits two blocks' shared
    memory in an SM up to 64 depth numbers and falls back to one block per SM
    for longer chains; explicit shapes keep the one-block budget."""
    from paper_1803_01516_gb300 import gazecut as gc
    for D in (4, 16, 33, 64, 128, 200):
        p = gc.Params(w=2 * (D - 1) + 200, h=120, D=D, tau=30, lam=10)
        info = gc.gs_tile_info(p, gc.SolveOpts(cta_threads=256))
        assert info["smem_bytes"] <= 180 * 1024
        if D <= 64:
            assert info["smem_bytes"] <= 80 * 1024, (D, info)
        # a tile's own nodes: at most 8 per thread of the 256
        assert info["tile_w"] * info["tile_h"] * (D - 1) <= 8 * 256
    p = gc.Params(w=384, h=288, D=16, tau=30, lam=10)
    info = gc.gs_tile_info(p, gc.SolveOpts(cta_threads=256, tile_w=16, tile_h=8))
    assert (info["tile_w"], info["tile_h"]) == (16, 8) and info["smem_bytes"] > 80 * 1024

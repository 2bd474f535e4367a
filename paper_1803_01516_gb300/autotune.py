"""Autotuner for the solver schedule, per problem-size bucket, cached in JSON.

What is tuned: the tile shape (sites per tile along W and y; every tile holds
whole depth chains) and the schedule (sweep rounds between global relabels,
local push/relabel iterations per tile visit, the pass cap of intermediate
relabels; an entry may add the local iterations of a tail visit as a sixth
value).  A bucket is (depth numbers, log2 of the node count); its entry is
measured on seeded synthetic pairs of that size (the same scene generator as
the tests) with CUDA events, the best median over a few runs kept.

The cache lives in $GAZECUT_TUNE_CACHE or ~/.cache/gazecut_gb300/autotune.json;
buckets missing there fall back to ``tuned_defaults.json`` beside this module
(entries measured on a GB300 with ``python -m paper_1803_01516_gb300.autotune``),
then to the library defaults.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import gazecut as gc
from . import synth

SCHEDULES = [(spr, li, rp, tf) for spr in (8, 16, 32, 64) for li in (4, 8, 16) for rp in (4, 8, 16)
             for tf in (2, 4)]       # tf: tail iterations = tf x local iterations
SHAPES = [(16, 8), (8, 8), (16, 4), (32, 4), (8, 4), (16, 2), (8, 2), (4, 4)]
CTA_THREADS = (512, 256)     # one block per SM, or two half-size blocks


def cache_path() -> str:
    return os.environ.get("GAZECUT_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gazecut_gb300",
                                       "autotune.json"))


def _key(D: int, nodes: int):
    return 8 * int(round(D / 8)), int(round(math.log2(max(nodes, 1))))


def bucket(p: gc.Params) -> str:
    """(depth numbers rounded to a multiple of 8, log2 of the node count)."""
    d, n = _key(p.D, p.ng * p.h * (p.D - 1))
    return f"D{d}-n{n}"


def _nearest(table: dict, p: gc.Params):
    """Entry of the bucket nearest to p's (same depth group first)."""
    d, n = _key(p.D, p.ng * p.h * (p.D - 1))
    best, dist = None, None
    for k, v in table.items():
        try:
            kd, kn = (int(x[1:]) for x in k.split("-"))
        except ValueError:
            continue
        dd = abs(kd - d) * 4 + abs(kn - n)
        if dist is None or dd < dist:
            best, dist = v, dd
    return best


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d: dict):
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_config(p: gc.Params, pairs, cfg, reps: int = 2) -> float:
    spr, li, rp, tw, th = cfg[:5]
    ti = cfg[5] if len(cfg) > 5 else 0
    bt = cfg[6] if len(cfg) > 6 else 0
    o = gc.SolveOpts(sweeps_per_relabel=spr, local_iters=li, relabel_passes=rp, tile_w=tw,
                     tile_h=th, tail_iters=ti, cta_threads=bt)
    try:
        gc.gs_tile_info(p, o)
    except RuntimeError:
        return float("inf")          # the shape does not fit this depth range
    buf = gc.Buffers(p, o)
    ts = []
    for L, R in pairs:
        gc.gs_stereo_cost_volume(L, R, p, buf.cost)
        for _ in range(reps):
            gc.gs_build_graph(buf.cost, p, buf.graph, buf.status)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            try:
                gc.gs_maxflow_solve(buf.graph, p, o, buf.work, buf.status)
            except RuntimeError:
                return float("inf")
            b.record()
            b.synchronize()
            if int(buf.status.item()) != gc.GS_OK:
                return float("inf")
            ts.append(a.elapsed_time(b))
    ts.sort()
    return ts[len(ts) // 2]


def tune(p: gc.Params, n_pairs: int = 2, save: bool = True, pairs=None) -> dict:
    """Tile shape and block size first (default schedule), then the schedule on
    the best of those, each measured on `pairs` -- the caller's own image
    pairs of p's size, a list of (left, right) uint8 device tensors -- or, by
    default, on n_pairs synthetic pairs of that size.  An entry is
    [sweeps_per_relabel, local_iters, relabel_passes, tile_w, tile_h,
    tail_iters, cta_threads]."""
    if pairs is None:
        wl = synth.Workload(f"tune-{bucket(p)}", p.w, p.h, p.D, tau=30, lam=p.lam, sigma=2.0,
                            scene="layers", n_layers=5, n_slanted=2,
                            max_disp=min(2 * (p.D - 1), 40), seed_base=77)
        pairs = []
        for i in range(n_pairs):
            L, R, _ = synth.make_pair(wl, i)
            pairs.append((torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()))
    else:
        pairs = list(pairs)
        if not pairs:
            raise ValueError("tune: no pairs to measure on")
        for L, R in pairs:
            if tuple(L.shape) != (p.h, p.w) or tuple(R.shape) != (p.h, p.w):
                raise ValueError(f"tune: pair of shape {tuple(L.shape)} / {tuple(R.shape)}, "
                                 f"expected {(p.h, p.w)}")
    results = {}
    for tw, th in SHAPES:
        for bt in CTA_THREADS:
            results[f"16,8,8,{tw},{th},0,{bt}"] = _time_config(p, pairs, (16, 8, 8, tw, th, 0, bt))
    first = [int(x) for x in min(results, key=results.get).split(",")]
    tw, th, bt = first[3], first[4], first[6]
    for spr, li, rp, tf in SCHEDULES:
        key = f"{spr},{li},{rp},{tw},{th},{tf * li},{bt}"
        if key not in results:
            results[key] = _time_config(p, pairs, (spr, li, rp, tw, th, tf * li, bt))
    best = min(results, key=results.get)
    entry = {"best": [int(x) for x in best.split(",")], "ms": results[best], "all_ms": results}
    if save:
        d = _load()
        d[bucket(p)] = entry
        _save(d)
    return entry


def _defaults() -> dict:
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                               "tuned_defaults.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tuned_opts(p: gc.Params, tune_if_missing: bool = False, **kw) -> gc.SolveOpts:
    """Solve options for p from the cache (library defaults when absent)."""
    entry = _load().get(bucket(p)) or _defaults().get(bucket(p))
    if entry is None and tune_if_missing:
        entry = tune(p)
    if entry is None:
        entry = _nearest(_load(), p) or _nearest(_defaults(), p)
    if entry is None:
        return gc.SolveOpts(**kw)
    best = entry["best"]
    spr, li, rp = best[:3]
    tw, th = (best[3], best[4]) if len(best) >= 5 else (0, 0)
    ti = best[5] if len(best) >= 6 else 0          # tail iterations (0: library default)
    bt = best[6] if len(best) >= 7 else 0          # threads per block (0: library default)
    o = gc.SolveOpts(sweeps_per_relabel=spr, local_iters=li, relabel_passes=rp, tile_w=tw,
                     tile_h=th, tail_iters=ti, cta_threads=bt, **kw)
    try:
        gc.gs_tile_info(p, o)
    except RuntimeError:
        # a shape borrowed from another bucket may not fit this depth range:
        # let the library choose one
        o.tile_w = o.tile_h = 0
    return o


if __name__ == "__main__":
    import sys
    # tune the buckets given as w,h,D triples (default: the benchmark's size),
    # or, with --defaults, a size for every bucket of tuned_defaults.json
    if sys.argv[1:] == ["--defaults"]:
        sizes = []
        for k in sorted(_defaults()):
            d, n = (int(x[1:]) for x in k.split("-"))
            h = 240
            ng = max(8, round(2 ** n / (h * (d - 1))))
            sizes.append((ng + 2 * (d - 1), h, d))
    else:
        sizes = [tuple(int(x) for x in a.split(",")) for a in sys.argv[1:]] or [(384, 288, 16)]
    for w, h, D in sizes:
        p = gc.Params(w=w, h=h, D=D, tau=30, lam=10)
        e = tune(p)
        print(json.dumps({bucket(p): e}), flush=True)

"""Seeded synthetic rectified stereo pairs (the stand-in for the paper's Middlebury input, §4.1).

This module only draws images and ground-truth disparity maps.  It holds none
of the method's arithmetic (no cost volume, no graph, no cut): both the CUDA
path and the CPU oracle consume the arrays it returns, so neither side can
drift from the other through its inputs.

Scene recipe (one recipe, parameterised per workload):

* texture: left image ``L`` = uniform integers 0..255, 3x3 box blur, uint8;
* layers: a disparity map ``d_R(x, y)`` in right-image coordinates, built as a
  z-buffer over fronto-parallel or slanted layers ``d = a + b*x + c*y``
  (the largest disparity, i.e. the nearest surface, wins), rounded with
  ``floor(d + 0.5)``;
* warp: ``R(x, y) = L(min(x + d_R(x, y), w - 1), y)``, which leaves the
  occluded band left of every foreground edge that the paper's visibility term
  (§3, Fig. 3) is about;
* noise: Gaussian noise of standard deviation ``sigma`` added to ``R`` only,
  rounded half-to-even and clipped to 0..255.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

__all__ = ["Workload", "TINY", "MAIN", "LARGE", "make_pair", "make_pair_rgb", "make_batch",
           "random_costs"]


@dataclass(frozen=True)
class Workload:
    """One named synthetic workload: image size, depth numbers and scene recipe."""

    name: str
    w: int
    h: int
    D: int                 # number of depth numbers (labels)
    tau: int               # truncation of the absolute-difference data cost
    lam: int               # penalty h~1 (smoothness weight)
    inhibit: int = 1023    # inhibit h~2 (visibility weight), the paper's value (§4.3)
    sigma: float = 2.0     # noise on the right image
    scene: str = "rects"   # "rects" | "layers" | "planes"
    n_layers: int = 3
    n_slanted: int = 0
    max_disp: int = 12
    rect_disps: tuple = (2, 7, 12)
    seed_base: int = 0     # seed = seed_base * 1000 + pair index


# 64x48, 16 depth numbers: 3 fronto-parallel rectangles (disparities 2, 7, 12).
TINY = Workload("tiny-64x48x16", 64, 48, 16, tau=30, lam=8, sigma=2.0,
                scene="rects", rect_disps=(2, 7, 12), max_disp=12, seed_base=1)
# 384x288, 16 depth numbers: 5 piecewise-planar layers, 2 slanted, max disparity 15.
MAIN = Workload("main-384x288x16", 384, 288, 16, tau=30, lam=10, sigma=3.0,
                scene="layers", n_layers=5, n_slanted=2, max_disp=15, seed_base=2)
# 1920x1080, 128 depth numbers: 12 random slanted planes, random depth order.
LARGE = Workload("large-1920x1080x128", 1920, 1080, 128, tau=40, lam=12, sigma=2.0,
                 scene="planes", n_layers=12, n_slanted=12, max_disp=254, seed_base=3)


def _box_blur3(a: np.ndarray) -> np.ndarray:
    p = np.pad(a.astype(np.int32), 1, mode="edge")
    s = np.zeros_like(a, dtype=np.int32)
    for dy in range(3):
        for dx in range(3):
            s += p[dy:dy + a.shape[0], dx:dx + a.shape[1]]
    return ((s + 4) // 9).astype(np.uint8)


def _layer_disparity(rng: np.random.Generator, wl: Workload) -> np.ndarray:
    """Z-buffered integer disparity map d_R[y, x] (right-image coordinates)."""
    w, h = wl.w, wl.h
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    d = np.zeros((h, w), dtype=np.float64)
    if wl.scene == "rects":
        for disp in wl.rect_disps:
            rw = int(rng.integers(w // 6, w // 3 + 1))
            rh = int(rng.integers(h // 6, h // 3 + 1))
            x0 = int(rng.integers(0, w - rw))
            y0 = int(rng.integers(0, h - rh))
            m = (xx >= x0) & (xx < x0 + rw) & (yy >= y0) & (yy < y0 + rh)
            d = np.where(m, np.maximum(d, float(disp)), d)
    else:
        # background: a gentle plane well behind the layers
        if wl.scene == "planes":
            d[:] = rng.uniform(0, 0.25 * wl.max_disp)
        n = wl.n_layers
        slanted = set(rng.choice(n, size=min(wl.n_slanted, n), replace=False).tolist())
        # layer depth order: bases spread over [0.3, 1] * max_disp, the nearest
        # layer exactly at max_disp (fronto-parallel), drawn in random order
        bases = np.sort(rng.uniform(0.3, 1.0, size=n)) * wl.max_disp
        bases[-1] = wl.max_disp
        order = rng.permutation(n)
        for i in order:
            cx, cy = rng.uniform(0, w), rng.uniform(0, h)
            ax = rng.uniform(w * 0.08, w * 0.3)
            ay = rng.uniform(h * 0.08, h * 0.3)
            base = bases[i]
            if i in slanted and i != n - 1:
                # d = base + b*(x-cx) + c*(y-cy), varying by up to 30% of max_disp over the patch
                b = rng.uniform(-1, 1) * 0.15 * wl.max_disp / max(ax, 1.0)
                c = rng.uniform(-1, 1) * 0.15 * wl.max_disp / max(ay, 1.0)
            else:
                b = c = 0.0
            plane = np.clip(base + b * (xx - cx) + c * (yy - cy), 0, wl.max_disp)
            if wl.scene == "layers" and rng.random() < 0.5:
                m = ((xx - cx) / ax) ** 2 + ((yy - cy) / ay) ** 2 <= 1.0
            else:
                m = (np.abs(xx - cx) <= ax) & (np.abs(yy - cy) <= ay)
            d = np.where(m, np.maximum(d, plane), d)
    d = np.floor(d + 0.5)
    return np.clip(d, 0, wl.max_disp).astype(np.int32)


def make_pair(wl: Workload, index: int = 0):
    """Return (L, R, d_R) for pair ``index`` of workload ``wl``.

    L, R: uint8 [h, w] (C-contiguous); d_R: int32 [h, w] ground-truth disparity
    of each right-image pixel (x_l = x_r + d_R).
    """
    rng = np.random.default_rng(wl.seed_base * 1000 + index)
    tex = rng.integers(0, 256, size=(wl.h, wl.w), dtype=np.int32).astype(np.uint8)
    L = _box_blur3(tex)
    dR = _layer_disparity(rng, wl)
    xs = np.minimum(np.arange(wl.w)[None, :] + dR, wl.w - 1)
    R = np.take_along_axis(L, xs, axis=1).astype(np.float64)
    R = R + rng.normal(0.0, wl.sigma, size=R.shape)
    R = np.clip(np.rint(R), 0, 255).astype(np.uint8)
    return np.ascontiguousarray(L), np.ascontiguousarray(R), dR


def make_pair_rgb(wl: Workload, index: int = 0):
    """Colour version of ``make_pair``: the same scene recipe with an
    independent texture per channel.  Returns (L, R, d_R) with L, R uint8
    [h, w, 3] (interleaved R, G, B per pixel) and d_R int32 [h, w]."""
    rng = np.random.default_rng(wl.seed_base * 1000 + 500 + index)
    tex = rng.integers(0, 256, size=(3, wl.h, wl.w), dtype=np.int32).astype(np.uint8)
    L = np.stack([_box_blur3(tex[c]) for c in range(3)], axis=-1)
    dR = _layer_disparity(rng, wl)
    xs = np.minimum(np.arange(wl.w)[None, :] + dR, wl.w - 1)
    R = np.stack([np.take_along_axis(L[:, :, c], xs, axis=1) for c in range(3)], axis=-1)
    R = R.astype(np.float64) + rng.normal(0.0, wl.sigma, size=R.shape)
    R = np.clip(np.rint(R), 0, 255).astype(np.uint8)
    return np.ascontiguousarray(L), np.ascontiguousarray(R), dR


def make_batch(n: int = 64, seed_base: int = 4, wmin=160, wmax=640, hmin=120, hmax=480,
               dmin=16, dmax=64):
    """Uneven batch: sizes ~U[wmin,wmax] x U[hmin,hmax], depth numbers ~U[dmin,dmax]."""
    rng = np.random.default_rng(seed_base * 1000)
    out = []
    for i in range(n):
        w = int(rng.integers(wmin, wmax + 1))
        h = int(rng.integers(hmin, hmax + 1))
        D = int(rng.integers(dmin, dmax + 1))
        w = max(w, 2 * (D - 1) + 8)
        wl = Workload(f"batch-{i}", w, h, D, tau=30, lam=10, sigma=2.0, scene="layers",
                      n_layers=int(rng.integers(3, 7)), n_slanted=1,
                      max_disp=min(2 * (D - 1), 40), seed_base=seed_base)
        L, R, dR = make_pair(replace(wl, seed_base=seed_base * 100 + i), 0)
        out.append((wl, L, R, dR))
    return out


def random_costs(rng: np.random.Generator, n_g: int, h: int, D: int, hi: int) -> np.ndarray:
    """Uniform integer data costs C[y, W, S] in [0, hi] (for solver-only tests)."""
    return rng.integers(0, hi + 1, size=(h, n_g, D), dtype=np.int32)

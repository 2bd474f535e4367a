"""Level-1 hierarchical approximation of §4.5 (test infrastructure only).

The paper combines 2x2x2 or 3x3x3 neighbouring cross points into one delegate
point, cuts the delegate graph first, then cuts again exactly among the cross
points of a thin skin around the first cut; block size 1 is the exact
minimisation.  It does not give the delegate data term, the delegate
interaction or the thickness of the skin, so this oracle fixes them (the CUDA
path implements the same definitions independently):

* delegate grid  block size b: delegate site (Wc, yc) stands for the sites
                 W in [b Wc, b Wc + b), y in [b yc, b yc + b) (fewer at the
                 far edges), delegate depth number Lc for the depth numbers
                 [b Lc, b Lc + b) (fewer in the last bin); n_gc = ceil(n_g/b),
                 h_c = ceil(h/b), D_c = ceil(D/b)
* delegate data  Cc[yc, Wc, Lc] = sum over the block's sites of the smallest
                 data term in the depth bin (the best cross point each gaze
                 line has inside the delegate)
* delegate pairs the interaction of §3 with h~1 and h~2 multiplied by b (a
                 delegate pair stands for b neighbouring site pairs along the
                 block border)
* thin skin      a site whose delegate has label Lc keeps the depth numbers
                 [b Lc - b, b Lc + 2b - 1] clipped to [0, D-1]: its delegate's
                 bin and one bin on each side
* second cut     exact minimum of E(X) (§2) over labelings inside the skin
                 (``solve_band``), canonical smallest minimiser

With b = 1 the delegate problem is the problem itself and its minimiser lies
inside the skin, so the result is the exact canonical minimiser.
"""
from __future__ import annotations

import numpy as np

from . import solve, solve_band, energy


def coarse_shape(h: int, ng: int, D: int, b: int):
    return -(-h // b), -(-ng // b), -(-D // b)


def coarse_costs(C: np.ndarray, b: int) -> np.ndarray:
    """Delegate data term, int64 [h_c, n_gc, D_c] (plain loops over blocks)."""
    C = np.asarray(C, dtype=np.int64)
    h, ng, D = C.shape
    hc, ngc, Dc = coarse_shape(h, ng, D, b)
    Cc = np.zeros((hc, ngc, Dc), dtype=np.int64)
    for yc in range(hc):
        for Wc in range(ngc):
            block = C[yc * b:(yc + 1) * b, Wc * b:(Wc + 1) * b, :]
            for Lc in range(Dc):
                Cc[yc, Wc, Lc] = block[:, :, Lc * b:(Lc + 1) * b].min(axis=2).sum()
    return Cc


def skin_bounds(Xc: np.ndarray, b: int, h: int, ng: int, D: int):
    """Per-site depth bounds lo, hi (int32 [h, n_g]) around delegate labels Xc."""
    Xc = np.asarray(Xc, dtype=np.int64)
    lo = np.zeros((h, ng), dtype=np.int32)
    hi = np.zeros((h, ng), dtype=np.int32)
    for y in range(h):
        for W in range(ng):
            Lc = int(Xc[y // b, W // b])
            lo[y, W] = max(0, b * Lc - b)
            hi[y, W] = min(D - 1, b * Lc + 2 * b - 1)
    return lo, hi


def level1(C: np.ndarray, lam: int, inhibit: int, vinhibit: int, b: int):
    """Returns dict(labels, energy, coarse_labels, lo, hi)."""
    h, ng, D = np.asarray(C).shape
    Cc = coarse_costs(C, b)
    assert Cc.max(initial=0) < 2 ** 31
    first = solve(Cc.astype(np.int32), b * lam, b * inhibit, vinhibit)
    lo, hi = skin_bounds(first["labels"], b, h, ng, D)
    second = solve_band(C, lam, inhibit, vinhibit, lo, hi)
    X = second["labels"]
    return {"labels": X, "energy": energy(C, X, lam, inhibit, vinhibit),
            "coarse_labels": first["labels"], "lo": lo, "hi": hi}

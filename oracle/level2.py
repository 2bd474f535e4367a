"""Level-2 hierarchical approximation of §4.5 (test infrastructure only).

The paper's level 2 keeps level 1's first (delegate) cut and thin skin, but its
push-relabel loop "cuts each block separately" while an undisclosed wave-front
pass handles the skin as a whole.  This oracle fixes a reading that can be
checked:

* first cut, skin   as level 1 (``level1``): delegate labels Xc, per-site
                    bounds lo <= X <= hi
* start labels      each site takes its best cross point inside its delegate's
                    depth bin: the first argmin of C_v over
                    [b Xc, min(b Xc + b - 1, D - 1)]
* block cut         block (bx, by) = the b x b sites of one delegate; with
                    every site outside the block held at its current label,
                    the block's labels become the exact minimum of E(X) (§2)
                    inside the skin, canonical smallest minimiser -- the pairs
                    that leave the block turn into unary terms h~(l - X_u) of
                    the block site (the interaction of §3)
* order             blocks coloured like a checkerboard ((bx + by) mod 2); a
                    pass cuts every colour-0 block, then every colour-1 block
                    with the new colour-0 labels (blocks of one colour share
                    no pair, so each half-pass is an exact minimisation over
                    their sites and E never increases)

The wave-front pass's role -- coupling the blocks -- is played by the
neighbours' labels in the border terms.
"""
from __future__ import annotations

import numpy as np

from . import energy, solve, solve_band
from .level1 import coarse_costs, skin_bounds
from .small import htilde


def start_labels(C: np.ndarray, Xc: np.ndarray, b: int) -> np.ndarray:
    """First argmin of each site's data term inside its delegate's depth bin."""
    C = np.asarray(C)
    h, ng, D = C.shape
    X = np.zeros((h, ng), dtype=np.int32)
    for y in range(h):
        for W in range(ng):
            a = b * int(Xc[y // b, W // b])
            z = min(a + b, D)
            X[y, W] = a + int(np.argmin(C[y, W, a:z]))
    return X


def border_costs(C, X, lam, inhibit, vinhibit, b):
    """Data terms of every site with the pairs that leave the site's block
    (b x b sites, blocks aligned at 0) folded in against the neighbour's label
    in X: C_v(l) + sum over such neighbours u of h~(l - X_u), int64 [h, n_g, D]."""
    C = np.asarray(C, dtype=np.int64)
    X = np.asarray(X, dtype=np.int64)
    h, ng, D = C.shape
    l = np.arange(D)[None, None, :]
    yy, ww = np.meshgrid(np.arange(h), np.arange(ng), indexing="ij")
    out = C.copy()
    for dy, dW in ((0, -1), (0, 1), (-1, 0), (1, 0)):
        yu, wu = yy + dy, ww + dW
        inside = (yu >= 0) & (yu < h) & (wu >= 0) & (wu < ng)
        other_block = inside & ((yu // b != yy // b) | (wu // b != ww // b))
        xu = np.where(inside, X[np.clip(yu, 0, h - 1), np.clip(wu, 0, ng - 1)], 0)
        inh = inhibit if (dy == 0 or vinhibit) else 0
        out += np.where(other_block[:, :, None], htilde(l - xu[:, :, None], lam, inh), 0)
    return out


def block_descent(C, X, lam, inhibit, vinhibit, b, lo, hi, passes, trace=None):
    """`passes` two-colour passes of exact block cuts on a copy of X.  trace
    (a list) receives E after every half-pass."""
    C = np.asarray(C)
    h, ng, D = C.shape
    X = np.array(X, dtype=np.int32, copy=True)
    nby, nbx = -(-h // b), -(-ng // b)
    for _ in range(passes):
        for colour in (0, 1):
            Cb_all = border_costs(C, X, lam, inhibit, vinhibit, b)
            assert Cb_all.max() < 2 ** 31
            new = X.copy()
            for by in range(nby):
                for bx in range(nbx):
                    if (bx + by) % 2 != colour:
                        continue
                    y0, W0 = by * b, bx * b
                    y1, W1 = min(y0 + b, h), min(W0 + b, ng)
                    r = solve_band(Cb_all[y0:y1, W0:W1].astype(np.int32), lam, inhibit, vinhibit,
                                   lo[y0:y1, W0:W1], hi[y0:y1, W0:W1])
                    new[y0:y1, W0:W1] = r["labels"]
            X = new
            if trace is not None:
                trace.append(energy(C, X, lam, inhibit, vinhibit))
    return X


def level2(C: np.ndarray, lam: int, inhibit: int, vinhibit: int, b: int, passes: int = 2):
    """Returns dict(labels, energy, coarse_labels, lo, hi, start, trace)."""
    C = np.asarray(C)
    h, ng, D = C.shape
    Cc = coarse_costs(C, b)
    assert Cc.max(initial=0) < 2 ** 31
    first = solve(Cc.astype(np.int32), b * lam, b * inhibit, vinhibit)
    lo, hi = skin_bounds(first["labels"], b, h, ng, D)
    X0 = start_labels(C, first["labels"], b)
    trace = [energy(C, X0, lam, inhibit, vinhibit)]
    X = block_descent(C, X0, lam, inhibit, vinhibit, b, lo, hi, passes, trace)
    return {"labels": X, "energy": energy(C, X, lam, inhibit, vinhibit),
            "coarse_labels": first["labels"], "lo": lo, "hi": hi, "start": X0, "trace": trace}

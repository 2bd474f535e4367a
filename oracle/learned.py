"""Learned data term and the adjoint of the minimum energy (test infrastructure).

* ``dx``                central difference (I[x+1] - I[x-1]) / 2, replicated border
* ``cost_volume_f32``   c = w1 |L - R| + w2 |dxL - dxR| at every cross point (§3
                        geometry), min(c, tau), then rint(scale * c) -- in float32
                        with every product and sum rounded on its own, the
                        precision the quantised code is decided in
* ``cost_grad_sums``    the chain rule through that cost at given labels
* ``energy_adjoint``    dE/dC = one-hot of the labels, dE/dlambda = number of
                        label jumps, dE/dinhibit = jumps beyond one (§2, §3 h~)

The adjoint is pinned in ``tests/test_learning.py`` by the concavity of the
minimum energy: forward and backward differences of the oracle's own E*
bracket it.
"""
from __future__ import annotations

import numpy as np


def dx(I: np.ndarray) -> np.ndarray:
    I = np.asarray(I, dtype=np.float32)
    Ip = np.concatenate([I[:, 1:], I[:, -1:]], axis=1)
    Im = np.concatenate([I[:, :1], I[:, :-1]], axis=1)
    return np.float32(0.5) * (Ip - Im)


def _features(L, R, D, dis0):
    """a[y, W, S] = |L - R|, b[y, W, S] = |dxL - dxR| at cross point (W, S, y)."""
    L = np.asarray(L)
    R = np.asarray(R)
    h, w = L.shape
    ng = w - dis0
    Lf, Rf = L.astype(np.float32), R.astype(np.float32)
    dL, dR = dx(L), dx(R)
    a = np.zeros((h, ng, D), np.float32)
    b = np.zeros((h, ng, D), np.float32)
    W = np.arange(ng)
    for S in range(D):
        xr, xl = W + S, W + dis0 - S
        a[:, :, S] = np.abs(Lf[:, xl] - Rf[:, xr])
        b[:, :, S] = np.abs(dL[:, xl] - dR[:, xr])
    return a, b


def cost_volume_f32(L, R, D, dis0, w1, w2, tau, scale=256.0):
    a, b = _features(L, R, D, dis0)
    c = np.float32(w1) * a + np.float32(w2) * b          # float32, each op rounded
    c = np.minimum(c, np.float32(tau))
    return np.rint(np.float32(scale) * c).astype(np.int32)


def cost_grad_sums(L, R, D, dis0, w1, w2, tau, X):
    """(sum |L-R| [c<tau], sum 2|dxL-dxR| [c<tau], sum [c>=tau]) at labels X."""
    a, b = _features(L, R, D, dis0)
    h, ng = X.shape
    yy, ww = np.meshgrid(np.arange(h), np.arange(ng), indexing="ij")
    av, bv = a[yy, ww, X], b[yy, ww, X]
    c = np.float32(w1) * av + np.float32(w2) * bv
    inside = c < np.float32(tau)
    return (int(av[inside].astype(np.int64).sum()), int((2 * bv[inside]).astype(np.int64).sum()),
            int((~inside).sum()))


def energy_adjoint(X: np.ndarray, D: int, vinhibit: int = 1):
    """(one-hot dE/dC [h, n_g, D], jumps, jumps beyond one on inhibit pairs)."""
    X = np.asarray(X, dtype=np.int64)
    h, ng = X.shape
    onehot = np.zeros((h, ng, D), np.float32)
    yy, ww = np.meshgrid(np.arange(h), np.arange(ng), indexing="ij")
    onehot[yy, ww, X] = 1.0
    dh = np.abs(np.diff(X, axis=1))
    dv = np.abs(np.diff(X, axis=0))
    jumps = int(dh.sum() + dv.sum())
    viol = int(np.maximum(dh - 1, 0).sum() + (np.maximum(dv - 1, 0).sum() if vinhibit else 0))
    return onehot, jumps, viol

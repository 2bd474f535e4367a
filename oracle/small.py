"""Small-case solvers that pin the max-flow oracle (test infrastructure only).

* ``energy_np``     E(X) of §2 with the interaction h~ of §3, vectorised over
                    many labelings at once.
* ``brute_force``   every labeling of a tiny grid (D^n of them): the exact
                    minimum and the component-wise smallest minimiser.
* ``brute_force_band``  every labeling inside per-site bounds lo <= X <= hi:
                    the restricted minimum and its smallest minimiser.
* ``viterbi_row``   one row of sites with no vertical pairs is a chain MRF;
                    min-sum dynamic programming gives its exact minimum, and
                    forward + backward messages give, per site, the smallest
                    label used by any minimiser.
"""
from __future__ import annotations

import itertools

import numpy as np


def htilde(delta, lam: int, inhibit: int):
    """h~(δ) = h~1|δ| + h~2 (|δ|-1) T(|δ|>1)  (§3)."""
    d = np.abs(np.asarray(delta, dtype=np.int64))
    return lam * d + inhibit * np.maximum(d - 1, 0)


def energy_np(C: np.ndarray, X: np.ndarray, lam: int, inhibit: int, vinhibit: int = 1) -> np.ndarray:
    """E for a stack of labelings X[..., h, n_g] over costs C[h, n_g, D]."""
    C = np.asarray(C, dtype=np.int64)
    X = np.asarray(X, dtype=np.int64)
    h, ng, D = C.shape
    yy, ww = np.meshgrid(np.arange(h), np.arange(ng), indexing="ij")
    E = C[yy, ww, X].sum(axis=(-2, -1))
    E = E + htilde(X[..., :, 1:] - X[..., :, :-1], lam, inhibit).sum(axis=(-2, -1))
    E = E + htilde(X[..., 1:, :] - X[..., :-1, :], lam, inhibit if vinhibit else 0).sum(axis=(-2, -1))
    return E


def brute_force(C: np.ndarray, lam: int, inhibit: int, vinhibit: int = 1):
    """Exhaustive minimum.  Returns (E*, X_min, n_minimisers)."""
    C = np.asarray(C, dtype=np.int64)
    h, ng, D = C.shape
    n = h * ng
    assert D ** n <= 2_000_000, "too many labelings"
    allX = np.array(list(itertools.product(range(D), repeat=n)), dtype=np.int64).reshape(-1, h, ng)
    E = energy_np(C, allX, lam, inhibit, vinhibit)
    Emin = int(E.min())
    mins = allX[E == Emin]
    return Emin, mins.min(axis=0).astype(np.int32), int(mins.shape[0])


def brute_force_band(C: np.ndarray, lam: int, inhibit: int, vinhibit: int, lo: np.ndarray,
                     hi: np.ndarray):
    """Exhaustive minimum over labelings with lo <= X <= hi.  Returns
    (E*, X_min, n_minimisers) of the restricted problem."""
    C = np.asarray(C, dtype=np.int64)
    h, ng, D = C.shape
    ranges = [range(int(a), int(b) + 1) for a, b in zip(np.ravel(lo), np.ravel(hi))]
    count = int(np.prod([len(r) for r in ranges]))
    assert count <= 2_000_000, "too many labelings"
    allX = np.array(list(itertools.product(*ranges)), dtype=np.int64).reshape(-1, h, ng)
    E = energy_np(C, allX, lam, inhibit, vinhibit)
    Emin = int(E.min())
    mins = allX[E == Emin]
    return Emin, mins.min(axis=0).astype(np.int32), int(mins.shape[0])


def viterbi_row(C_row: np.ndarray, lam: int, inhibit: int):
    """Exact min over one row of sites C_row[n, D].  Returns (E*, X_min)."""
    C = np.asarray(C_row, dtype=np.int64)
    n, D = C.shape
    l = np.arange(D)
    P = htilde(l[:, None] - l[None, :], lam, inhibit)            # P[a, b] = h~(a - b)
    F = np.zeros((n, D), dtype=np.int64)                          # best prefix ending at label
    F[0] = C[0]
    for i in range(1, n):
        F[i] = C[i] + (F[i - 1][:, None] + P).min(axis=0)
    B = np.zeros((n, D), dtype=np.int64)                          # best suffix after label
    for i in range(n - 2, -1, -1):
        B[i] = (P + (C[i + 1] + B[i + 1])[None, :]).min(axis=1)
    Estar = int(F[-1].min())
    M = F + B                                                     # best total with X_i = l
    X = np.array([int(np.flatnonzero(M[i] == Estar)[0]) for i in range(n)], dtype=np.int32)
    return Estar, X

"""CPU oracle for the gaze-line / depth-number stereo min-cut (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_1803_01516_gb300``: the C part (``gazecut_oracle.c``) and
the numpy part (``small.py``) are written from the paper's definitions alone.

Functions (citations are to the paper):

* ``cost_volume``   data term g_v at every cross point, §4.3 / §3 (grayscale
                    absolute difference, truncated)
* ``cost_volume_rgb`` the paper's colour form of g_v, §4.3: the sum over R, G, B
                    of the absolute differences (0..765), optionally truncated
* ``solve``         exact min of E(X) (§2) by max-flow on the chain graph of
                    §3 / Fig. 4, with Boykov-Kolmogorov (§4.4) or Dinic;
                    returns flow, canonical labels X_min (smallest minimiser,
                    from S_min), the cut capacity of S_min and X_max
* ``energy``        E(X) = Σ g_v(X_v) + Σ h~(X_u - X_v), §2 and §3
* ``solve_band``    exact min of E(X) under per-site bounds lo <= X <= hi
                    (the second cut of the level-1 approximation, §4.5)
* ``small.brute_force`` / ``small.viterbi_row``  enumeration and the textbook
                    chain DP that pin ``solve`` (see ``small.py``)
* ``level1.level1`` the level-1 hierarchical approximation of §4.5 (delegate
                    points, first cut, thin skin, second cut; module ``level1``)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gazecut_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle in place (plain gcc, no GPU code)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-Wall", "-shared",
                               "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        lib.or_cost_volume.argtypes = [P, P, I, I, I, I, I, P]
        lib.or_cost_volume.restype = I
        lib.or_cost_volume_rgb.argtypes = [P, P, I, I, I, I, I, P]
        lib.or_cost_volume_rgb.restype = I
        lib.or_energy.argtypes = [P, P, I, I, I, I, I, I]
        lib.or_energy.restype = ctypes.c_int64
        lib.or_solve.argtypes = [P, I, I, I, I, I, I, I, P, P, P, P]
        lib.or_solve.restype = I
        lib.or_solve_band.argtypes = [P, I, I, I, I, I, I, P, P, I, P, P]
        lib.or_solve_band.restype = I
        lib.or_graph_size.argtypes = [I, I, I, I, P, P]
        lib.or_graph_size.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def cost_volume(L: np.ndarray, R: np.ndarray, D: int, dis0: int, tau: int) -> np.ndarray:
    """C[y, W, S] = min(|L[y, W+dis0-S] - R[y, W+S]|, tau), int32 [h, n_g, D]."""
    lib = _load()
    L = np.ascontiguousarray(L, dtype=np.uint8)
    R = np.ascontiguousarray(R, dtype=np.uint8)
    h, w = L.shape
    ng = w - dis0
    C = np.zeros((h, max(ng, 0), D), dtype=np.int32)
    rc = lib.or_cost_volume(_ptr(L), _ptr(R), w, h, D, dis0, tau, _ptr(C))
    if rc:
        raise ValueError(f"or_cost_volume: bad sizes (rc={rc})")
    return C


def cost_volume_rgb(L: np.ndarray, R: np.ndarray, D: int, dis0: int, tau: int = 765) -> np.ndarray:
    """C[y, W, S] = min(sum_c |L[y, W+dis0-S, c] - R[y, W+S, c]|, tau), int32 [h, n_g, D];
    L, R uint8 [h, w, 3]."""
    lib = _load()
    L = np.ascontiguousarray(L, dtype=np.uint8)
    R = np.ascontiguousarray(R, dtype=np.uint8)
    assert L.ndim == 3 and L.shape[2] == 3 and R.shape == L.shape
    h, w, _ = L.shape
    ng = w - dis0
    C = np.zeros((h, max(ng, 0), D), dtype=np.int32)
    rc = lib.or_cost_volume_rgb(_ptr(L), _ptr(R), w, h, D, dis0, tau, _ptr(C))
    if rc:
        raise ValueError(f"or_cost_volume_rgb: bad sizes (rc={rc})")
    return C


def energy(C: np.ndarray, X: np.ndarray, lam: int, inhibit: int, vinhibit: int = 1) -> int:
    lib = _load()
    C = np.ascontiguousarray(C, dtype=np.int32)
    X = np.ascontiguousarray(X, dtype=np.int32)
    h, ng, D = C.shape
    assert X.shape == (h, ng)
    assert X.min() >= 0 and X.max() < D
    return int(lib.or_energy(_ptr(C), _ptr(X), ng, h, D, lam, inhibit, vinhibit))


def solve(C: np.ndarray, lam: int, inhibit: int, vinhibit: int = 1, method: str = "bk"):
    """Exact minimiser of E(X).  Returns dict(flow, labels, cut, labels_max)."""
    lib = _load()
    C = np.ascontiguousarray(C, dtype=np.int32)
    h, ng, D = C.shape
    X = np.zeros((h, ng), dtype=np.int32)
    Xmax = np.zeros((h, ng), dtype=np.int32)
    flow = np.zeros(1, dtype=np.int64)
    cut = np.zeros(1, dtype=np.int64)
    rc = lib.or_solve(_ptr(C), ng, h, D, lam, inhibit, vinhibit, 0 if method == "bk" else 1,
                      _ptr(flow), _ptr(X), _ptr(cut), _ptr(Xmax))
    if rc:
        raise RuntimeError(f"or_solve failed (rc={rc})")
    return {"flow": int(flow[0]), "labels": X, "cut": int(cut[0]), "labels_max": Xmax}


def solve_band(C: np.ndarray, lam: int, inhibit: int, vinhibit: int, lo: np.ndarray,
               hi: np.ndarray, method: str = "bk"):
    """Exact minimiser of E(X) subject to lo <= X <= hi (int32 [h, n_g] each).
    Returns dict(flow, labels): the canonical smallest minimiser of the
    restricted problem and its energy (= the flow of the pinned graph)."""
    lib = _load()
    C = np.ascontiguousarray(C, dtype=np.int32)
    h, ng, D = C.shape
    lo = np.ascontiguousarray(lo, dtype=np.int32)
    hi = np.ascontiguousarray(hi, dtype=np.int32)
    assert lo.shape == (h, ng) and hi.shape == (h, ng)
    X = np.zeros((h, ng), dtype=np.int32)
    flow = np.zeros(1, dtype=np.int64)
    rc = lib.or_solve_band(_ptr(C), ng, h, D, lam, inhibit, vinhibit, _ptr(lo), _ptr(hi),
                           0 if method == "bk" else 1, _ptr(flow), _ptr(X))
    if rc:
        raise RuntimeError(f"or_solve_band failed (rc={rc})")
    return {"flow": int(flow[0]), "labels": X}


def graph_size(ng: int, h: int, D: int, vinhibit: int = 1):
    lib = _load()
    n = ctypes.c_int64()
    m = ctypes.c_int64()
    lib.or_graph_size(ng, h, D, vinhibit, ctypes.byref(n), ctypes.byref(m))
    return n.value, m.value

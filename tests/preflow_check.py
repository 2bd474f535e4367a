"""Certificate check of a solved state at any size (test infrastructure).

If the solver's final state is a valid preflow of the chain graph whose value
is F (the sink capacity it used), then F <= max-flow = min E <= E(X) for any
labeling X.  So a state that is a valid preflow, plus labels whose energy
(computed independently by the oracle) equals F, proves both optimal -- at
sizes the oracle cannot solve.

The state layout is the library's: a 256-byte header (int32 at byte 36 = 1
when the state is the label-reversed problem), then nine int32 arrays
(rc, rr, rd, ri0, ri1, ri2, ri3, ex, ht), each over the padded node grid
[h][K][P] (K = D-1, P = n_g rounded up to 32) and padded to 64 entries.
Flows are read back from residuals: data arc n_j -> n_(j+1) carries
C(j+1) - rc, penalty arcs carry lambda - rr (rd), inhibit arcs h2 - ri.
"""
from __future__ import annotations

import numpy as np


def state_arrays(graph_bytes: np.ndarray, h: int, ng: int, D: int):
    K = D - 1
    P = (ng + 31) // 32 * 32
    N = h * K * P
    stride = (N + 63) // 64 * 64
    words = graph_bytes[256:256 + 9 * stride * 4].view(np.int32)
    names = ["rc", "rr", "rd", "ri0", "ri1", "ri2", "ri3", "ex", "ht"]
    out = {}
    for i, n in enumerate(names):
        out[n] = words[i * stride:i * stride + N].reshape(h, K, P)[:, :, :ng].astype(np.int64)
    return out


def check_preflow(graph_bytes: np.ndarray, C: np.ndarray, lam: int, inhibit: int,
                  vinhibit: int) -> dict:
    """Capacity bounds and flow conservation at every node.  Returns the flow
    value (sink capacity used); raises AssertionError on a violation."""
    h, ng, D = C.shape
    K = D - 1
    s = state_arrays(graph_bytes, h, ng, D)
    # a state built for the label-reversed problem uses C'(l) = C(D-1-l)
    rev = int(graph_bytes[36:40].view(np.int32)[0])
    if rev:
        C = C[:, :, ::-1]
    Ct = np.transpose(C, (0, 2, 1)).astype(np.int64)          # [h][D][ng]
    h2h, h2v = inhibit, (inhibit if vinhibit else 0)
    rc, rr, rd, ex = s["rc"], s["rr"], s["rd"], s["ex"]
    ri = [s["ri0"], s["ri1"], s["ri2"], s["ri3"]]
    # capacity bounds
    assert (rc[:, :K - 1, :] >= 0).all(), "negative data-arc residual"
    assert (rr >= 0).all() and (rr <= 2 * lam).all(), "penalty residual out of range"
    assert (rd >= 0).all() and (rd <= 2 * lam).all(), "penalty residual out of range"
    for d in range(4):
        cap = h2h if d < 2 else h2v
        assert (ri[d] >= 0).all() and (ri[d] <= cap).all(), "inhibit residual out of range"
    # flows on the arcs
    fc = np.zeros((h, K, ng), np.int64)                        # n_j -> n_(j+1)
    fc[:, :K - 1, :] = Ct[:, 1:K, :] - rc[:, :K - 1, :]
    fr = lam - rr                                              # W -> W+1
    fr[:, :, ng - 1] = 0
    fdn = lam - rd                                             # y -> y+1
    fdn[h - 1] = 0
    fi = []
    for d in range(4):                                         # u_j -> nbr(d)_(j-1)
        f = (h2h if d < 2 else h2v) - ri[d]
        f[:, 0, :] = 0
        if d == 0:
            f[:, :, 0] = 0
        if d == 1:
            f[:, :, ng - 1] = 0
        if d == 2:
            f[0] = 0
        if d == 3:
            f[h - 1] = 0
        fi.append(f)
    net = np.zeros((h, K, ng), np.int64)
    net[:, 0, :] += Ct[:, 0, :]                                # supply C(0)
    net[:, K - 1, :] -= Ct[:, K, :]                            # demand C(D-1)
    net[:, 1:, :] += fc[:, :K - 1, :]                          # in from j-1
    net -= fc                                                  # out to j+1
    net -= fr
    net[:, :, 1:] += fr[:, :, :-1]
    net -= fdn
    net[1:] += fdn[:-1]
    for d in range(4):
        net -= fi[d]
    # in along inhibit arcs from the neighbours' layer j+1
    net[:, :K - 1, 1:] += fi[1][:, 1:, :-1]      # from W-1 (its arc to W+1 side)
    net[:, :K - 1, :-1] += fi[0][:, 1:, 1:]      # from W+1
    net[1:, :K - 1, :] += fi[3][:-1, 1:, :]      # from y-1 (its arc downwards)
    net[:-1, :K - 1, :] += fi[2][1:, 1:, :]      # from y+1
    bad = np.argwhere(net != ex)
    assert bad.size == 0, f"conservation fails at {bad[:5].tolist()}"
    # preflow: no node but a sink node below zero, sink nodes within their capacity
    assert (ex[:, :K - 1, :] >= 0).all() if K > 1 else True, "negative excess off the sink layer"
    assert (ex[:, K - 1, :] >= -Ct[:, K, :]).all(), "sink capacity exceeded"
    used = int(Ct[:, K, :].sum() + np.minimum(ex[:, K - 1, :], 0).sum())
    return {"flow": used, "nodes": int(h * K * ng)}


_SMIN = None


def _smin_lib():
    """Compile ``state_smin.c`` (plain gcc) next to this file, once."""
    global _SMIN
    if _SMIN is None:
        import ctypes
        import os
        import subprocess
        here = os.path.dirname(os.path.abspath(__file__))
        src = os.path.join(here, "state_smin.c")
        out_dir = os.path.join(here, "_build")
        os.makedirs(out_dir, exist_ok=True)
        lib = os.path.join(out_dir, "libstate_smin.so")
        if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            tmp = lib + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp,
                                   src])
            os.replace(tmp, lib)
        L = ctypes.CDLL(lib)
        L.smin_labels.argtypes = [ctypes.c_void_p] + [ctypes.c_int64] * 6 + [ctypes.c_int,
                                                                            ctypes.c_void_p]
        L.smin_labels.restype = ctypes.c_int
        _SMIN = L
    return _SMIN


def smin_labels(graph_bytes: np.ndarray, h: int, ng: int, D: int, lam: int, inhibit: int,
                vinhibit: int) -> np.ndarray:
    """Canonical (smallest-minimiser) labels read from a solved state: S_min by
    reachability from the remaining excess, or for a label-reversed state the
    mirrored largest minimiser from reachability to the remaining sink
    capacity.  Raises AssertionError when a chain's side is not a prefix."""
    import ctypes
    K = D - 1
    P = (ng + 31) // 32 * 32
    N = h * K * P
    stride = (N + 63) // 64 * 64
    words = np.ascontiguousarray(graph_bytes[256:256 + 9 * stride * 4]).view(np.int32)
    rev = int(graph_bytes[36:40].view(np.int32)[0])
    ptrs = (ctypes.c_void_p * 9)(*[words[i * stride:].ctypes.data for i in range(9)])
    X = np.zeros((h, ng), dtype=np.int32)
    rc = _smin_lib().smin_labels(ptrs, h, ng, D, lam, inhibit, inhibit if vinhibit else 0, rev,
                                 X.ctypes.data)
    assert rc == 0, f"smin_labels failed (rc={rc})"
    return X

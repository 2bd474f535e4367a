"""The CPU reader of canonical labels from a solved state (tests/state_smin.c),
pinned without a GPU.

With no interaction terms (lambda = inhibit = 0) every chain is its own
problem, and the chain-local preflow -- node n_j holding F_j - F_(j+1),
F_j = min C(0..j), the data arcs carrying the prefix minima -- is already a
maximum preflow.  The smallest minimiser is then each site's first argmin, a
closed form.  The state is written here in the library's layout (a 256-byte
header, the label-reversed flag at byte 36, nine int32 arrays over [h][K][P])."""
import numpy as np

from preflow_check import smin_labels


def _chain_state(C: np.ndarray, rev: int) -> np.ndarray:
    h, ng, D = C.shape
    Cs = C[:, :, ::-1] if rev else C                 # costs of the direction solved
    K = D - 1
    P = (ng + 31) // 32 * 32
    N = h * K * P
    stride = (N + 63) // 64 * 64
    g = np.zeros(256 + 9 * stride * 4, dtype=np.uint8)
    g[36:40] = np.array([rev], dtype=np.int32).view(np.uint8)
    words = g[256:].view(np.int32)
    arr = {n: words[i * stride:i * stride + N].reshape(h, K, P)
           for i, n in enumerate(["rc", "rr", "rd", "ri0", "ri1", "ri2", "ri3", "ex", "ht"])}
    F = np.minimum.accumulate(Cs.astype(np.int64), axis=2)    # F_j = min C(0..j)
    for j in range(K):
        if j < K - 1:
            arr["ex"][:, j, :ng] = F[:, :, j] - F[:, :, j + 1]
            arr["rc"][:, j, :ng] = Cs[:, :, j + 1] - F[:, :, j + 1]
        else:
            arr["ex"][:, j, :ng] = F[:, :, j] - Cs[:, :, D - 1]
    return g


def test_reader_gives_first_argmin_without_interaction():
    rng = np.random.default_rng(5)
    for shape in [(3, 4, 4), (5, 33, 6), (2, 7, 2), (4, 40, 17)]:
        C = rng.integers(0, 6, size=shape).astype(np.int32)   # many ties
        h, ng, D = shape
        first = np.argmin(C, axis=2).astype(np.int32)
        for rev in (0, 1):
            X = smin_labels(_chain_state(C, rev), h, ng, D, 0, 0, 1)
            assert np.array_equal(X, first), (shape, rev)


"""Full-size parity by certificate: a valid preflow whose value equals the
oracle's energy of the GPU labels proves both optimal, at sizes (1920x1080
with 128 depth numbers, 228.5 M graph nodes) the oracle cannot solve; the
canonical labels (smallest minimiser) are then recomputed on the CPU from the
solved state by reachability and compared element by element."""
import numpy as np
import pytest

import oracle
from paper_1803_01516_gb300 import synth
from preflow_check import check_preflow, smin_labels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_01516_gb300 import build
    build.build()
    from paper_1803_01516_gb300 import gazecut
    return gazecut


def _solve(gc, wl, vi=1, direction=0):
    L, R, _ = synth.make_pair(wl, 0)
    p = gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit,
                  vertical_inhibit=vi, direction=direction)
    o = gc.SolveOpts()
    buf = gc.Buffers(p, o)
    gc.solve_pair(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), p, o, buf)
    torch.cuda.synchronize()
    C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    return buf, C


def test_certificate_checker_on_the_main_pair(gc):
    """The checker accepts the solved state of the 384x288 pair (whose flow the
    oracle also computes), and rejects a copy with one residual changed."""
    wl = synth.MAIN
    buf, C = _solve(gc, wl)
    ref = oracle.solve(C, wl.lam, wl.inhibit, 1)
    g = buf.graph.cpu().numpy()
    r = check_preflow(g, C, wl.lam, wl.inhibit, 1)
    assert r["flow"] == ref["flow"] == int(buf.flow.item())
    bad = g.copy()
    words = bad[256:].view(np.int32)
    K, P = wl.D - 1, (C.shape[1] + 31) // 32 * 32
    stride = (wl.h * K * P + 63) // 64 * 64
    words[1 * stride + (5 * K + 3) * P + 7] -= 1          # one penalty residual (rr)
    with pytest.raises(AssertionError):
        check_preflow(bad, C, wl.lam, wl.inhibit, 1)


@pytest.mark.parametrize("direction", [1, 2])
def test_state_smin_reader_on_the_main_pair(gc, direction):
    """The CPU reader of canonical labels from a solved state, pinned where the
    oracle solves: on the 384x288 pair, solved as given (forward reachability
    from excess) and label-reversed (mirrored reachability to sink capacity),
    it returns the oracle's smallest minimiser."""
    wl = synth.MAIN
    buf, C = _solve(gc, wl, direction=direction)
    ref = oracle.solve(C, wl.lam, wl.inhibit, 1)
    g = buf.graph.cpu().numpy()
    assert int(g[36:40].view(np.int32)[0]) == (direction == 2)
    X = smin_labels(g, wl.h, C.shape[1], wl.D, wl.lam, wl.inhibit, 1)
    assert np.array_equal(X, ref["labels"])
    assert np.array_equal(buf.labels.cpu().numpy(), ref["labels"])


def test_large_configuration_certified(gc):
    """1920x1080, 128 depth numbers, 12 slanted planes: cost volume bit-exact,
    valid preflow at every node, flow == E(labels) (energy by the oracle)."""
    wl = synth.LARGE
    buf, C = _solve(gc, wl)
    assert int(buf.status.item()) == gc.GS_OK
    cost = buf.cost.cpu().numpy().reshape(C.shape)
    assert np.array_equal(cost, C)
    X = buf.labels.cpu().numpy()
    E = oracle.energy(C, X, wl.lam, wl.inhibit, 1)
    g = buf.graph.cpu().numpy()
    r = check_preflow(g, C, wl.lam, wl.inhibit, 1)
    assert E == int(buf.flow.item()) == r["flow"]
    # the state is a maximum preflow: its reachability sets give the canonical
    # smallest minimiser, which the GPU labels must equal element by element
    Xmin = smin_labels(g, wl.h, C.shape[1], wl.D, wl.lam, wl.inhibit, 1)
    assert np.array_equal(Xmin, X)

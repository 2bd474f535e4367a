"""Full-size parity by certificate: a valid preflow whose value equals the
oracle's energy of the GPU labels proves both optimal, at sizes (1920x1080
with 128 depth numbers, 228.5 M graph nodes) the oracle cannot solve."""
import numpy as np
import pytest

import oracle
from paper_1803_01516_gb300 import synth
from preflow_check import check_preflow

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


def _solve(gc, wl, vi=1):
    L, R, _ = synth.make_pair(wl, 0)
    p = gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit,
                  vertical_inhibit=vi)
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
    r = check_preflow(buf.graph.cpu().numpy(), C, wl.lam, wl.inhibit, 1)
    assert E == int(buf.flow.item()) == r["flow"]

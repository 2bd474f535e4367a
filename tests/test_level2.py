"""Level-2 approximation (§4.5) on the GPU vs the oracle (oracle/level2.py),
element by element: start labels, block descent on random bounds and labels,
and the whole pipeline (delegate cut, skin, start, two passes of block cuts) on
the tiny, a ragged and the main workload for block sizes 1, 2 and 3."""
import numpy as np
import pytest

import oracle
from oracle import level1 as l1
from oracle import level2 as l2
from paper_1803_01516_gb300 import synth

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


def _params(gc, C, lam, inhibit, vi=1):
    h, ng, D = C.shape
    return gc.Params(w=ng + 2 * (D - 1), h=h, D=D, tau=0, lam=lam, inhibit=inhibit,
                     vertical_inhibit=vi)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("b", [1, 2, 3])
@pytest.mark.parametrize("vi", [1, 0])
@pytest.mark.parametrize("seed", range(3))
def test_block_descent_matches_oracle(gc, b, vi, seed):
    """Random costs, delegate labels and start labels inside the skin; 1 and 2
    passes of block cuts, ragged grid edges (partial blocks)."""
    rng = np.random.default_rng(100 * b + 10 * vi + seed)
    h, ng, D = int(rng.integers(5, 17)), int(rng.integers(5, 23)), int(rng.integers(b + 2, 14))
    C = rng.integers(0, 40, size=(h, ng, D)).astype(np.int32)
    lam, inh = int(rng.integers(1, 9)), int(rng.integers(0, 60))
    hc, ngc, Dc = l1.coarse_shape(h, ng, D, b)
    Xc = rng.integers(0, Dc, size=(hc, ngc)).astype(np.int32)
    lo, hi = l1.skin_bounds(Xc, b, h, ng, D)
    X0 = (lo + rng.integers(0, 1 << 20, size=(h, ng)) % (hi - lo + 1)).astype(np.int32)
    p = _params(gc, C, lam, inh, vi)
    for passes in (1, 2):
        want = l2.block_descent(C, X0, lam, inh, vi, b, lo, hi, passes)
        X = _dev(X0)
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        gc.gs_block_descent(_dev(C).reshape(-1), p, b, _dev(lo), _dev(hi), X, passes, st)
        assert int(st.item()) == gc.GS_OK
        assert np.array_equal(X.cpu().numpy(), want), passes


def test_start_labels_match_oracle(gc):
    rng = np.random.default_rng(3)
    C = rng.integers(0, 9, size=(11, 13, 10)).astype(np.int32)    # many ties
    for b in (1, 2, 3):
        hc, ngc, Dc = l1.coarse_shape(11, 13, 10, b)
        Xc = rng.integers(0, Dc, size=(hc, ngc)).astype(np.int32)
        p = _params(gc, C, 2, 5)
        X = torch.empty((11, 13), dtype=torch.int32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        gc.gs_level2_start(_dev(C).reshape(-1), p, b, _dev(Xc), X, st)
        assert int(st.item()) == gc.GS_OK
        assert np.array_equal(X.cpu().numpy(), l2.start_labels(C, Xc, b))


def test_block_range_wider_than_the_skin_is_flagged(gc):
    """A block whose label range exceeds min(3b, D) labels cannot be cut by the
    row-state DP: the call flags GS_ERR_INVAL and leaves the block as it is."""
    C = np.zeros((6, 6, 16), np.int32)
    p = _params(gc, C, 1, 1)
    lo = np.zeros((6, 6), np.int32)
    hi = np.full((6, 6), 15, np.int32)
    X = torch.full((6, 6), 4, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    gc.gs_block_descent(_dev(C).reshape(-1), p, 3, _dev(lo), _dev(hi), X, 1, st)
    assert int(st.item()) == gc.GS_ERR_INVAL
    assert (X.cpu().numpy() == 4).all()


def _workload_costs(wl, i=0):
    L, R, _ = synth.make_pair(wl, i)
    return oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)


RAGGED = synth.Workload("ragged-101x37x11", 101, 37, 11, tau=25, lam=6, sigma=2.0,
                        scene="layers", n_layers=3, n_slanted=1, max_disp=20, seed_base=9)


@pytest.mark.parametrize("b", [1, 2, 3])
@pytest.mark.parametrize("which", ["tiny", "ragged", "main"])
def test_level2_pipeline_matches_oracle(gc, b, which):
    wl = {"tiny": synth.TINY, "ragged": RAGGED, "main": synth.MAIN}[which]
    C = _workload_costs(wl)
    p = gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit)
    X, Xc, st = gc.solve_level2(_dev(C), p, b, passes=2)
    torch.cuda.synchronize()
    assert int(st.item()) == gc.GS_OK
    want = l2.level2(C, wl.lam, wl.inhibit, 1, b, passes=2)
    assert np.array_equal(Xc.cpu().numpy(), want["coarse_labels"])
    assert np.array_equal(X.cpu().numpy(), want["labels"])
    e = torch.zeros(1, dtype=torch.int64, device="cuda")
    gc.gs_energy(_dev(C).reshape(-1), X, p, e)
    assert int(e.item()) == want["energy"]

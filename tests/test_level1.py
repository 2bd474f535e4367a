"""Level-1 approximation of §4.5 on the GPU against the oracle: delegate costs
and skin bounds bit-exact, the restricted second cut bit-exact (labels and
energy) on random bounds and on the skins of real workloads, and the whole
two-cut pipeline bit-exact for block sizes 1, 2 and 3."""
import numpy as np
import pytest

import oracle
from oracle import level1 as l1
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


def _workload_costs(wl, i=0):
    L, R, _ = synth.make_pair(wl, i)
    return oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)


RAGGED = synth.Workload("ragged-77x53x11", 77 + 20, 53, 11, tau=25, lam=6, sigma=2.0,
                        scene="layers", n_layers=4, n_slanted=1, max_disp=20, seed_base=5)


@pytest.mark.parametrize("b", [2, 3, 4])
@pytest.mark.parametrize("which", ["tiny", "ragged", "main"])
def test_delegate_cost_and_skin_bit_exact(gc, b, which):
    wl = {"tiny": synth.TINY, "ragged": RAGGED, "main": synth.MAIN}[which]
    C = _workload_costs(wl)
    p = _params(gc, C, wl.lam, wl.inhibit)
    pc = gc.gs_delegate_params(p, b)
    ref = l1.coarse_costs(C, b)
    assert ref.shape == (pc.h, pc.ng, pc.D)
    coarse = torch.empty(ref.size, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    gc.gs_delegate_cost(torch.from_numpy(C).cuda().reshape(-1), p, b, coarse, st)
    assert int(st.item()) == gc.GS_OK
    assert np.array_equal(coarse.cpu().numpy().reshape(ref.shape), ref)
    Xc = np.random.default_rng(b).integers(0, pc.D, size=(pc.h, pc.ng)).astype(np.int32)
    lo = torch.empty((p.h, p.ng), dtype=torch.int32, device="cuda")
    hi = torch.empty_like(lo)
    gc.gs_skin_bounds(torch.from_numpy(Xc).cuda(), p, b, lo, hi, st)
    rlo, rhi = l1.skin_bounds(Xc, b, p.h, p.ng, p.D)
    assert int(st.item()) == gc.GS_OK
    assert np.array_equal(lo.cpu().numpy(), rlo) and np.array_equal(hi.cpu().numpy(), rhi)


def _skin_solve(gc, C, p, lo, hi, o):
    buf = gc.Buffers(p, o)
    c = torch.from_numpy(np.ascontiguousarray(C)).cuda().reshape(-1)
    gc.gs_build_graph_skin(c, p, torch.from_numpy(lo).cuda(), torch.from_numpy(hi).cuda(),
                           buf.graph, buf.status)
    gc.gs_maxflow_solve(buf.graph, p, o, buf.work, buf.status)
    gc.gs_extract_labels(buf.graph, p, o, buf.work, buf.labels, buf.flow, buf.status)
    torch.cuda.synchronize()
    return buf.labels.cpu().numpy(), int(buf.status.item())


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_skin_cut_matches_oracle_on_random_bounds(gc, engine, seed):
    rng = np.random.default_rng(seed)
    C = rng.integers(0, 30, size=(13, 21, 9)).astype(np.int32)
    lo = rng.integers(0, 9, size=(13, 21)).astype(np.int32)
    hi = np.minimum(lo + rng.integers(0, 5, size=(13, 21)), 8).astype(np.int32)
    lam, inh = (4, 60) if seed % 2 else (7, 1023)
    p = _params(gc, C, lam, inh)
    ref = oracle.solve_band(C, lam, inh, 1, lo, hi)
    X, status = _skin_solve(gc, C, p, lo, hi, gc.SolveOpts(engine=engine))
    assert status == gc.GS_OK
    assert np.array_equal(X, ref["labels"])
    assert oracle.energy(C, X, lam, inh, 1) == ref["flow"]


def test_skin_cut_with_full_bounds_is_the_exact_cut(gc):
    wl = synth.TINY
    C = _workload_costs(wl, 1)
    p = _params(gc, C, wl.lam, wl.inhibit)
    lo = np.zeros((p.h, p.ng), np.int32)
    hi = np.full((p.h, p.ng), p.D - 1, np.int32)
    X, status = _skin_solve(gc, C, p, lo, hi, gc.SolveOpts())
    ref = oracle.solve(C, wl.lam, wl.inhibit, 1)
    assert status == gc.GS_OK and np.array_equal(X, ref["labels"])


def test_skin_bounds_out_of_order_flagged(gc):
    C = np.zeros((4, 8, 4), np.int32)
    p = _params(gc, C, 1, 1)
    lo = np.full((4, 8), 2, np.int32)
    hi = np.full((4, 8), 1, np.int32)
    buf = gc.Buffers(p, gc.SolveOpts())
    gc.gs_build_graph_skin(torch.from_numpy(C).cuda().reshape(-1), p, torch.from_numpy(lo).cuda(),
                           torch.from_numpy(hi).cuda(), buf.graph, buf.status)
    assert int(buf.status.item()) == gc.GS_ERR_INVAL


@pytest.mark.parametrize("b", [1, 2, 3])
@pytest.mark.parametrize("which", ["tiny", "ragged", "main"])
def test_level1_pipeline_matches_oracle(gc, b, which):
    wl = {"tiny": synth.TINY, "ragged": RAGGED, "main": synth.MAIN}[which]
    C = _workload_costs(wl, 2)
    p = _params(gc, C, wl.lam, wl.inhibit)
    ref = l1.level1(C, wl.lam, wl.inhibit, 1, b)
    o = gc.SolveOpts()
    X, Xc, st = gc.solve_level1(torch.from_numpy(C).cuda(), p, b, o)
    torch.cuda.synchronize()
    assert int(st.item()) == gc.GS_OK
    assert np.array_equal(Xc.cpu().numpy(), ref["coarse_labels"])
    assert np.array_equal(X.cpu().numpy(), ref["labels"])
    E = torch.zeros(1, dtype=torch.int64, device="cuda")
    gc.gs_energy(torch.from_numpy(C).cuda().reshape(-1), X, p, E)
    assert int(E.item()) == ref["energy"]
    if b == 1:
        assert ref["energy"] == oracle.solve(C, wl.lam, wl.inhibit, 1)["flow"]

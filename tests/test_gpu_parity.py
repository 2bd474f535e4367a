"""GPU path vs the CPU oracle, element by element (bit-exact: everything is integer)."""
import numpy as np
import pytest

import oracle
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


def _params(gc, wl, vi=1):
    return gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit,
                     vertical_inhibit=vi)


def _solve_costs(gc, C, lam, inhibit, vi, opts=None, direction=0):
    h, ng, D = C.shape
    p = gc.Params(w=ng + 2 * (D - 1), h=h, D=D, tau=0, lam=lam, inhibit=inhibit, vertical_inhibit=vi,
                  direction=direction)
    opts = opts or gc.SolveOpts()
    labels, flow, status = gc.solve_costs(torch.from_numpy(np.ascontiguousarray(C)).cuda(), p, opts)
    torch.cuda.synchronize()
    return labels.cpu().numpy(), int(flow.item()), int(status.item()), p


@pytest.mark.parametrize("which", ["tiny", "main"])
def test_cost_volume_bit_exact(gc, which):
    wl = synth.TINY if which == "tiny" else synth.MAIN
    L, R, _ = synth.make_pair(wl, 0)
    p = _params(gc, wl)
    cost = torch.empty(gc.gs_cost_volume_bytes(p) // 4, dtype=torch.int32, device="cuda")
    gc.gs_stereo_cost_volume(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), p, cost)
    ref = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    assert np.array_equal(cost.cpu().numpy().reshape(ref.shape), ref)


def _offset_copy(a: np.ndarray, off: int):
    """A device copy of `a` whose data starts `off` bytes past an allocation's
    start (a view into a larger buffer): not 16-byte aligned when off % 16."""
    flat = torch.zeros(a.size + off, dtype=torch.uint8, device="cuda")
    flat[off:] = torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()
    return flat[off:].view(*a.shape)


@pytest.mark.parametrize("shape,off", [((48, 64), 0), ((33, 101), 0), ((20, 96), 3),
                                       ((288, 384), 0)])
def test_cost_volume_bit_exact_any_row_alignment(gc, shape, off):
    """128-bit row staging (aligned images, pitch a multiple of 16) and the
    byte path (odd pitch 101, or images starting 3 bytes past a boundary)
    give the oracle's cost volume."""
    h, w = shape
    rng = np.random.default_rng(h * w + off)
    L = rng.integers(0, 256, size=shape).astype(np.uint8)
    R = rng.integers(0, 256, size=shape).astype(np.uint8)
    for D in (2, 16, 23):
        if w - 2 * (D - 1) < 1:
            continue
        p = gc.Params(w=w, h=h, D=D, tau=37, lam=1)
        cost = torch.empty(gc.gs_cost_volume_bytes(p) // 4, dtype=torch.int32, device="cuda")
        gc.gs_stereo_cost_volume(_offset_copy(L, off), _offset_copy(R, off), p, cost)
        ref = oracle.cost_volume(L, R, D, 2 * (D - 1), 37)
        assert np.array_equal(cost.cpu().numpy().reshape(ref.shape), ref), D


@pytest.mark.parametrize("shape,off,tau", [((48, 64), 0, 765), ((33, 101), 0, 765),
                                           ((20, 96), 5, 100), ((288, 384), 0, 765)])
def test_rgb_cost_volume_bit_exact(gc, shape, off, tau):
    """Colour data term of §4.3 (sum of |dR|+|dG|+|dB|, 0..765) on interleaved
    RGB rows: aligned (128-bit staging), odd pitch 303 and misaligned images."""
    h, w = shape
    rng = np.random.default_rng(7 * h + w + off)
    L = rng.integers(0, 256, size=(h, w, 3)).astype(np.uint8)
    R = rng.integers(0, 256, size=(h, w, 3)).astype(np.uint8)
    for D in (2, 16, 23):
        if w - 2 * (D - 1) < 1:
            continue
        p = gc.Params(w=w, h=h, D=D, tau=tau, lam=1)
        cost = torch.empty(gc.gs_cost_volume_bytes(p) // 4, dtype=torch.int32, device="cuda")
        gc.gs_stereo_cost_volume_rgb(_offset_copy(L, off), _offset_copy(R, off), p, cost)
        ref = oracle.cost_volume_rgb(L, R, D, 2 * (D - 1), tau)
        assert np.array_equal(cost.cpu().numpy().reshape(ref.shape), ref), D


@pytest.mark.parametrize("which", ["tiny", "main"])
def test_rgb_pair_exact(gc, which):
    """The colour pipeline end to end: RGB SAD data term (no truncation, the
    paper's form), graph, exact solve, labels -- flow and labels equal the
    oracle's on the colour version of the workload (lambda = 14, the paper's
    best penalty for its colour data term)."""
    wl = synth.TINY if which == "tiny" else synth.MAIN
    L, R, _ = synth.make_pair_rgb(wl, 0)
    p = gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=765, lam=14, inhibit=1023)
    o = gc.SolveOpts()
    buf = gc.Buffers(p, o)
    gc.gs_stereo_cost_volume_rgb(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), p,
                                 buf.cost)
    gc.solve_costs(buf.cost, p, o, buf)
    C = oracle.cost_volume_rgb(L, R, wl.D, 2 * (wl.D - 1), 765)
    ref = oracle.solve(C, 14, 1023, 1)
    assert int(buf.status.item()) == gc.GS_OK
    assert int(buf.flow.item()) == ref["flow"]
    assert np.array_equal(buf.labels.cpu().numpy(), ref["labels"])


ENGINES = [0, 1]   # tiled persistent, simple


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("vi", [1, 0])
def test_tiny_pair_exact(gc, vi, engine):
    wl = synth.TINY
    for idx in range(3):
        L, R, _ = synth.make_pair(wl, idx)
        p = _params(gc, wl, vi)
        o = gc.SolveOpts(engine=engine)
        labels, flow, status = gc.solve_pair(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), p, o)
        torch.cuda.synchronize()
        C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
        ref = oracle.solve(C, wl.lam, wl.inhibit, vi)
        assert int(status.item()) == gc.GS_OK
        assert int(flow.item()) == ref["flow"]
        assert np.array_equal(labels.cpu().numpy(), ref["labels"])


@pytest.mark.parametrize("shape,lam,inh,vi,hi", [
    ((37, 45, 5), 3, 50, 1, 20),      # ragged in both site dimensions
    ((19, 70, 9), 2, 1023, 0, 30),    # W spans 3 warps with a ragged tail
    ((1, 100, 16), 4, 1023, 1, 30),   # one row (chain MRF)
    ((50, 1, 6), 3, 1023, 1, 30),     # one column
    ((13, 33, 2), 5, 1023, 1, 30),    # D = 2: one node per site, base flow
    ((8, 40, 3), 0, 0, 1, 30),        # no interaction: per-site argmin
    ((21, 64, 7), 1, 3, 1, 40),       # weak inhibit: many jumps of more than 1
    ((9, 31, 12), 100, 1023, 1, 30),  # strong penalty: nearly constant labeling
    ((7, 45, 64), 3, 1023, 1, 30),    # long chains (D = 64)
    ((3, 21, 128), 2, 1023, 0, 40),   # D = 128, narrow tiles
    ((2, 9, 200), 2, 1023, 1, 40),    # D = 200: depth layers past 7 bits of the node word
    ((11, 97, 16), 10, 1023, 1, 30),  # several tiles in both directions
])
@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("direction", [1, 2])
def test_random_costs_exact(gc, shape, lam, inh, vi, hi, engine, direction):
    """Both solve directions (as given, label-reversed) give the canonical cut."""
    rng = np.random.default_rng(sum(shape) * 7 + lam)
    C = rng.integers(0, hi + 1, size=shape).astype(np.int32)
    X, flow, status, _ = _solve_costs(gc, C, lam, inh, vi, gc.SolveOpts(engine=engine), direction)
    ref = oracle.solve(C, lam, inh, vi)
    assert status == gc.GS_OK
    assert flow == ref["flow"]
    assert np.array_equal(X, ref["labels"])


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_ties_canonical_labels(gc, direction):
    """Constant costs: every constant labeling is optimal; the canonical answer
    is the smallest one (all zeros), in either solve direction."""
    C = np.full((10, 40, 6), 7, dtype=np.int32)
    X, flow, status, _ = _solve_costs(gc, C, 3, 1023, 1, direction=direction)
    assert status == gc.GS_OK and flow == 7 * 400 and (X == 0).all()
    C = np.random.default_rng(0).integers(0, 3, size=(12, 35, 4)).astype(np.int32)
    X, flow, status, _ = _solve_costs(gc, C, 1, 2, 1, direction=direction)
    ref = oracle.solve(C, 1, 2, 1)
    assert flow == ref["flow"] and np.array_equal(X, ref["labels"])
    assert (ref["labels"] != ref["labels_max"]).any()


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("vi", [1, 0])
def test_main_pair_exact(gc, vi, engine):
    """The 384x288 pair with 16 depth numbers."""
    wl = synth.MAIN
    L, R, _ = synth.make_pair(wl, 0)
    p = _params(gc, wl, vi)
    o = gc.SolveOpts(engine=engine)
    labels, flow, status = gc.solve_pair(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), p, o)
    torch.cuda.synchronize()
    C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    ref = oracle.solve(C, wl.lam, wl.inhibit, vi)
    assert int(status.item()) == gc.GS_OK
    assert int(flow.item()) == ref["flow"]
    assert np.array_equal(labels.cpu().numpy(), ref["labels"])


def test_energy_kernel_matches_oracle(gc):
    rng = np.random.default_rng(4)
    C = rng.integers(0, 30, size=(17, 29, 8)).astype(np.int32)
    X = rng.integers(0, 8, size=(17, 29)).astype(np.int32)
    p = gc.Params(w=29 + 14, h=17, D=8, tau=0, lam=5, inhibit=99, vertical_inhibit=1)
    e = torch.zeros(1, dtype=torch.int64, device="cuda")
    gc.gs_energy(torch.from_numpy(C).cuda().reshape(-1), torch.from_numpy(X).cuda(), p, e)
    assert int(e.item()) == oracle.energy(C, X, 5, 99, 1)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("direction", [1, 2])
def test_fixed_sweeps_gap_is_nonnegative(gc, engine, direction):
    wl = synth.TINY
    L, R, _ = synth.make_pair(wl, 1)
    C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    ref = oracle.solve(C, wl.lam, wl.inhibit, 1)
    for n in (0, 1, 4, 16):
        o = gc.SolveOpts(mode=gc.GS_MODE_FIXED_SWEEPS, fixed_sweeps=n, sweeps_per_relabel=4,
                         engine=engine)
        X, flow, status, _ = _solve_costs(gc, C, wl.lam, wl.inhibit, 1, o, direction)
        assert status == gc.GS_OK
        E = oracle.energy(C, X, wl.lam, wl.inhibit, 1)
        assert flow <= ref["flow"] <= E          # weak duality on both sides


@pytest.mark.parametrize("engine", ENGINES)
def test_timeout_then_resume(gc, engine):
    wl = synth.TINY
    L, R, _ = synth.make_pair(wl, 2)
    C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    ref = oracle.solve(C, wl.lam, wl.inhibit, 1)
    h, ng, D = C.shape
    p = gc.Params(w=ng + 2 * (D - 1), h=h, D=D, tau=0, lam=wl.lam, inhibit=wl.inhibit)
    o = gc.SolveOpts(max_iters=1, sweeps_per_relabel=1, engine=engine)
    buf = gc.Buffers(p, o)
    gc.gs_build_graph(torch.from_numpy(C).cuda().reshape(-1), p, buf.graph, buf.status)
    gc.gs_maxflow_solve(buf.graph, p, o, buf.work, buf.status)
    assert int(buf.status.item()) == gc.GS_ERR_TIMEOUT
    buf.status.zero_()
    o2 = gc.SolveOpts(engine=engine)
    gc.gs_maxflow_solve(buf.graph, p, o2, buf.work, buf.status)
    gc.gs_extract_labels(buf.graph, p, o2, buf.work, buf.labels, buf.flow, buf.status)
    assert int(buf.status.item()) == gc.GS_OK
    assert int(buf.flow.item()) == ref["flow"]
    assert np.array_equal(buf.labels.cpu().numpy(), ref["labels"])


def test_idle_limit_runs_out_then_resume(gc):
    """A caller-set idle limit is a bounded device-side wait that returns: with
    a 1 us limit the blocks of the persistent launch that find no work give up
    at once, the solve ends with GS_ERR_TIMEOUT and the state is still a valid
    preflow; a second call with the default limit resumes it to the oracle's
    exact cut (384x288, 16 depth numbers, hundreds of tiles)."""
    from preflow_check import check_preflow
    wl = synth.MAIN
    L, R, _ = synth.make_pair(wl, 1)
    C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    ref = oracle.solve(C, wl.lam, wl.inhibit, 1)
    p = _params(gc, wl)
    o = gc.SolveOpts(idle_limit_us=1)
    buf = gc.Buffers(p, o)
    gc.gs_build_graph(torch.from_numpy(C).cuda().reshape(-1), p, buf.graph, buf.status)
    gc.gs_maxflow_solve(buf.graph, p, o, buf.work, buf.status)
    assert int(buf.status.item()) == gc.GS_ERR_TIMEOUT
    check_preflow(buf.graph.cpu().numpy(), C, wl.lam, wl.inhibit, 1)
    buf.status.zero_()
    o2 = gc.SolveOpts()
    gc.gs_maxflow_solve(buf.graph, p, o2, buf.work, buf.status)
    gc.gs_extract_labels(buf.graph, p, o2, buf.work, buf.labels, buf.flow, buf.status)
    assert int(buf.status.item()) == gc.GS_OK
    assert int(buf.flow.item()) == ref["flow"]
    assert np.array_equal(buf.labels.cpu().numpy(), ref["labels"])


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_fixed_sweeps_labels_valid_at_main_size(gc, direction):
    """Fixed-sweep mode on the 384x288x16 pair: after 8, 32 and 128 sweep
    rounds the labels are one depth number per gaze line (the cut is a cut),
    the flow routed so far is a lower and the labels' energy an upper bound of
    the exact minimum."""
    wl = synth.MAIN
    L, R, _ = synth.make_pair(wl, 2)
    C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    Estar = oracle.solve(C, wl.lam, wl.inhibit, 1)["flow"]
    for n in (8, 32, 128):
        o = gc.SolveOpts(mode=gc.GS_MODE_FIXED_SWEEPS, fixed_sweeps=n, sweeps_per_relabel=8)
        X, flow, status, _ = _solve_costs(gc, C, wl.lam, wl.inhibit, 1, o, direction)
        assert status == gc.GS_OK
        assert X.shape == (wl.h, C.shape[1]) and X.min() >= 0 and X.max() <= wl.D - 1
        E = oracle.energy(C, X, wl.lam, wl.inhibit, 1)
        assert flow <= Estar <= E


def test_overflow_and_negative_cost_flagged(gc):
    p = gc.Params(w=20 + 6, h=4, D=4, tau=0, lam=1, inhibit=10)
    o = gc.SolveOpts()
    buf = gc.Buffers(p, o)
    C = np.zeros((4, 20, 4), dtype=np.int32)
    C[..., 0] = 1 << 28                      # 80 sites x 2^28 source capacity > 2^30
    gc.gs_build_graph(torch.from_numpy(C).cuda().reshape(-1), p, buf.graph, buf.status)
    assert int(buf.status.item()) == gc.GS_ERR_OVERFLOW
    C[...] = 1
    C[2, 3, 1] = -1
    gc.gs_build_graph(torch.from_numpy(C).cuda().reshape(-1), p, buf.graph, buf.status)
    assert int(buf.status.item()) == gc.GS_ERR_INVAL


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("which", ["tiny", "main"])
def test_chain_prepass_changes_time_not_the_cut(gc, engine, which):
    """The chain-local initial flow is only a head start: building without it
    gives the same flow and canonical labels (and both equal the oracle's)."""
    wl = synth.TINY if which == "tiny" else synth.MAIN
    L, R, _ = synth.make_pair(wl, 3)
    C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    ref = oracle.solve(C, wl.lam, wl.inhibit, 1)
    p = _params(gc, wl)
    o = gc.SolveOpts(engine=engine)
    c = torch.from_numpy(C).cuda().reshape(-1)
    for flags in (0, gc.GS_BUILD_CHAIN_PREFLOW):
        buf = gc.Buffers(p, o)
        gc.gs_build_graph_flags(c, p, flags, buf.graph, buf.status)
        gc.gs_maxflow_solve(buf.graph, p, o, buf.work, buf.status)
        gc.gs_extract_labels(buf.graph, p, o, buf.work, buf.labels, buf.flow, buf.status)
        assert int(buf.status.item()) == gc.GS_OK
        assert int(buf.flow.item()) == ref["flow"]
        assert np.array_equal(buf.labels.cpu().numpy(), ref["labels"])


@pytest.mark.parametrize("shape,lam,inh,vi,hi,tile", [
    ((37, 45, 5), 3, 50, 1, 20, (0, 0)),
    ((19, 70, 9), 2, 1023, 0, 30, (8, 8)),
    ((7, 45, 64), 3, 1023, 1, 30, (0, 0)),
    ((2, 9, 200), 2, 1023, 1, 40, (0, 0)),
    ((11, 97, 16), 10, 1023, 1, 30, (16, 8)),
    ((21, 64, 7), 1, 3, 1, 40, (4, 4)),
])
@pytest.mark.parametrize("direction", [1, 2])
def test_two_blocks_per_sm_exact(gc, shape, lam, inh, vi, hi, tile, direction):
    """256-thread blocks (two per SM where two tiles fit): the library's shape
    and explicit ones give the canonical cut in both solve directions."""
    rng = np.random.default_rng(sum(shape) * 11 + lam)
    C = rng.integers(0, hi + 1, size=shape).astype(np.int32)
    o = gc.SolveOpts(cta_threads=256, tile_w=tile[0], tile_h=tile[1])
    X, flow, status, _ = _solve_costs(gc, C, lam, inh, vi, o, direction)
    ref = oracle.solve(C, lam, inh, vi)
    assert status == gc.GS_OK
    assert flow == ref["flow"]
    assert np.array_equal(X, ref["labels"])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_two_blocks_per_sm_main_pair(gc, seed):
    """384x288 pairs with 16 depth numbers on 256-thread blocks (8x8 tiles, two
    blocks per SM), with the autotuned schedule, equal the oracle."""
    wl = synth.MAIN
    L, R, _ = synth.make_pair(wl, seed)
    p = _params(gc, wl)
    o = gc.SolveOpts(cta_threads=256, tile_w=8, tile_h=8, tail_iters=16, relabel_passes=16)
    assert gc.gs_tile_info(p, o)["smem_bytes"] < 80 * 1024
    labels, flow, status = gc.solve_pair(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), p, o)
    torch.cuda.synchronize()
    C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    ref = oracle.solve(C, wl.lam, wl.inhibit, 1)
    assert int(status.item()) == gc.GS_OK
    assert int(flow.item()) == ref["flow"]
    assert np.array_equal(labels.cpu().numpy(), ref["labels"])

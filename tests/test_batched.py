"""Batched solve: uneven pairs in one persistent launch, each bit-exact against
the oracle and against the single-pair path; CUDA-graph capture and replay."""
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


def _uneven_batch(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        D = int(rng.integers(4, 41))
        w = int(rng.integers(2 * (D - 1) + 20, 2 * (D - 1) + 140))
        h = int(rng.integers(9, 60))
        wl = synth.Workload(f"b{i}", w, h, D, tau=30, lam=int(rng.integers(2, 12)), sigma=2.0,
                            scene="layers", n_layers=3, n_slanted=1,
                            max_disp=min(2 * (D - 1), 20), seed_base=50 + seed)
        L, R, _ = synth.make_pair(wl, i)
        out.append((wl, L, R, int(rng.integers(0, 2))))
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_batched_matches_oracle_and_single(gc, seed):
    pairs = _uneven_batch(7, seed)
    params = [gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit,
                        vertical_inhibit=vi) for wl, _, _, vi in pairs]
    opts = [gc.SolveOpts() for _ in pairs]
    batch = gc.Batch(params, opts)
    Ls = [torch.from_numpy(L).cuda() for _, L, _, _ in pairs]
    Rs = [torch.from_numpy(R).cuda() for _, _, R, _ in pairs]
    gc.gs_solve_batched(batch, Ls, Rs)
    torch.cuda.synchronize()
    for (wl, L, R, vi), p, b, Ld, Rd in zip(pairs, params, batch.bufs, Ls, Rs):
        C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
        ref = oracle.solve(C, wl.lam, wl.inhibit, vi)
        assert int(b.status.item()) == gc.GS_OK
        assert int(b.flow.item()) == ref["flow"]
        assert np.array_equal(b.labels.cpu().numpy(), ref["labels"])
        lab, flow, status = gc.solve_pair(Ld, Rd, p)
        assert int(flow.item()) == ref["flow"] and np.array_equal(lab.cpu().numpy(), ref["labels"])


def test_batched_fixed_sweeps_and_mixed_options(gc):
    pairs = _uneven_batch(4, 3)
    params = [gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit)
              for wl, _, _, _ in pairs]
    opts = [gc.SolveOpts(), gc.SolveOpts(mode=gc.GS_MODE_FIXED_SWEEPS, fixed_sweeps=2),
            gc.SolveOpts(sweeps_per_relabel=2, local_iters=4), gc.SolveOpts(relabel_passes=16)]
    batch = gc.Batch(params, opts)
    gc.gs_solve_batched(batch, [torch.from_numpy(L).cuda() for _, L, _, _ in pairs],
                        [torch.from_numpy(R).cuda() for _, _, R, _ in pairs])
    torch.cuda.synchronize()
    for (wl, L, R, _), o, b in zip(pairs, opts, batch.bufs):
        C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
        ref = oracle.solve(C, wl.lam, wl.inhibit, 1)
        assert int(b.status.item()) == gc.GS_OK
        if o.mode == gc.GS_MODE_EXACT:
            assert int(b.flow.item()) == ref["flow"]
            assert np.array_equal(b.labels.cpu().numpy(), ref["labels"])
        else:
            E = oracle.energy(C, b.labels.cpu().numpy(), wl.lam, wl.inhibit, 1)
            assert int(b.flow.item()) <= ref["flow"] <= E


def test_batched_call_captured_in_a_cuda_graph(gc):
    pairs = _uneven_batch(5, 4)
    params = [gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit)
              for wl, _, _, _ in pairs]
    opts = [gc.SolveOpts() for _ in pairs]
    batch = gc.Batch(params, opts)
    Ls = [torch.from_numpy(L).cuda() for _, L, _, _ in pairs]
    Rs = [torch.from_numpy(R).cuda() for _, _, R, _ in pairs]
    gc.gs_solve_batched(batch, Ls, Rs)          # first call outside capture (set-up)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            gc.gs_solve_batched(batch, Ls, Rs)
    for b in batch.bufs:
        b.flow.zero_()
        b.labels.zero_()
    g.replay()
    torch.cuda.synchronize()
    for (wl, L, R, _), b in zip(pairs, batch.bufs):
        C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
        ref = oracle.solve(C, wl.lam, wl.inhibit, 1)
        assert int(b.status.item()) == gc.GS_OK
        assert int(b.flow.item()) == ref["flow"]
        assert np.array_equal(b.labels.cpu().numpy(), ref["labels"])


def test_full_batch_with_trivial_and_timed_out_pairs(gc):
    """64 pairs stepping independently: uneven random pairs, pairs with zero
    cost (nothing to route, E* = 0) and one pair held to a single relabel
    (GS_ERR_TIMEOUT) -- every other pair still ends exact and bit-equal to
    the oracle, and the timed-out pair's state resumes to the exact cut."""
    pairs = _uneven_batch(60, 7)
    flat = np.full((12, 40), 77, np.uint8)
    for i in range(3):
        wl = synth.Workload(f"flat{i}", 40, 12, 6 + i, tau=30, lam=3, sigma=0.0, scene="layers",
                            n_layers=1, n_slanted=0, max_disp=2, seed_base=1)
        pairs.append((wl, flat, flat, 1))
    tiny = synth.TINY
    L, R, _ = synth.make_pair(tiny, 2)
    pairs.append((tiny, L, R, 1))
    params = [gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit,
                        vertical_inhibit=vi) for wl, _, _, vi in pairs]
    opts = [gc.SolveOpts() for _ in pairs]
    opts[-1] = gc.SolveOpts(max_iters=1, sweeps_per_relabel=1)
    batch = gc.Batch(params, opts)
    Ls = [torch.from_numpy(np.ascontiguousarray(L)).cuda() for _, L, _, _ in pairs]
    Rs = [torch.from_numpy(np.ascontiguousarray(R)).cuda() for _, _, R, _ in pairs]
    gc.gs_solve_batched(batch, Ls, Rs)
    torch.cuda.synchronize()
    for i, ((wl, L, R, vi), p, b) in enumerate(zip(pairs, params, batch.bufs)):
        C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
        ref = oracle.solve(C, wl.lam, wl.inhibit, vi)
        if i == len(pairs) - 1:
            assert int(b.status.item()) == gc.GS_ERR_TIMEOUT
            b.status.zero_()
            o = gc.SolveOpts()
            gc.gs_maxflow_solve(b.graph, p, o, b.work, b.status)
            gc.gs_extract_labels(b.graph, p, o, b.work, b.labels, b.flow, b.status)
            torch.cuda.synchronize()
        assert int(b.status.item()) == gc.GS_OK, i
        assert int(b.flow.item()) == ref["flow"], i
        assert np.array_equal(b.labels.cpu().numpy(), ref["labels"]), i
        if i >= 60 and i < 63:
            assert ref["flow"] == 0


def _golden_batch64():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "batch64_oracle.txt")
    rows = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, w, h, D, sL, sR, flow, sX = line.split()
        rows[int(k)] = (int(w), int(h), int(D), sL, sR, int(flow), sX)
    return rows


def _sha16(a):
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:16]


def test_batch_workload_of_64_pairs_matches_oracle_pair_by_pair(gc):
    """The whole 64-pair batch workload (w ~ U[160, 640], h ~ U[120, 480],
    16-64 depth numbers, 224 M graph nodes) in one batched call with the
    autotuned options the bench uses: every pair's flow and labels equal the
    CPU oracle's exact cut.  The oracle's results come from
    golden/batch64_oracle.txt (written by golden/make_batch64_oracle.py, which
    calls only the oracle: flow and a SHA-256 of the labels per pair); a pair
    whose generated images hash differently on this machine is solved by the
    oracle here instead."""
    from paper_1803_01516_gb300 import autotune
    gold = _golden_batch64()
    batch = synth.make_batch(64)
    same = [(gold[k][3], gold[k][4]) == (_sha16(L), _sha16(R))
            for k, (_, L, R, _) in enumerate(batch)]
    assert sum(not x for x in same) <= 4, "the generated inputs differ from the golden run"
    params = [gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit,
                        vertical_inhibit=1) for wl, _, _, _ in batch]
    opts = [autotune.tuned_opts(p) for p in params]
    B = gc.Batch(params, opts)
    Ls = [torch.from_numpy(L).cuda() for _, L, _, _ in batch]
    Rs = [torch.from_numpy(R).cuda() for _, _, R, _ in batch]
    gc.gs_solve_batched(B, Ls, Rs)
    torch.cuda.synchronize()
    for k, ((wl, L, R, _), b) in enumerate(zip(batch, B.bufs)):
        w, h, D, sL, sR, flow, sX = gold[k]
        assert (w, h, D) == (wl.w, wl.h, wl.D), k
        assert int(b.status.item()) == gc.GS_OK, k
        X = b.labels.cpu().numpy().astype("<i4")
        if same[k]:
            assert int(b.flow.item()) == flow, k
            assert _sha16(X) == sX, k
        else:
            C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
            ref = oracle.solve(C, wl.lam, wl.inhibit, 1)
            assert int(b.flow.item()) == ref["flow"], k
            assert np.array_equal(X, ref["labels"]), k


@pytest.mark.parametrize("all256", [True, False])
def test_batched_block_size(gc, all256):
    """A batch runs on 256-thread blocks when every pair asks for them and on
    512-thread blocks otherwise; either way each pair equals the oracle."""
    pairs = _uneven_batch(6, 4)
    params = [gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit,
                        vertical_inhibit=vi) for wl, _, _, vi in pairs]
    opts = [gc.SolveOpts(cta_threads=256 if (all256 or i % 2) else 0) for i in range(len(pairs))]
    batch = gc.Batch(params, opts)
    gc.gs_solve_batched(batch, [torch.from_numpy(L).cuda() for _, L, _, _ in pairs],
                        [torch.from_numpy(R).cuda() for _, _, R, _ in pairs])
    torch.cuda.synchronize()
    for (wl, L, R, vi), b in zip(pairs, batch.bufs):
        C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
        ref = oracle.solve(C, wl.lam, wl.inhibit, vi)
        assert int(b.status.item()) == gc.GS_OK
        assert int(b.flow.item()) == ref["flow"]
        assert np.array_equal(b.labels.cpu().numpy(), ref["labels"])

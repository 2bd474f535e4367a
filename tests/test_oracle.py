"""Pins for the CPU oracle: brute force, the textbook chain DP, closed forms,
invariants and the numbers the paper prints.  CPU only."""
import os

import numpy as np
import pytest

import oracle
from oracle import small
from paper_1803_01516_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(t) for t in line.split()])
    return rows


# ---------------------------------------------------------------- h~ (§3) --

@pytest.mark.parametrize("lam,inh", [(14, 1023), (0, 0), (3, 7), (10, 0)])
def test_interaction_is_convex_eq1(lam, inh):
    """Eq. 1: h~(i+1) - 2h~(i) + h~(i-1) >= 0; for h~ of §3 the second
    difference is 2*h~1 at 0, h~2 at |i| = 1 and 0 beyond."""
    i = np.arange(-20, 21)
    h = small.htilde(i, lam, inh)
    d2 = h[2:] - 2 * h[1:-1] + h[:-2]
    mid = i[1:-1]
    assert (d2 >= 0).all()
    expect = np.where(mid == 0, 2 * lam, np.where(np.abs(mid) == 1, inh, 0))
    assert (d2 == expect).all()


# --------------------------------------------------------- brute force -----

def _random_case(rng, h, ng, D, hi=12):
    C = rng.integers(0, hi + 1, size=(h, ng, D)).astype(np.int32)
    return C, int(rng.integers(0, 7)), int(rng.integers(0, 25)), int(rng.integers(0, 2))


@pytest.mark.parametrize("seed", range(6))
def test_bk_dinic_match_brute_force_3x3x3(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(8):
        C, lam, inh, vi = _random_case(rng, 3, 3, 3)
        E, Xmin, _ = small.brute_force(C, lam, inh, vi)
        for method in ("bk", "dinic"):
            r = oracle.solve(C, lam, inh, vi, method)
            assert r["flow"] == E
            assert r["cut"] == E
            assert (r["labels"] == Xmin).all()
            assert oracle.energy(C, r["labels"], lam, inh, vi) == E
            assert oracle.energy(C, r["labels_max"], lam, inh, vi) == E
            assert (r["labels"] <= r["labels_max"]).all()


def test_brute_force_4x3x3_and_ties():
    """Larger enumeration (3^12 labelings) and costs with many ties, where the
    smallest minimiser differs from the largest."""
    rng = np.random.default_rng(7)
    saw_tie = False
    for _ in range(4):
        C = rng.integers(0, 3, size=(4, 3, 3)).astype(np.int32)
        E, Xmin, nmin = small.brute_force(C, 1, 2, 1)
        r = oracle.solve(C, 1, 2, 1, "bk")
        assert r["flow"] == E and (r["labels"] == Xmin).all()
        saw_tie |= nmin > 1 and (r["labels_max"] != r["labels"]).any()
    assert saw_tie


def test_brute_force_on_tiny_workload_subcrops():
    """3x3 sites x 3 consecutive depth numbers cut out of the 64x48x16 cost volume."""
    wl = synth.TINY
    L, R, _ = synth.make_pair(wl, 0)
    C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    rng = np.random.default_rng(11)
    for _ in range(10):
        y = int(rng.integers(0, C.shape[0] - 3))
        W = int(rng.integers(0, C.shape[1] - 3))
        S = int(rng.integers(0, wl.D - 3))
        crop = np.ascontiguousarray(C[y:y + 3, W:W + 3, S:S + 3])
        for vi in (0, 1):
            E, Xmin, _ = small.brute_force(crop, wl.lam, wl.inhibit, vi)
            r = oracle.solve(crop, wl.lam, wl.inhibit, vi, "bk")
            assert r["flow"] == E and (r["labels"] == Xmin).all()


def test_two_labels_and_single_site():
    rng = np.random.default_rng(3)
    for shape in [(1, 1, 2), (1, 1, 5), (2, 3, 2), (3, 1, 4), (1, 6, 2)]:
        C = rng.integers(0, 9, size=shape).astype(np.int32)
        E, Xmin, _ = small.brute_force(C, 2, 5, 1)
        r = oracle.solve(C, 2, 5, 1, "dinic")
        assert r["flow"] == E and (r["labels"] == Xmin).all()


# ------------------------------------------------------- textbook chain DP --

@pytest.mark.parametrize("which", ["tiny", "main"])
def test_single_row_matches_viterbi(which):
    """One row of sites is a chain MRF: min-sum DP is exact at any length."""
    wl = synth.TINY if which == "tiny" else synth.MAIN
    L, R, _ = synth.make_pair(wl, 0)
    C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    for y in (0, C.shape[0] // 2):
        row = np.ascontiguousarray(C[y:y + 1])
        E, X = small.viterbi_row(row[0], wl.lam, wl.inhibit)
        for method in ("bk", "dinic"):
            r = oracle.solve(row, wl.lam, wl.inhibit, 1, method)
            assert r["flow"] == E
            assert (r["labels"][0] == X).all()


def test_viterbi_is_exact_on_tiny_rows():
    """Pins the DP itself against enumeration."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        n, D = int(rng.integers(1, 7)), int(rng.integers(2, 4))
        C = rng.integers(0, 6, size=(1, n, D)).astype(np.int32)
        lam, inh = int(rng.integers(0, 4)), int(rng.integers(0, 6))
        E, Xmin, _ = small.brute_force(C, lam, inh)
        E2, X2 = small.viterbi_row(C[0], lam, inh)
        assert E == E2 and (Xmin[0] == X2).all()


# ------------------------------------------------------------ closed forms --

def test_no_interaction_is_per_site_argmin():
    rng = np.random.default_rng(8)
    C = rng.integers(0, 50, size=(9, 11, 7)).astype(np.int32)
    r = oracle.solve(C, 0, 0, 1)
    assert r["flow"] == int(C.min(axis=2).sum())
    assert (r["labels"] == C.argmin(axis=2)).all()          # first argmin = smallest


def test_constant_costs_give_zero_labels():
    C = np.full((6, 8, 5), 9, dtype=np.int32)
    r = oracle.solve(C, 3, 100, 1)
    assert r["flow"] == 9 * 6 * 8
    assert (r["labels"] == 0).all()
    assert (r["labels_max"] == 4).all()


def test_huge_penalty_gives_constant_labeling():
    rng = np.random.default_rng(9)
    C = rng.integers(0, 20, size=(5, 6, 6)).astype(np.int32)
    lam = int(C.max()) * C.shape[0] * C.shape[1] + 1
    r = oracle.solve(C, lam, 0, 1)
    tot = C.sum(axis=(0, 1))
    assert r["flow"] == int(tot.min())
    assert (r["labels"] == int(np.argmin(tot))).all()


def test_planted_surface():
    """Costs 0 on a surface with only +-1 steps and M elsewhere (M larger than
    every smoothness cost) -> E* = h~1 * #unit jumps and X = the surface."""
    rng = np.random.default_rng(10)
    h, ng, D, lam = 7, 9, 8, 3
    X = np.zeros((h, ng), dtype=np.int64)
    X[0, 0] = 4
    for y in range(h):
        for W in range(ng):
            if y == 0 and W == 0:
                continue
            base = X[y, W - 1] if W > 0 else X[y - 1, W]
            cand = [base + s for s in (-1, 0, 1) if 0 <= base + s < D]
            if y > 0:
                cand = [c for c in cand if abs(c - X[y - 1, W]) <= 1]
            X[y, W] = cand[int(rng.integers(0, len(cand)))]
    jumps = int(np.abs(np.diff(X, axis=1)).sum() + np.abs(np.diff(X, axis=0)).sum())
    M = lam * 4 * h * ng + 1
    C = np.full((h, ng, D), M, dtype=np.int32)
    yy, ww = np.meshgrid(np.arange(h), np.arange(ng), indexing="ij")
    C[yy, ww, X] = 0
    r = oracle.solve(C, lam, 1023, 1)
    assert r["flow"] == lam * jumps
    assert (r["labels"] == X).all()


# ------------------------------------------------------------ invariants ----

def test_energy_identity_and_solvers_agree_on_tiny_workload():
    wl = synth.TINY
    L, R, _ = synth.make_pair(wl, 0)
    C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    for vi in (0, 1):
        a = oracle.solve(C, wl.lam, wl.inhibit, vi, "bk")
        b = oracle.solve(C, wl.lam, wl.inhibit, vi, "dinic")
        assert a["flow"] == b["flow"] == a["cut"] == b["cut"]
        assert (a["labels"] == b["labels"]).all()
        assert oracle.energy(C, a["labels"], wl.lam, wl.inhibit, vi) == a["flow"]
        assert int(small.energy_np(C, a["labels"], wl.lam, wl.inhibit, vi)) == a["flow"]


def test_inhibit_1023_is_enough_big():
    """§4.3: doubling the inhibit constant does not increase the max flow."""
    wl = synth.TINY
    for i in range(2):
        L, R, _ = synth.make_pair(wl, i)
        C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
        a = oracle.solve(C, wl.lam, 1023, 1)
        b = oracle.solve(C, wl.lam, 2046, 1)
        assert a["flow"] == b["flow"]


# --------------------------------------------------------- cost volume -----

@pytest.mark.parametrize("D,parity", [(16, 0), (5, 1), (2, 0)])
def test_cost_volume_zero_on_true_depth(D, parity):
    """R(x) = L(x + dis) with dis = dis0 - 2 S*: the data term vanishes exactly
    on depth number S* (the cross points of §3 lie on that depth line)."""
    rng = np.random.default_rng(D)
    w, h = 80, 5
    dis0 = 2 * (D - 1) + parity
    L = rng.integers(0, 256, size=(h, w)).astype(np.uint8)
    for S_true in range(D):
        dis = dis0 - 2 * S_true
        xs = np.minimum(np.arange(w) + dis, w - 1)
        R = np.ascontiguousarray(L[:, xs])
        C = oracle.cost_volume(L, R, D, dis0, 255)
        assert C.shape == (h, w - dis0, D)
        assert (C[:, :, S_true] == 0).all()
        other = [s for s in range(D) if s != S_true]
        if other:
            assert (C[:, :, other] > 0).mean() > 0.9


def test_cost_volume_truncation_and_symmetry():
    """g_v is symmetric in the two images and truncated at tau."""
    rng = np.random.default_rng(1)
    L = rng.integers(0, 256, size=(4, 40)).astype(np.uint8)
    R = rng.integers(0, 256, size=(4, 40)).astype(np.uint8)
    C = oracle.cost_volume(L, R, 6, 10, 1000)
    Ct = oracle.cost_volume(L, R, 6, 10, 30)
    assert (Ct == np.minimum(C, 30)).all()
    assert C.max() <= 255
    # swapping the images and mirroring x maps cross point (W, S) to (n_g-1-W, S)
    Cs = oracle.cost_volume(R[:, ::-1].copy(), L[:, ::-1].copy(), 6, 10, 1000)
    assert (Cs[:, ::-1, :] == C).all()


def test_bad_sizes_raise():
    L = np.zeros((4, 10), dtype=np.uint8)
    with pytest.raises(ValueError):
        oracle.cost_volume(L, L, 6, 10, 30)       # n_g = 0
    with pytest.raises(ValueError):
        oracle.cost_volume(L, L, 6, 9, 30)        # dis0 < 2(D-1)


# ---------------------------------------------------- numbers in the paper --

def test_paper_node_count():
    for sw, sh, D, nodes in _read_golden("paper_node_count.txt"):
        n, _ = oracle.graph_size(sw, sh, D)
        assert n == nodes


def test_paper_table1_error_total():
    """Eq. 2: error = sum over d of d x (number of sites); Table 1 totals 11578."""
    from paper_1803_01516_gb300.metrics import depth_error_from_hist
    rows = _read_golden("paper_table1.txt")
    hist = np.zeros(max(d for d, _ in rows) + 1, dtype=np.int64)
    for d, n in rows:
        hist[d] = n
    assert depth_error_from_hist(hist) == 11578


# ------------------------------------------------ colour data term (§4.3) ---

def test_rgb_cost_of_gray_images_is_three_times_the_gray_cost():
    """A grey image copied into all three channels: every channel contributes
    the grey absolute difference, so the colour sum is three times it."""
    L, R, _ = synth.make_pair(synth.TINY, 0)
    L3, R3 = np.repeat(L[:, :, None], 3, axis=2), np.repeat(R[:, :, None], 3, axis=2)
    C3 = oracle.cost_volume_rgb(L3, R3, 16, 30, 10 ** 6)
    C1 = oracle.cost_volume(L, R, 16, 30, 10 ** 6)
    assert np.array_equal(C3, 3 * C1)
    # truncation applies to the sum
    assert np.array_equal(oracle.cost_volume_rgb(L3, R3, 16, 30, 40), np.minimum(3 * C1, 40))


def test_rgb_cost_range_channels_and_geometry():
    """Black against white costs 765 (the paper's maximum); one differing
    channel costs that channel's difference; permuting the channels of both
    images changes nothing; the cross point (W, S) pairs left pixel
    W + dis0 - S with right pixel W + S."""
    h, w, D, dis0 = 2, 12, 3, 4
    L = np.zeros((h, w, 3), np.uint8)
    R = np.full((h, w, 3), 255, np.uint8)
    assert (oracle.cost_volume_rgb(L, R, D, dis0, 10 ** 6) == 765).all()
    R = L.copy()
    R[:, :, 1] = 7
    assert (oracle.cost_volume_rgb(L, R, D, dis0, 10 ** 6) == 7).all()
    rng = np.random.default_rng(3)
    L = rng.integers(0, 256, size=(h, w, 3)).astype(np.uint8)
    R = rng.integers(0, 256, size=(h, w, 3)).astype(np.uint8)
    C = oracle.cost_volume_rgb(L, R, D, dis0, 10 ** 6)
    perm = [2, 0, 1]
    assert np.array_equal(oracle.cost_volume_rgb(L[:, :, perm], R[:, :, perm], D, dis0, 10 ** 6), C)
    for (y, W, S) in [(0, 0, 0), (1, 7, 2), (0, 3, 1)]:
        want = int(np.abs(L[y, W + dis0 - S].astype(int) - R[y, W + S].astype(int)).sum())
        assert C[y, W, S] == want


def test_rgb_cost_zero_on_true_depth():
    """Noise-free colour pair warped by a constant even disparity 2s: the
    cross point at depth number D-1-s (dis = 2s) matches exactly."""
    wl = synth.Workload("rgbflat", 40, 6, 5, tau=765, lam=1, sigma=0.0, scene="rects",
                        rect_disps=(), max_disp=8)
    L, _, _ = synth.make_pair_rgb(wl, 0)
    for s in range(3):
        d = 2 * s
        R = np.concatenate([L[:, d:], L[:, -1:].repeat(d, axis=1)], axis=1) if d else L.copy()
        C = oracle.cost_volume_rgb(L, R, 5, 8, 765)
        S = 4 - s                                   # dis(S) = 8 - 2S = d
        assert (C[:, :, S] == 0).all()

"""Pins of the level-1 approximation oracle (§4.5): the restricted second cut
against enumeration, its reduction to the exact cut, and the b = 1 case that
the paper states is the exact minimisation."""
import numpy as np
import pytest

import oracle
from oracle import level1 as l1
from oracle import small


def _rand(seed, h, ng, D, hi=30):
    return np.random.default_rng(seed).integers(0, hi, size=(h, ng, D)).astype(np.int32)


def _rand_bounds(seed, h, ng, D, width):
    rng = np.random.default_rng(seed)
    lo = rng.integers(0, D, size=(h, ng))
    hi = np.minimum(lo + rng.integers(0, width, size=(h, ng)), D - 1)
    return lo.astype(np.int32), hi.astype(np.int32)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("vi", [1, 0])
def test_band_solve_matches_enumeration(seed, vi):
    """Restricted minimum and its smallest minimiser equal exhaustive search
    over every labeling inside the bounds (3x3 sites, D = 5, up to 3 labels each)."""
    C = _rand(seed, 3, 3, 5)
    lo, hi = _rand_bounds(100 + seed, 3, 3, 5, 3)
    lam, inh = (3, 7) if seed % 2 else (6, 50)
    Eb, Xb, _ = small.brute_force_band(C, lam, inh, vi, lo, hi)
    r = oracle.solve_band(C, lam, inh, vi, lo, hi)
    assert r["flow"] == Eb
    assert np.array_equal(r["labels"], Xb)
    assert oracle.energy(C, r["labels"], lam, inh, vi) == Eb
    d = oracle.solve_band(C, lam, inh, vi, lo, hi, method="dinic")
    assert d["flow"] == Eb and np.array_equal(d["labels"], Xb)


def test_band_solve_with_full_bounds_is_the_exact_cut():
    C = _rand(7, 9, 11, 8)
    lo = np.zeros((9, 11), np.int32)
    hi = np.full((9, 11), 7, np.int32)
    ref = oracle.solve(C, 5, 60, 1)
    r = oracle.solve_band(C, 5, 60, 1, lo, hi)
    assert r["flow"] == ref["flow"]
    assert np.array_equal(r["labels"], ref["labels"])


def test_band_solve_pins_every_site_when_bounds_are_single_labels():
    """lo = hi = X forces the labeling: labels X, flow E(X)."""
    C = _rand(8, 5, 6, 6)
    X = np.random.default_rng(9).integers(0, 6, size=(5, 6)).astype(np.int32)
    r = oracle.solve_band(C, 4, 30, 1, X, X)
    assert np.array_equal(r["labels"], X)
    assert r["flow"] == oracle.energy(C, X, 4, 30, 1)


def test_bad_bounds_rejected():
    C = _rand(1, 2, 2, 4)
    lo = np.array([[0, 2], [1, 0]], np.int32)
    hi = np.array([[1, 1], [3, 3]], np.int32)      # lo > hi at one site
    with pytest.raises(RuntimeError):
        oracle.solve_band(C, 1, 1, 1, lo, hi)


def test_coarse_costs_closed_forms():
    """b = 1 is the identity; a constant volume gives the number of sites of
    the block times the constant (ragged edge blocks included); a volume that
    depends on the depth bin only sums that value over the block."""
    C = _rand(3, 7, 9, 8)
    assert np.array_equal(l1.coarse_costs(C, 1), C)
    K = np.full((7, 9, 8), 5, np.int32)
    Cc = l1.coarse_costs(K, 3)
    assert Cc.shape == (3, 3, 3)
    for yc in range(3):
        for Wc in range(3):
            n = (min(7, 3 * yc + 3) - 3 * yc) * (min(9, 3 * Wc + 3) - 3 * Wc)
            assert (Cc[yc, Wc] == 5 * n).all()
    f = np.random.default_rng(4).integers(0, 20, size=(4, 6, 4))       # value per bin
    B = np.repeat(f, 2, axis=2).astype(np.int32)                       # D = 8, bins of 2
    Cc = l1.coarse_costs(B, 2)
    assert np.array_equal(Cc, f.reshape(2, 2, 3, 2, 4).sum(axis=(1, 3)))


def test_skin_bounds_cover_the_delegate_bin():
    Xc = np.array([[0, 3], [2, 1]])
    lo, hi = l1.skin_bounds(Xc, 2, 4, 3, 8)
    assert lo.shape == (4, 3)
    for y in range(4):
        for W in range(3):
            Lc = Xc[y // 2, W // 2]
            assert lo[y, W] <= 2 * Lc and min(2 * Lc + 1, 7) <= hi[y, W]
            assert lo[y, W] == max(0, 2 * Lc - 2) and hi[y, W] == min(7, 2 * Lc + 3)


@pytest.mark.parametrize("seed", range(4))
def test_level1_block_size_one_is_exact(seed):
    """§4.5: with block size 1 the first cut finds the real cross points."""
    C = _rand(20 + seed, 8, 10, 8)
    ref = oracle.solve(C, 4, 40, 1)
    r = l1.level1(C, 4, 40, 1, 1)
    assert r["energy"] == ref["flow"]
    assert np.array_equal(r["labels"], ref["labels"])


@pytest.mark.parametrize("b", [2, 3])
@pytest.mark.parametrize("seed", range(3))
def test_level1_gap_nonnegative_and_zero_when_skin_holds_the_optimum(b, seed):
    C = _rand(30 + seed, 9, 12, 10)
    ref = oracle.solve(C, 4, 40, 1)
    r = l1.level1(C, 4, 40, 1, b)
    assert r["energy"] >= ref["flow"]
    assert (r["lo"] <= r["labels"]).all() and (r["labels"] <= r["hi"]).all()
    X = ref["labels"]
    if ((r["lo"] <= X) & (X <= r["hi"])).all():
        assert r["energy"] == ref["flow"]
        assert np.array_equal(r["labels"], X)
    # the second cut is the exact restricted minimum: enumerating around it
    # cannot improve (checked site by site: any single in-skin change)
    E0 = r["energy"]
    lab = r["labels"].copy()
    for y in range(C.shape[0]):
        for W in range(C.shape[1]):
            for l in range(r["lo"][y, W], r["hi"][y, W] + 1):
                t = lab.copy()
                t[y, W] = l
                assert oracle.energy(C, t, 4, 40, 1) >= E0


def test_level1_on_the_tiny_workload():
    from paper_1803_01516_gb300 import synth
    wl = synth.TINY
    L, R, _ = synth.make_pair(wl, 0)
    C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    ref = oracle.solve(C, wl.lam, wl.inhibit, 1)
    for b in (2, 3):
        r = l1.level1(C, wl.lam, wl.inhibit, 1, b)
        assert r["energy"] >= ref["flow"]
        assert r["coarse_labels"].shape == tuple(-(-n // b) for n in C.shape[:2])

"""Pins of the level-2 approximation oracle (oracle/level2.py, §4.5).

The block cut is checked against enumeration of the whole grid's energy with
the sites outside the block held (so a wrong border term, a doubled pair or a
vertical inhibit applied when it should not be fails), one block spanning the
grid against the level-1 second cut, the two-colour order by a non-increasing
energy after every half-pass, and the whole approximation by the bracket
E* <= E(level 1) <= E(level 2) <= E(start).
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import level1 as l1
from oracle import level2 as l2
from oracle import small
from paper_1803_01516_gb300 import synth


def _rand(seed, h, ng, D, hi=30):
    return np.random.default_rng(seed).integers(0, hi + 1, size=(h, ng, D)).astype(np.int32)


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("vi", [1, 0])
def test_block_cut_is_the_exact_conditional_minimum(seed, vi):
    rng = np.random.default_rng(50 + seed)
    h, ng, D = 4, 6, 6
    C = _rand(seed, h, ng, D, 12)
    lam, inh = int(rng.integers(1, 7)), int(rng.integers(2, 14))
    lo = rng.integers(0, 3, size=(h, ng)).astype(np.int32)
    hi = np.minimum(lo + rng.integers(1, 4, size=(h, ng)), D - 1).astype(np.int32)
    X = rng.integers(0, D, size=(h, ng)).astype(np.int32)      # any labels outside
    y0, y1, W0, W1 = 2, 4, 2, 4                      # the 2 x 2 block (1, 1) of b = 2
    Cb = l2.border_costs(C, X, lam, inh, vi, 2)[y0:y1, W0:W1]
    got = oracle.solve_band(Cb.astype(np.int32), lam, inh, vi, lo[y0:y1, W0:W1],
                            hi[y0:y1, W0:W1])["labels"]
    # enumerate the block's labelings inside the bounds, whole-grid energy
    ranges = [range(int(lo[y, W]), int(hi[y, W]) + 1) for y in range(y0, y1)
              for W in range(W0, W1)]
    best, mins = None, []
    for lab in itertools.product(*ranges):
        Y = X.copy()
        Y[y0:y1, W0:W1] = np.array(lab).reshape(y1 - y0, W1 - W0)
        E = int(small.energy_np(C, Y, lam, inh, vi))
        if best is None or E < best:
            best, mins = E, [Y[y0:y1, W0:W1].copy()]
        elif E == best:
            mins.append(Y[y0:y1, W0:W1].copy())
    assert np.array_equal(got, np.min(mins, axis=0))


@pytest.mark.parametrize("seed", range(4))
def test_one_block_spanning_the_grid_is_the_level1_second_cut(seed):
    """With a block covering every site there is no border term: the block cut
    is the exact restricted minimum, whatever the start labels."""
    rng = np.random.default_rng(80 + seed)
    h, ng, D = 5, 7, 9
    C = _rand(seed + 10, h, ng, D, 25)
    lo = rng.integers(0, 4, size=(h, ng)).astype(np.int32)
    hi = np.minimum(lo + 4, D - 1).astype(np.int32)
    X0 = lo.copy()
    X = l2.block_descent(C, X0, 3, 9, 1, 8, lo, hi, passes=1)
    want = oracle.solve_band(C, 3, 9, 1, lo, hi)["labels"]
    assert np.array_equal(X, want)


@pytest.mark.parametrize("b", [2, 3])
@pytest.mark.parametrize("seed", range(3))
def test_energy_never_increases_and_is_bracketed(b, seed):
    C = _rand(seed + 20, 9, 11, 10, 30)
    lam, inh = 4, 15
    r = l2.level2(C, lam, inh, 1, b, passes=3)
    t = r["trace"]
    assert all(t[i + 1] <= t[i] for i in range(len(t) - 1)), t
    Estar = oracle.solve(C, lam, inh, 1)["flow"]
    E1 = l1.level1(C, lam, inh, 1, b)["energy"]
    assert Estar <= E1 <= r["energy"] <= t[0]
    assert ((r["labels"] >= r["lo"]) & (r["labels"] <= r["hi"])).all()


def test_start_labels_are_the_best_cross_point_in_the_delegate_bin():
    C = _rand(5, 6, 7, 11, 40)
    b = 3
    Xc = np.random.default_rng(1).integers(0, 4, size=(2, 3))
    X = l2.start_labels(C, Xc, b)
    for y in range(6):
        for W in range(7):
            a = b * int(Xc[y // b, W // b])
            z = min(a + b, 11)
            assert a <= X[y, W] < z
            seg = C[y, W, a:z]
            assert C[y, W, X[y, W]] == seg.min()
            assert X[y, W] == a + int(np.flatnonzero(seg == seg.min())[0])


def test_block_size_one_keeps_the_exact_minimum():
    """b = 1: the delegate cut is the exact cut and the start labels are its
    labels, a global minimiser; single-site cuts keep the energy at E*."""
    C = _rand(7, 6, 8, 6, 20)
    r = l2.level2(C, 3, 9, 1, 1, passes=2)
    assert r["energy"] == oracle.solve(C, 3, 9, 1)["flow"]


def test_level2_on_the_tiny_workload():
    wl = synth.TINY
    L, R, _ = synth.make_pair(wl, 0)
    C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
    Estar = oracle.solve(C, wl.lam, wl.inhibit, 1)["flow"]
    for b in (2, 3):
        r = l2.level2(C, wl.lam, wl.inhibit, 1, b, passes=2)
        assert Estar <= r["energy"] <= r["trace"][0]

"""The seeded input generator and the accuracy report (both shared by the CUDA
path and the oracle, neither holds method arithmetic): determinism, the
scene recipe's invariants, and closed forms of Eq. 2 and the ground-truth
depth of §4.1."""
from dataclasses import replace

import numpy as np

from paper_1803_01516_gb300 import metrics, synth


def test_pairs_are_seeded_and_distinct():
    a = synth.make_pair(synth.TINY, 3)
    b = synth.make_pair(synth.TINY, 3)
    c = synth.make_pair(synth.TINY, 4)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert not np.array_equal(a[0], c[0])
    L, R, dR = a
    assert L.dtype == R.dtype == np.uint8 and dR.dtype == np.int32
    assert L.shape == R.shape == dR.shape == (synth.TINY.h, synth.TINY.w)
    assert L.flags["C_CONTIGUOUS"] and R.flags["C_CONTIGUOUS"]


def test_noise_free_warp_matches_the_disparity_map():
    """R(x, y) = L(min(x + d_R(x, y), w - 1), y) exactly when sigma = 0."""
    for wl in (synth.TINY, synth.MAIN):
        quiet = replace(wl, sigma=0.0)
        L, R, dR = synth.make_pair(quiet, 1)
        xs = np.minimum(np.arange(wl.w)[None, :] + dR, wl.w - 1)
        assert np.array_equal(R, np.take_along_axis(L, xs, axis=1))
        assert dR.min() >= 0 and dR.max() <= wl.max_disp


def test_scene_recipes():
    # rectangles: only the background and the three rectangle disparities
    _, _, dR = synth.make_pair(synth.TINY, 0)
    assert set(np.unique(dR).tolist()) <= {0, 2, 7, 12}
    # layers: the nearest layer sits at the maximum disparity
    _, _, dR = synth.make_pair(synth.MAIN, 0)
    assert dR.max() == synth.MAIN.max_disp
    # texture: a 3x3 box blur of uniform noise stays inside 0..255 and is not flat
    L, _, _ = synth.make_pair(synth.MAIN, 0)
    assert 20 < L.std() < 80


def test_batch_follows_its_size_ranges():
    batch = synth.make_batch(16)
    assert len(batch) == 16
    for wl, L, R, dR in batch:
        assert 120 <= wl.h <= 480 and 16 <= wl.D <= 64
        assert 160 <= wl.w <= 640 or wl.w == 2 * (wl.D - 1) + 8
        assert wl.w - 2 * (wl.D - 1) >= 8                   # sites left on every gaze line
        assert L.shape == (wl.h, wl.w) and dR.max() <= wl.max_disp <= 2 * (wl.D - 1)
    again = synth.make_batch(16)
    assert all(np.array_equal(a[1], b[1]) for a, b in zip(batch, again))


def test_ground_truth_depth_of_constant_disparity():
    """§4.1: dis(S) = dis0 - 2S; the first cross point at or behind the surface
    is S = ceil((dis0 - d) / 2) -- an odd difference rounds away from the front."""
    D, dis0, w, h = 16, 30, 64, 3
    for d in range(0, 31):
        gt = metrics.gt_depth(np.full((h, w), d), D, dis0)
        want = min(D - 1, -(-(dis0 - d) // 2))
        assert (gt == want).all(), d


def test_ground_truth_depth_reads_the_gaze_line_pixel():
    """Site W at depth S looks at right pixel W + S: a step in d_R shows up at
    the depth whose cross point first lands on the near side."""
    D, dis0, w = 8, 14, 40
    dR = np.zeros((1, w), np.int64)
    dR[0, 20:] = 14                           # near surface (dis = 14 at S = 0) right of x = 20
    gt = metrics.gt_depth(dR, D, dis0)[0]
    for W in range(w - dis0):
        # the smallest S with dis0 - 2S <= dR[W + S]
        S = next((s for s in range(D) if dis0 - 2 * s <= dR[0, W + s]), D - 1)
        assert gt[W] == S
    assert gt[20] == 0 and gt[0] == D - 1


def test_eq2_error_closed_forms():
    gt = np.array([[0, 1, 2], [3, 4, 5]])
    assert metrics.depth_error(gt, gt) == (0, 1.0)
    err, frac = metrics.depth_error(gt + 1, gt)
    assert err == 6 and frac == 0.0
    X = gt.copy()
    X[0, 0] = 3                                # one site off by 3
    hist = metrics.depth_error_hist(X, gt)
    assert hist.tolist() == [5, 0, 0, 1]
    assert metrics.depth_error_from_hist(hist) == 3

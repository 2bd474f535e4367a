"""The learned data term and the adjoint of the minimum energy.

CPU part: the oracle's FP32 cost and adjoint are pinned by closed forms and by
the concavity of E* (forward and backward differences bracket the gradient).
GPU part: the CUDA cost volume is bit-exact against the oracle; the backward
kernels equal the oracle's adjoint at the oracle's minimiser; autograd through
the exact solve; a few hinge-loss steps.
"""
import numpy as np
import pytest

import oracle
from oracle import learned, small
from paper_1803_01516_gb300 import synth


# ------------------------------------------------------------- CPU pins ---

def test_dx_of_a_ramp():
    I = (3 * np.arange(10))[None, :].repeat(2, axis=0).astype(np.uint8)
    d = learned.dx(I)
    assert np.allclose(d[:, 1:-1], 3.0) and np.allclose(d[:, [0, -1]], 1.5)


def test_f32_cost_reduces_to_integer_cost():
    """w2 = 0, tau beyond the largest value: the quantised cost is the integer
    absolute difference times scale * w1 (w1 a multiple of 1/256)."""
    L, R, _ = synth.make_pair(synth.TINY, 0)
    for w1 in (1.0, 0.5, 3.0 / 256):
        q = learned.cost_volume_f32(L, R, 16, 30, w1, 0.0, 1e6, 256.0)
        base = oracle.cost_volume(L, R, 16, 30, 1 << 20)
        assert np.array_equal(q, (base * round(256 * w1)).astype(np.int32))


def test_f32_cost_truncation_and_rounding():
    L, R, _ = synth.make_pair(synth.TINY, 1)
    q = learned.cost_volume_f32(L, R, 16, 30, 1.0, 1.0, 30.0, 256.0)
    assert q.max() == 30 * 256 and q.min() >= 0
    # w2 / 256 * (half-integer) -> ties at .5 round to even
    q2 = learned.cost_volume_f32(L, R, 4, 6, 0.0, 1.0 / 256, 1e6, 256.0)
    a, b = learned._features(L, R, 4, 6)
    assert np.array_equal(q2, np.rint(b).astype(np.int32))


def _sandwich_costs(C, lam, inh, vi, X, rng, trials=12):
    E0 = oracle.solve(C, lam, inh, vi)["flow"]
    h, ng, D = C.shape
    onehot, _, _ = learned.energy_adjoint(X, D, vi)
    for _ in range(trials):
        y, w, l = int(rng.integers(h)), int(rng.integers(ng)), int(rng.integers(D))
        Cp = C.copy()
        Cp[y, w, l] += 1
        up = oracle.solve(Cp, lam, inh, vi)["flow"] - E0
        if C[y, w, l] >= 1:
            Cm = C.copy()
            Cm[y, w, l] -= 1
            down = E0 - oracle.solve(Cm, lam, inh, vi)["flow"]
        else:
            down = 1
        assert up <= onehot[y, w, l] <= down


@pytest.mark.parametrize("seed", range(3))
def test_adjoint_is_bracketed_by_finite_differences(seed):
    """E* is concave in each cost and weight: E*(x+1) - E*(x) <= dE*/dx <=
    E*(x) - E*(x-1) at any minimiser (integer steps, exact)."""
    rng = np.random.default_rng(200 + seed)
    C = rng.integers(0, 12, size=(4, 5, 5)).astype(np.int32)
    lam, inh, vi = 3, 7, 1
    X = oracle.solve(C, lam, inh, vi)["labels"]
    _sandwich_costs(C, lam, inh, vi, X, rng)
    _, J, V = learned.energy_adjoint(X, 5, vi)
    E = {d: oracle.solve(C, lam + d, inh, vi)["flow"] for d in (-1, 0, 1)}
    assert E[1] - E[0] <= J <= E[0] - E[-1]
    E = {d: oracle.solve(C, lam, inh + d, vi)["flow"] for d in (-1, 0, 1)}
    assert E[1] - E[0] <= V <= E[0] - E[-1]


def test_adjoint_equals_difference_when_minimiser_unique():
    """With a unique minimiser (brute force), the forward difference in lambda
    equals the jump count exactly."""
    rng = np.random.default_rng(9)
    hits = 0
    for _ in range(40):
        C = rng.integers(0, 20, size=(2, 3, 4)).astype(np.int32)
        E, Xmin, nmin = small.brute_force(C, 2, 5, 1)
        if nmin != 1:
            continue
        _, J, _ = learned.energy_adjoint(Xmin, 4, 1)
        Ep, Xp, np_ = small.brute_force(C, 3, 5, 1)
        if np_ == 1 and np.array_equal(Xp, Xmin):
            assert Ep - E == J
            hits += 1
    assert hits > 5


def _tiny_images(rng, h=3, ng=3, D=3):
    """Random uint8 images for h x ng sites and D depth numbers (dis0 = 2(D-1)),
    values in 0..60: every feature is then at most 60, so a step of 1/256 in w1
    or 2/256 in w2 moves a cost below tau by less than half a unit and never
    across tau (costs at w1 = w2 = 1 are multiples of 1/2, tau is an integer)."""
    w = 2 * (D - 1) + ng
    L = rng.integers(0, 61, size=(h, w)).astype(np.uint8)
    R = rng.integers(0, 61, size=(h, w)).astype(np.uint8)
    return L, R


def test_cost_grad_sums_equal_exact_finite_differences():
    """cost_grad_sums against finite differences of the oracle's E* where the
    minimiser is unique on both sides of the step (brute force over all 3^9
    labelings): scaled by 256 the costs change exactly by the summed features,
        E*(w1 + 1/256) - E*(w1)   = sums[0]           (sum |L-R| [c < tau])
        E*(w2 + 2/256) - E*(w2)   = sums[1]           (sum 2|dxL-dxR| [c < tau])
        E*(tau) - E*(tau - 1/256) = sums[2]           (sum [c >= tau], left derivative)
        E*(tau + 1/256) - E*(tau) <= sums[2]          (right derivative counts c > tau)
    in units of 1/256 of the energy.  A dropped factor 2, a swapped feature or
    [c <= tau] against [c < tau] fails one of them."""
    rng = np.random.default_rng(77)
    D, dis0, scale = 3, 4, 256.0
    w1, w2, tau, lam, inh = 1.0, 1.0, 20.0, 6, 9
    lam_i, inh_i = int(lam * scale), int(inh * scale)
    hits = {"w1": 0, "w2": 0, "tau": 0, "tau_tie": 0}

    def bf(L, R, a, b, t):
        C = learned.cost_volume_f32(L, R, D, dis0, a, b, t, scale)
        return small.brute_force(C, lam_i, inh_i, 1)

    for _ in range(60):
        L, R = _tiny_images(rng)
        E0, X0, n0 = bf(L, R, w1, w2, tau)
        if n0 != 1:
            continue
        s = learned.cost_grad_sums(L, R, D, dis0, w1, w2, tau, X0)
        E, X, n = bf(L, R, w1 + 1 / scale, w2, tau)
        if n == 1 and np.array_equal(X, X0):
            assert E - E0 == s[0]
            hits["w1"] += 1
        E, X, n = bf(L, R, w1, w2 + 2 / scale, tau)
        if n == 1 and np.array_equal(X, X0):
            assert E - E0 == s[1]
            hits["w2"] += 1
        Em, Xm, nm = bf(L, R, w1, w2, tau - 1 / scale)
        Ep, Xp, np_ = bf(L, R, w1, w2, tau + 1 / scale)
        if nm == 1 and np.array_equal(Xm, X0):
            assert E0 - Em == s[2]
            hits["tau"] += 1
            if np_ == 1 and np.array_equal(Xp, X0):
                assert Ep - E0 <= s[2]
                hits["tau_tie"] += int(Ep - E0 < s[2])    # a site with c == tau at X*
    assert hits["w1"] >= 10 and hits["w2"] >= 10 and hits["tau"] >= 10, hits
    assert hits["tau_tie"] >= 1, hits


@pytest.mark.parametrize("seed", range(3))
def test_cost_grad_sums_bracketed_at_any_minimiser(seed):
    """E* is concave in w1, w2 and tau (a minimum of functions concave in each):
    at the oracle's minimiser the backward difference is an upper and the
    forward difference a lower bound of the chain-rule sums (no uniqueness
    needed; 4 x 5 sites, 4 depth numbers, max-flow oracle)."""
    rng = np.random.default_rng(300 + seed)
    D, dis0, scale = 4, 6, 256.0
    w1, w2, tau, lam, inh = 1.0, 1.0, 25.0, 5, 11
    L, R = _tiny_images(rng, h=4, ng=5, D=D)

    def Estar(a, b, t):
        C = learned.cost_volume_f32(L, R, D, dis0, a, b, t, scale)
        return oracle.solve(C, int(lam * scale), int(inh * scale), 1)

    r0 = Estar(w1, w2, tau)
    s = learned.cost_grad_sums(L, R, D, dis0, w1, w2, tau, r0["labels"])
    E0 = r0["flow"]
    for k, (dw1, dw2, dt, g) in enumerate([(1, 0, 0, s[0]), (0, 2, 0, s[1]), (0, 0, 1, s[2])]):
        up = Estar(w1 + dw1 / scale, w2 + dw2 / scale, tau + dt / scale)["flow"] - E0
        down = E0 - Estar(w1 - dw1 / scale, w2 - dw2 / scale, tau - dt / scale)["flow"]
        assert up <= g <= down, (k, up, g, down)


# -------------------------------------------------------------- GPU part ---

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_01516_gb300 import build
    build.build()
    from paper_1803_01516_gb300 import gazecut
    return gazecut


def _pair(wl, idx, D=None):
    L, R, dR = synth.make_pair(wl, idx)
    return L, R, dR


@pytest.mark.gpu
@pytest.mark.parametrize("theta", [(1.0, 1.0, 30.0), (0.5, 2.0, 12.5), (1.25, 0.0, 1000.0),
                                   (0.0, 3.0 / 256, 7.0)])
def test_f32_cost_volume_bit_exact(gc, theta):
    w1, w2, tau = theta
    for wl, D in ((synth.TINY, 16), (synth.MAIN, 32)):
        L, R, _ = _pair(wl, 0)
        p = gc.Params(w=wl.w, h=wl.h, D=D, tau=0, lam=0)
        cost = torch.empty(gc.gs_cost_volume_bytes(p) // 4, dtype=torch.int32, device="cuda")
        gc.gs_stereo_cost_volume_f32(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), p,
                                     w1, w2, tau, 256.0, cost)
        ref = learned.cost_volume_f32(L, R, D, 2 * (D - 1), w1, w2, tau, 256.0)
        assert np.array_equal(cost.cpu().numpy().reshape(ref.shape), ref)


@pytest.mark.gpu
@pytest.mark.parametrize("vi", [1, 0])
def test_backward_kernels_match_oracle_adjoint(gc, vi):
    wl = synth.TINY
    L, R, _ = _pair(wl, 2)
    w1, w2, tau, scale = 1.0, 0.5, 20.0, 256.0
    D = wl.D
    C = learned.cost_volume_f32(L, R, D, 2 * (D - 1), w1, w2, tau, scale)
    lam_i, inh = 8 * 256, 1023 * 256
    ref = oracle.solve(C, lam_i, inh, vi)
    X = ref["labels"]
    p = gc.Params(w=wl.w, h=wl.h, D=D, tau=0, lam=lam_i, inhibit=inh, vertical_inhibit=vi)
    Xd = torch.from_numpy(X).cuda()
    dcost = torch.empty((wl.h, p.ng, D), dtype=torch.float32, device="cuda")
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    gc.gs_energy_backward(Xd, p, 0.75, dcost, counts)
    onehot, J, V = learned.energy_adjoint(X, D, vi)
    assert np.array_equal(dcost.cpu().numpy(), 0.75 * onehot)
    assert counts.cpu().tolist() == [J, V]
    sums = torch.zeros(3, dtype=torch.int64, device="cuda")
    gc.gs_cost_volume_f32_backward(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), p,
                                   w1, w2, tau, Xd, sums)
    assert tuple(sums.cpu().tolist()) == learned.cost_grad_sums(L, R, D, 2 * (D - 1), w1, w2, tau, X)


@pytest.mark.gpu
def test_autograd_value_and_gradient(gc):
    from paper_1803_01516_gb300 import learn
    wl = synth.TINY
    L, R, _ = _pair(wl, 0)
    D, scale = wl.D, 256.0
    theta = torch.tensor([1.0, 0.5, 20.0, 8.0], dtype=torch.float64, requires_grad=True)
    p = gc.Params(w=wl.w, h=wl.h, D=D, tau=0, lam=0, inhibit=1023 * 256)
    pr = learn.problem(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), p)
    E = learn.min_energy(theta, pr, scale)
    E.backward()
    C = learned.cost_volume_f32(L, R, D, 2 * (D - 1), 1.0, 0.5, 20.0, scale)
    ref = oracle.solve(C, 8 * 256, 1023 * 256, 1)
    assert float(E) == ref["flow"] / scale
    sa, sb, st = learned.cost_grad_sums(L, R, D, 2 * (D - 1), 1.0, 0.5, 20.0, ref["labels"])
    _, J, _ = learned.energy_adjoint(ref["labels"], D, 1)
    assert theta.grad.tolist() == [sa, sb / 2, st, J]


@pytest.mark.gpu
def test_finite_differences_bracket_the_gradient(gc):
    """Steps of 1/256 in lambda, w1 and tau (2/256 in w2) move the integer
    costs by exact integers; concavity brackets the analytic gradient."""
    from paper_1803_01516_gb300 import learn
    wl = synth.TINY
    L, R, _ = _pair(wl, 1)
    p = gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=0, lam=0, inhibit=1023 * 256)
    pr = learn.problem(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), p)
    base = np.array([1.0, 1.0, 25.0, 8.0])
    theta = torch.tensor(base, requires_grad=True)
    learn.min_energy(theta, pr).backward()
    g = theta.grad.numpy()
    for k, step in ((0, 1 / 256), (1, 2 / 256), (2, 1 / 256), (3, 1 / 256)):
        e = {}
        for d in (-1, 0, 1):
            t = base.copy()
            t[k] += d * step
            e[d] = float(learn.min_energy(torch.tensor(t), pr))
        assert (e[1] - e[0]) / step <= g[k] + 1e-9
        assert g[k] <= (e[0] - e[-1]) / step + 1e-9


@pytest.mark.gpu
def test_hinge_loss_descends(gc):
    """A few Adam steps on (w1, w2, tau, lambda) against the synthetic
    ground truth lower the structured hinge loss."""
    from paper_1803_01516_gb300 import learn
    from paper_1803_01516_gb300.metrics import gt_depth
    wl = synth.TINY
    probs = []
    for i in range(2):
        L, R, dR = _pair(wl, i)
        p = gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=0, lam=0, inhibit=1023 * 256)
        gt = torch.from_numpy(gt_depth(dR, wl.D, 2 * (wl.D - 1))).int().cuda()
        probs.append((learn.problem(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), p), gt))
    theta = torch.tensor([1.0, 1.0, 30.0, 8.0], dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([theta], lr=0.5)
    losses = []
    for _ in range(6):
        opt.zero_grad()
        loss = sum(learn.hinge_loss(theta, pr, gt) for pr, gt in probs)
        assert float(loss) >= 0
        loss.backward()
        opt.step()
        with torch.no_grad():
            theta.clamp_(min=0.0)
        losses.append(float(loss))
    assert min(losses[1:]) < losses[0]

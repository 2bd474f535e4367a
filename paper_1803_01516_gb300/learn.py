"""Differentiating the exact minimum energy (torch.autograd on top of the C ABI).

E*(theta) = min_X E(X; theta) with the learned data term
    C[v][l] = rint(scale * min(w1 |dI| + w2 |d dxI|, tau))       (int32)
and the interaction h~ of §3 with lambda_int = rint(scale * lam) and a fixed
inhibit.  E* is concave and piecewise linear in (costs, lambda, inhibit); its
gradient where the minimiser X* is unique is
    dE*/dC = one-hot(X*),  dE*/dlambda = sum |X_u - X_v|,
and through the cost (quantiser taken as the identity)
    dE*/dw1 = sum |dI| [c < tau],  dE*/dw2 = sum |d dxI| [c < tau],
    dE*/dtau = sum [c >= tau]        (all at v, X*_v),
returned in cost units (energy / scale).  Forward = the four C-ABI calls of the
exact solve; backward = gs_cost_volume_f32_backward + gs_energy_backward.

The forward never waits for the device: the energy comes back as a 0-d tensor
on the problem's device and the solve's status is folded into the problem's
device error word; the backward (or ``_Problem.check()``) reads it and raises
on a failed solve.  Gradients are returned on theta's device.

``hinge_loss`` is the structured hinge loss used to learn theta from a
ground-truth labeling X_gt (not in the paper, which tunes h~1 by grid search):
    loss = E(X_gt; theta) - min_X [E(X; theta) - Hamming(X, X_gt)]   (>= 0),
the inner minimum taken exactly with the loss-augmented cost (scale added to
the ground-truth label's cost, a constant shift of -Hamming).
"""
from __future__ import annotations

import torch

from . import gazecut as gc


class _Problem:
    """Device buffers for one stereo pair and parameter shape."""

    def __init__(self, L: torch.Tensor, R: torch.Tensor, p: gc.Params, o: gc.SolveOpts):
        self.L, self.R, self.p, self.o = L, R, p, o
        self.buf = gc.Buffers(p, o, device=L.device)
        self.counts = torch.zeros(2, dtype=torch.int64, device=L.device)
        self.sums = torch.zeros(3, dtype=torch.int64, device=L.device)
        self.energy = torch.zeros(1, dtype=torch.int64, device=L.device)
        self.err = torch.zeros(1, dtype=torch.int32, device=L.device)   # first failed status

    def note_status(self):
        """Fold the last solve's device status into the error word (no sync)."""
        self.err.copy_(torch.where(self.err != gc.GS_OK, self.err, self.buf.status))

    def check(self):
        """Raise if any solve on this problem failed (reads the device word)."""
        e = int(self.err.item())
        if e != gc.GS_OK:
            raise RuntimeError(f"solve failed: {gc.STATUS_NAMES.get(e, e)}")


def _int_params(p: gc.Params, lam: float, scale: float) -> gc.Params:
    return gc.Params(w=p.w, h=p.h, D=p.D, tau=0, lam=int(round(scale * lam)), inhibit=p.inhibit,
                     vertical_inhibit=p.vertical_inhibit, dis0=p.dis0)


def _theta(theta: torch.Tensor):
    w1, w2, tau, lam = (float(x) for x in theta.detach().cpu().tolist())
    return max(w1, 0.0), max(w2, 0.0), max(tau, 0.0), max(lam, 0.0)


def _grads(pr: _Problem, w1, w2, tau, labels, pi: gc.Params) -> torch.Tensor:
    gc.gs_cost_volume_f32_backward(pr.L, pr.R, pi, w1, w2, tau, labels, pr.sums)
    gc.gs_energy_backward(labels, pi, 1.0, None, pr.counts)
    s = pr.sums.double()
    return torch.stack([s[0], s[1] / 2, s[2], pr.counts[0].double()])


class MinEnergy(torch.autograd.Function):
    """E*(theta) / scale for one pair; theta = (w1, w2, tau, lam) float tensor."""

    @staticmethod
    def forward(ctx, theta, pr: _Problem, scale: float, aug_labels):
        w1, w2, tau, lam = _theta(theta)
        pi = _int_params(pr.p, lam, scale)
        b = pr.buf
        gc.gs_stereo_cost_volume_f32(pr.L, pr.R, pi, w1, w2, tau, scale, b.cost)
        if aug_labels is not None:
            gc.gs_cost_add_at_labels(b.cost, aug_labels, pi, int(round(scale)))
        gc.gs_build_graph(b.cost, pi, b.graph, b.status)
        gc.gs_maxflow_solve(b.graph, pi, pr.o, b.work, b.status)
        gc.gs_extract_labels(b.graph, pi, pr.o, b.work, b.labels, b.flow, b.status)
        pr.note_status()
        labels = b.labels.clone()
        g = _grads(pr, w1, w2, tau, labels, pi)
        ctx.save_for_backward(g)
        ctx.labels = labels
        ctx.pr = pr
        ctx.theta_to = (theta.device, theta.dtype)
        e = b.flow.double() / scale
        if aug_labels is not None:
            e = e - labels.numel()          # undo the constant shift of the augmentation
        return e.reshape(())

    @staticmethod
    def backward(ctx, gE):
        (g,) = ctx.saved_tensors
        ctx.pr.check()
        return (gE * g).to(*ctx.theta_to), None, None, None


class EnergyAt(torch.autograd.Function):
    """E(X; theta) / scale at fixed labels X (int32 [h, n_g] on the device)."""

    @staticmethod
    def forward(ctx, theta, pr: _Problem, scale: float, labels):
        w1, w2, tau, lam = _theta(theta)
        pi = _int_params(pr.p, lam, scale)
        gc.gs_stereo_cost_volume_f32(pr.L, pr.R, pi, w1, w2, tau, scale, pr.buf.cost)
        gc.gs_energy(pr.buf.cost, labels, pi, pr.energy)
        g = _grads(pr, w1, w2, tau, labels, pi)
        ctx.save_for_backward(g)
        ctx.theta_to = (theta.device, theta.dtype)
        return (pr.energy.double() / scale).reshape(())

    @staticmethod
    def backward(ctx, gE):
        (g,) = ctx.saved_tensors
        return (gE * g).to(*ctx.theta_to), None, None, None


def problem(L, R, p: gc.Params, o: gc.SolveOpts | None = None) -> _Problem:
    return _Problem(L, R, p, o or gc.SolveOpts())


def min_energy(theta: torch.Tensor, pr: _Problem, scale: float = 256.0) -> torch.Tensor:
    return MinEnergy.apply(theta, pr, scale, None)


def hinge_loss(theta: torch.Tensor, pr: _Problem, gt: torch.Tensor, scale: float = 256.0):
    """E(X_gt) - min_X [E(X) - Hamming(X, X_gt)]; gt int32 [h, n_g] on the device."""
    return EnergyAt.apply(theta, pr, scale, gt) - MinEnergy.apply(theta, pr, scale, gt)


def labels_at(theta, pr: _Problem, scale: float = 256.0) -> torch.Tensor:
    """The exact minimiser X*(theta) (int32 [h, n_g] on the device), no gradient."""
    with torch.no_grad():
        MinEnergy.apply(theta.detach(), pr, scale, None)
    return pr.buf.labels.clone()


def fit(theta0, problems, gts, steps: int = 200, lr: float = 0.1, scale: float = 256.0,
        log=None):
    """Learn theta = (w1, w2, tau, lambda) by Adam on the mean structured hinge
    loss over the problems (ground-truth labelings gts, int32 [h, n_g] on the
    device), projecting theta to >= 0 after every step.  Returns (theta,
    per-step mean losses).  One host read per step (the loss value)."""
    theta = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([theta], lr=lr)
    losses = []
    for it in range(steps):
        opt.zero_grad()
        loss = sum(hinge_loss(theta, pr, gt, scale) for pr, gt in zip(problems, gts)) / len(problems)
        loss.backward()
        opt.step()
        with torch.no_grad():
            theta.clamp_(min=0.0)
        losses.append(float(loss))
        if log is not None:
            log(it, losses[-1], theta.detach().tolist())
    for pr in problems:
        pr.check()
    return theta.detach(), losses

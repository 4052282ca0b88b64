"""Tensor completion through the masked TT evaluation (the completion
experiment of Sec. 4.2.2, on the fixed-rank TT manifold's coordinates).

Given observed entries m_e = M(i_e) of a tensor at row-major linear indices
i_e, the cores are initialised by a fixed-rank TT-URV sweep of the zero-filled
observations scaled by the inverse sampling rate, then fitted to the loss
f = 1/2 sum_e (x(i_e) - m_e)^2 by full-batch gradient descent: x and the core
gradients come from the library's masked evaluation and its backward
(interfaces recomputed per entry, one plan of the observation set reused
by every call), and each step length is found by Armijo
backtracking starting from twice the previous one, so the loss never
increases.  The paper's own solver (Riemannian gradient with a TT retraction)
is not reproduced; only its observation operator P_Omega and the TT-UTV
initialisation are.
"""
from __future__ import annotations

import math

import torch

from . import EvalPlan, tt_utv


def complete(values, idx, shape, ranks, p_obs=None, steps=200, c1=1e-4, alpha0=1.0,
             min_alpha=1e-12, precision="fp32", stream=None):
    """Fit TT cores of the given ranks to observed entries.

    values  device float32 [n]: observed entries m_e;
    idx     device int64 [n]: their row-major linear indices in `shape`;
    ranks   r_1 .. r_{d-1} of the TT;
    p_obs   sampling rate of the initialisation's rescaling (default n / prod(shape)).
    Returns (cores, losses): losses[0] is the initial loss, losses[t] the loss
    after step t; the loop stops early if no step length down to `min_alpha`
    decreases the loss.
    """
    if values.dtype != torch.float32 or idx.dtype != torch.int64:
        raise TypeError("values must be float32 and idx int64")
    if not (values.is_cuda and idx.is_cuda) or values.numel() != idx.numel():
        raise ValueError("values and idx must be device vectors of one length")
    n_total = math.prod(shape)
    if p_obs is None:
        p_obs = idx.numel() / n_total
    # initialisation: TT-URV (fixed ranks) of P_Omega(M) / p_obs
    z = torch.zeros(n_total, dtype=torch.float32, device=values.device)
    z[idx] = values / p_obs
    cores = tt_utv(z.view(*shape), ranks=list(ranks), variant="URV", precision=precision,
                   stream=stream).cores
    del z

    # one plan for the fixed observation set: every evaluation and gradient reuses it
    plan = EvalPlan(shape, [1, *ranks, 1], idx, stream)

    def loss_of(cs):
        r = plan.at(cs, stream) - values
        return r, 0.5 * float(torch.dot(r, r))

    r, loss = loss_of(cores)
    losses = [loss]
    alpha = alpha0
    for _ in range(steps):
        grads = plan.backward(cores, r, stream)
        gn2 = float(sum(torch.dot(g.reshape(-1), g.reshape(-1)) for g in grads))
        if gn2 == 0.0:
            break
        alpha *= 2.0
        while True:
            trial = [c - alpha * g for c, g in zip(cores, grads)]
            rt, lt = loss_of(trial)
            if lt <= loss - c1 * alpha * gn2:
                break
            alpha *= 0.5
            if alpha < min_alpha:
                return cores, losses
        cores, r, loss = trial, rt, lt
        losses.append(loss)
    return cores, losses

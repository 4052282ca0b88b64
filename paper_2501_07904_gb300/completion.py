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
increases (complete()).

rgrad() is the paper's own solver: Riemannian gradient descent on the
manifold of TT tensors of fixed ranks.  Each iteration projects the residual
P_Omega(X_k - M) onto the tangent space at X_k (tt_tangent_project: one
two-frame masked backward and an FP64 gauge), evaluates that Riemannian
gradient xi on the observed entries (through a second plan at ranks 2r, one
masked evaluation of the block TT of xi, when 2r fits the plan's limit of 64;
else tt_tangent_eval, one forward pass per core at the iterate's own ranks),
takes the exact line-search step
alpha_k = <P_Omega xi, P_Omega(X_k - M)> / <P_Omega xi, P_Omega xi>,
forms X_k - alpha_k xi in full (a rank-2r block TT contracted by tt_full) and
retracts it with a fixed-rank TT-URV, TT-ULV or TT-SVD sweep of the library.
The other orthogonal frame of the new point comes from tt_orthogonalize
(Cholesky-QR2 of its cores' unfoldings, no pass over the full tensor).
"""
from __future__ import annotations

import math

import torch

from . import EvalPlan, tt_full, tt_orthogonalize, tt_svd, tt_utv


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


def sketch_widths(ranks):
    """(l_full, oversample) of the retraction sweeps: the iterate X - alpha xi
    has TT-ranks at most 2 r_k, so every unfolding whose basis side exceeds
    l_full = 2 max(r) + 16 is sketched with l = r_k + max(r) + 16 >= 2 r_k + 16
    columns, which hold its whole range (no range miss: TT-SVD stays exact)."""
    rmax = max(ranks)
    return 2 * rmax + 16, rmax + 16


def _retract(full, ranks, method, precision, stream):
    """Fixed-rank decomposition of the full tensor: (cores, "left"|"right")."""
    l_full, p = sketch_widths(ranks)
    if method == "SVD":
        res = tt_svd(full, ranks=list(ranks), precision=precision, stream=stream, l_full=l_full,
                     oversample=p)
        return res.cores, res.orth
    if method not in ("URV", "ULV"):
        raise ValueError("retraction must be URV, ULV or SVD")
    res = tt_utv(full, ranks=list(ranks), variant=method, precision=precision, stream=stream,
                 l_full=l_full, oversample=p)
    return res.cores, res.orth


def _other_frame(cores, orth, stream):
    """The opposite orthogonal frame of the same tensor (Cholesky-QR2 of the
    cores' unfoldings)."""
    return tt_orthogonalize(cores, "left" if orth == "right" else "right", stream)


def tangent_block_cores(U, V, dU, alpha=None):
    """Cores (ranks 2 r_k) of the tangent vector xi = sum_k U_<k dU_k V_>k,
    or of X - alpha xi (X = U_1 .. U_d) when alpha is given."""
    d = len(U)
    c = 1.0 if alpha is None else -alpha
    if d == 1:
        return [dU[0] if alpha is None else U[0] - alpha * dU[0]]
    out = []
    for k in range(d):
        if k == 0:
            out.append(torch.cat([c * dU[0], U[0]], dim=2))
        elif k == d - 1:
            last = c * dU[k] if alpha is None else U[k] + c * dU[k]
            out.append(torch.cat([V[k], last], dim=0))
        else:
            top = torch.cat([V[k], V[k].new_zeros(V[k].shape[0], U[k].shape[1], U[k].shape[2])],
                            dim=2)
            out.append(torch.cat([top, torch.cat([c * dU[k], U[k]], dim=2)], dim=0))
    return [g.contiguous() for g in out]


def rgrad(values, idx, shape, ranks, steps=40, retraction="URV", p_obs=None,
          precision="fp32", stream=None, callback=None):
    """Riemannian gradient completion of Sec. 4.2.2.

    values  device float32 [n]: observed entries m_e;
    idx     device int64 [n]: their row-major linear indices in `shape`;
    ranks   r_1 .. r_{d-1} (each at most 64, the masked-evaluation plan's limit);
    retraction  "URV" (TT-URV, right-to-left), "ULV" (TT-ULV, left-to-right)
            or "SVD" (TT-SVD), each at the fixed ranks;
    p_obs   sampling rate of the spectral initialisation (default n / prod(shape)).
    The initial point is the retraction of P_Omega(M) / p_obs.  Returns
    (cores, losses, alphas): losses[t] = 1/2 ||P_Omega(X_t - M)||^2 for
    t = 0 .. steps, alphas[t] the step of iteration t.  callback(t, cores) is
    called for every iterate (t = 0 .. steps).
    """
    if values.dtype != torch.float32 or idx.dtype != torch.int64:
        raise TypeError("values must be float32 and idx int64")
    if not (values.is_cuda and idx.is_cuda) or values.numel() != idx.numel():
        raise ValueError("values and idx must be device vectors of one length")
    ranks = [int(r) for r in ranks]
    if len(ranks) != len(shape) - 1 or any(r < 1 or r > 64 for r in ranks):
        raise ValueError("need d - 1 ranks in [1, 64]")
    n_total = math.prod(shape)
    if p_obs is None:
        p_obs = idx.numel() / n_total
    z0 = torch.zeros(n_total, dtype=torch.float32, device=values.device)
    z0[idx] = values / p_obs
    X, orth = _retract(z0.view(*shape), ranks, retraction, precision, stream)
    del z0
    plan = EvalPlan(shape, [1, *ranks, 1], idx, stream)
    # P_Omega xi: one evaluation of xi's rank-2r block TT when 2r fits a plan
    # (faster than d passes), else d passes at the iterate's ranks
    plan2 = EvalPlan(shape, [1, *[2 * r for r in ranks], 1], idx, stream) \
        if 2 * max(ranks) <= 64 else None
    # losses and steps stay on the device (read once at the end): the loop's
    # only host synchronizations are the retraction sweep's rank reads
    losses, alphas = [], []
    for t in range(steps + 1):
        if callback is not None:
            callback(t, X)
        z = plan.at(X, stream) - values
        losses.append(0.5 * torch.dot(z, z))
        if t == steps:
            break
        other = _other_frame(X, orth, stream)
        U, V = (other, X) if orth == "right" else (X, other)
        dU = plan.tangent_project(U, V, z, stream)
        xi = plan2.at(tangent_block_cores(U, V, dU), stream) if plan2 is not None \
            else plan.tangent_eval(U, V, dU, stream)
        den = torch.dot(xi, xi)
        alpha = torch.where(den > 0, torch.dot(xi, z) / torch.where(den > 0, den, 1.0),
                            torch.zeros_like(den))
        alphas.append(alpha)
        full = tt_full(tangent_block_cores(U, V, dU, alpha), stream)
        X, orth = _retract(full, ranks, retraction, precision, stream)
        del full
    plan.close(stream)
    if plan2 is not None:
        plan2.close(stream)
    losses = [float(v) for v in torch.stack(losses).double().cpu()]
    alphas = [float(v) for v in torch.stack(alphas).double().cpu()] if alphas else []
    return X, losses, alphas

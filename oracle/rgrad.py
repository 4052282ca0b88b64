"""Riemannian gradient tensor completion with a TT-UTV retraction, in plain
FP64 (test infrastructure only).

Sec. 4.2.2 (MRI data completion) of arXiv 2501.07904 recovers a tensor M
from the entries on an index set Omega by Riemannian gradient descent on the
manifold of TT tensors of fixed ranks (1, r_1, ..., r_{d-1}, 1), minimising
f(X) = 1/2 ||P_Omega(X - M)||_F^2:

* the Riemannian gradient at X_k is the projection of the Euclidean one onto
  the tangent space, RG(X_k) = P_T(P_Omega(X_k - M));
* the step is the exact minimiser along -RG of the quadratic f,
  alpha_k = <P_Omega RG, P_Omega(X_k - M)> / <P_Omega RG, P_Omega RG>;
* X_hat = X_k - alpha_k RG is retracted to the manifold by a TT-UTV (or
  TT-SVD) of the full tensor X_hat at the fixed ranks;
* X_0 is the spectral initialisation: the same decomposition of P_Omega(M)/p,
  p = |Omega| / prod(I_k).

The tangent space at X (written in the left-orthogonal cores U_1..U_{d-1},
U_d and the right-orthogonal cores V_1, V_2..V_d of one tensor) holds the
sums xi = sum_k U_1..U_{k-1} dU_k V_{k+1}..V_d with the gauge
unfold_L(U_k)^T unfold_L(dU_k) = 0 for k < d, and the orthogonal projection
of a tensor Z onto it has
  Y_k = U_{<k}^T Z_(k) V_{>k}^T  (the contraction of Z with every core but k),
  dU_k = Y_k - U_k (unfold_L(U_k)^T unfold_L(Y_k))   (k < d),  dU_d = Y_d.
Here this is formed with dense contractions of the full tensor Z.
"""
from __future__ import annotations

import numpy as np

from . import tt as ott
from .linalg import householder_qr


def _left_unfold(g):
    return g.reshape(g.shape[0] * g.shape[1], g.shape[2])


def left_orthogonal(cores):
    """The same TT with cores 1..d-1 left-orthogonal (Householder QR sweep
    left to right, the triangular factor pushed into the next core)."""
    cores = [np.array(c, dtype=np.float64) for c in cores]
    for k in range(len(cores) - 1):
        r0, n, r1 = cores[k].shape
        Q, R, _ = householder_qr(_left_unfold(cores[k]))
        q = Q.shape[1]
        cores[k] = Q.reshape(r0, n, q)
        cores[k + 1] = np.einsum("ab,bjc->ajc", R, cores[k + 1])
    return cores


def right_orthogonal(cores):
    """The same TT with cores 2..d right-orthogonal (QR of the transposed
    right unfoldings, right to left)."""
    cores = [np.array(c, dtype=np.float64) for c in cores]
    for k in range(len(cores) - 1, 0, -1):
        r0, n, r1 = cores[k].shape
        Q, R, _ = householder_qr(cores[k].reshape(r0, n * r1).T)
        q = Q.shape[1]
        cores[k] = Q.T.reshape(q, n, r1)
        cores[k - 1] = np.einsum("ajb,cb->ajc", cores[k - 1], R)
    return cores


def _left_interface(U, k):
    """U_1..U_{k-1} as a matrix (I_1..I_{k-1}) x r_{k-1} (k = 0: [[1]])."""
    L = np.ones((1, 1))
    for j in range(k):
        g = U[j]
        L = (L @ g.reshape(g.shape[0], -1)).reshape(-1, g.shape[2])
    return L


def _right_interface(V, k):
    """V_{k+1}..V_d as a matrix r_k x (I_{k+1}..I_d) (k = d-1: [[1]])."""
    R = np.ones((1, 1))
    for j in range(len(V) - 1, k, -1):
        g = V[j]
        R = (g.reshape(-1, g.shape[2]) @ R).reshape(g.shape[0], -1)
    return R


def tangent_project(U, V, Z):
    """dU_1..dU_d of the projection of the full tensor Z onto the tangent
    space at the TT whose left-orthogonal cores are U and right-orthogonal
    cores are V (both of the same tensor)."""
    d = len(U)
    dims = [g.shape[1] for g in U]
    Z = np.asarray(Z, dtype=np.float64)
    dU = []
    for k in range(d):
        L = _left_interface(U, k)          # (I_<k) x r_{k-1}
        R = _right_interface(V, k)         # r_k x (I_>k)
        nl, nr = L.shape[0], R.shape[1]
        Zk = Z.reshape(nl, dims[k], nr)
        Y = np.einsum("la,lir,br->aib", L, Zk, R)
        if k < d - 1:
            Ul = _left_unfold(U[k])
            Yl = _left_unfold(Y)
            Y = (Yl - Ul @ (Ul.T @ Yl)).reshape(Y.shape)
        dU.append(Y)
    return dU


def mixed_eval_grad(left, right, lin_idx, gout):
    """Y_k[:, i, :] = sum_{e: i_k(e) = i} gout_e (L_1[i_1]..L_{k-1}[i_{k-1}])^T
    (R_{k+1}[i_{k+1}]..R_d[i_d])^T for every k: the core gradients of
    sum_e gout_e x(i_e) with the interfaces left of core k taken from the
    cores `left` and those right of it from `right` (the projection's Y_k on
    the observed entries when left = U, right = V).  Entry by entry."""
    d = len(left)
    dims = [g.shape[1] for g in left]
    multi = np.unravel_index(np.asarray(lin_idx, dtype=np.int64), dims)
    out = [np.zeros(g.shape) for g in left]
    for e in range(len(lin_idx)):
        i = [int(m[e]) for m in multi]
        for k in range(d):
            lv = np.ones(1)
            for j in range(k):
                lv = lv @ left[j][:, i[j], :]
            rv = np.ones(1)
            for j in range(d - 1, k, -1):
                rv = right[j][:, i[j], :] @ rv
            out[k][:, i[k], :] += gout[e] * np.outer(lv, rv)
    return out


def tangent_cores(U, V, dU, alpha=0.0, with_point=False):
    """Block TT cores (ranks 2 r_k) of xi = sum_k U_<k dU_k V_>k, or of
    X - alpha xi when with_point (X = U_1..U_d)."""
    d = len(U)
    c = -alpha if with_point else 1.0
    if d == 1:
        return [(U[0] if with_point else 0.0) + c * dU[0]]
    out = []
    for k in range(d):
        if k == 0:
            out.append(np.concatenate([c * dU[0], U[0]], axis=2))
        elif k == d - 1:
            last = c * dU[k] + (U[k] if with_point else 0.0)
            out.append(np.concatenate([V[k], last], axis=0))
        else:
            r0, n, r1 = U[k].shape
            top = np.concatenate([V[k], np.zeros((V[k].shape[0], n, r1))], axis=2)
            bot = np.concatenate([c * dU[k], U[k]], axis=2)
            out.append(np.concatenate([top, bot], axis=0))
    return out


def sketch_widths(ranks):
    """(l_full, p) of the retraction: X - alpha xi has TT-ranks at most 2 r_k,
    so a sketch of r_k + max(r) + 16 >= 2 r_k + 16 columns holds the range of
    every unfolding it is used on (basis side above 2 max(r) + 16)."""
    rmax = max(list(ranks)[1:-1])
    return 2 * rmax + 16, rmax + 16


def retract(Xhat_full, ranks, variant="URV"):
    """Fixed-rank TT-UTV (or TT-SVD with variant "SVD") of the full tensor."""
    r = list(ranks)[1:-1]
    l_full, p = sketch_widths(ranks)
    if variant == "SVD":
        res = ott.tt_svd(Xhat_full, ranks=r, l_full=l_full, p=p)
    else:
        res = ott.tt_utv(Xhat_full, ranks=r, variant=variant, l_full=l_full, p=p)
    return res["cores"]


def step_size(xi_obs, z):
    """alpha minimising ||z - alpha xi_obs||^2 (z = P_Omega(X - M) on Omega)."""
    den = float(np.dot(xi_obs, xi_obs))
    return float(np.dot(xi_obs, z)) / den if den > 0.0 else 0.0


def rgrad(values, idx, shape, ranks, steps, variant="URV", p_obs=None):
    """Riemannian gradient descent of Sec. 4.2.2.  values = M at the row-major
    linear indices idx.  Returns (cores of the last iterate, losses)."""
    shape = tuple(shape)
    ntot = int(np.prod(shape))
    values = np.asarray(values, dtype=np.float64)
    idx = np.asarray(idx, dtype=np.int64)
    if p_obs is None:
        p_obs = len(idx) / ntot
    Z0 = np.zeros(ntot)
    Z0[idx] = values / p_obs
    cores = retract(Z0.reshape(shape), ranks, variant)
    losses = []
    for _ in range(steps + 1):
        full = ott.tt_full(cores).reshape(-1)
        z = full[idx] - values
        losses.append(0.5 * float(np.dot(z, z)))
        if len(losses) == steps + 1:
            break
        U = left_orthogonal(cores)
        V = right_orthogonal(cores)
        G = np.zeros(ntot)
        G[idx] = z
        dU = tangent_project(U, V, G.reshape(shape))
        xi = ott.tt_full(tangent_cores(U, V, dU)).reshape(-1)
        alpha = step_size(xi[idx], z)
        cores = retract((full - alpha * xi).reshape(shape), ranks, variant)
    return cores, losses

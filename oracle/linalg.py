"""Dense FP64 linear algebra for the oracle (test infrastructure only).

* ``householder_qr``: Householder QR, optionally with column pivoting (the
  rank-revealing QR the paper lists as a UTV variant, Sec. 2.2).  Reflector
  sign: v = x + sign(x_1)||x|| e_1 with sign(0) = +1, so R's diagonal may be
  negative.  Pivot: largest remaining column norm, lowest index on ties.
* ``jacobi_svd``: one-sided (Hestenes) Jacobi SVD, the comparison TT-SVD's
  inner factorization.

Both are written from their textbook definitions, column by column, with no
blocking.
"""
from __future__ import annotations

import numpy as np


class NoConvergence(RuntimeError):
    pass


_ROWS = 1 << 16


def _rank1_update(R, j, tv, w, c0=None):
    """R[j:, c0:] -= outer(tv, w) (c0 = j by default), applied in row slices
    to bound temporaries."""
    m = R.shape[0]
    c0 = j if c0 is None else c0
    for r0 in range(j, m, _ROWS):
        r1 = min(m, r0 + _ROWS)
        R[r0:r1, c0:] -= np.outer(tv[r0 - j:r1 - j], w)


def householder_qr(A, pivoting=False, full_q=False):
    """Householder QR of an m x n matrix: A[:, perm] = Q R.

    Returns (Q, R, perm).  k = min(m, n) reflectors are applied.  R is k x n
    upper trapezoidal (m x n if ``full_q``); Q is m x k (m x m if ``full_q``)
    with orthonormal columns.  With ``pivoting`` the column of largest
    remaining 2-norm is moved to the front before each reflector, so
    |R[0,0]| >= |R[1,1]| >= ...
    """
    A = np.array(A, dtype=np.float64)
    m, n = A.shape
    k = min(m, n)
    R = A.copy()
    perm = np.arange(n)
    vs, taus = [], []
    for j in range(k):
        if pivoting:
            norms = np.einsum("ij,ij->j", R[j:, j:], R[j:, j:])
            p = j + int(np.argmax(norms))          # first maximum -> lowest index
            if p != j:
                R[:, [j, p]] = R[:, [p, j]]
                perm[[j, p]] = perm[[p, j]]
        x = R[j:, j].copy()
        alpha = np.sqrt(x @ x)
        if alpha == 0.0:
            vs.append(np.zeros_like(x))
            taus.append(0.0)
            continue
        s = 1.0 if x[0] >= 0.0 else -1.0
        v = x
        v[0] += s * alpha
        tau = 2.0 / (v @ v)
        w = v @ R[j:, j:]
        _rank1_update(R, j, tau * v, w)
        R[j + 1:, j] = 0.0
        R[j, j] = -s * alpha
        vs.append(v)
        taus.append(tau)
    ncols = m if full_q else k
    Q = np.zeros((m, ncols))
    Q[np.arange(ncols), np.arange(ncols)] = 1.0
    for j in range(k - 1, -1, -1):
        if taus[j] == 0.0:
            continue
        v = vs[j]
        _rank1_update(Q, j, taus[j] * v, v @ Q[j:, :], c0=0)
    if not full_q:
        R = R[:k, :]
    return Q, R, perm


def _round_robin_pairs(n):
    """Disjoint pairs of a round-robin tournament on n (even) players, n-1 rounds."""
    players = list(range(n))
    rounds = []
    for _ in range(n - 1):
        rounds.append([(players[i], players[n - 1 - i]) for i in range(n // 2)])
        players = [players[0]] + [players[-1]] + players[1:-1]
    return rounds


def jacobi_svd(A, tol=None, max_sweeps=60):
    """One-sided Jacobi SVD of an m x n matrix (Hestenes).

    Columns of U = A V are rotated pairwise until every pair is orthogonal to
    |a_i . a_j| <= tol * ||a_i|| ||a_j|| (default tol = m * machine epsilon,
    the Demmel-Veselic stopping rule).  Returns (sigma, V) with sigma sorted
    descending (length n; trailing entries may be 0) and V n x n orthogonal so
    that the columns of A V are orthogonal with norms sigma.
    """
    U = np.array(A, dtype=np.float64)
    n = U.shape[1]
    if tol is None:
        tol = max(U.shape[0], 1) * np.finfo(np.float64).eps
    # columns whose norm is at the rounding level of ||A||_F are treated as zero
    tiny2 = (np.finfo(np.float64).eps * np.sqrt(np.sum(U * U))) ** 2
    V = np.eye(n)
    if n == 1:
        return np.array([np.linalg.norm(U[:, 0])]), V
    nn = n + (n % 2)
    rounds = _round_robin_pairs(nn)
    for sweep in range(max_sweeps):
        off = 0.0
        for pairs in rounds:
            pr = np.array([(i, j) for i, j in pairs if i < n and j < n])
            if pr.size == 0:
                continue
            i, j = pr[:, 0], pr[:, 1]
            a = np.einsum("ij,ij->j", U[:, i], U[:, i])
            b = np.einsum("ij,ij->j", U[:, j], U[:, j])
            g = np.einsum("ij,ij->j", U[:, i], U[:, j])
            ab = np.sqrt(a * b)
            act = (np.minimum(a, b) > tiny2) & (np.abs(g) > tol * ab)
            if ab.size:
                live = np.minimum(a, b) > tiny2
                rel = np.where(live, np.abs(g) / np.where(live, ab, 1.0), 0.0)
                off = max(off, float(rel.max()))
            if not act.any():
                continue
            i, j, a, b, g = i[act], j[act], a[act], b[act], g[act]
            # rotation angle annihilating the (i,j) entry of U^T U
            zeta = (b - a) / (2.0 * g)
            t = np.sign(zeta) / (np.abs(zeta) + np.hypot(1.0, zeta))
            t = np.where(zeta == 0.0, 1.0, t)
            c = 1.0 / np.sqrt(1.0 + t * t)
            s = c * t
            Ui, Uj = U[:, i].copy(), U[:, j].copy()
            U[:, i] = c * Ui - s * Uj
            U[:, j] = s * Ui + c * Uj
            Vi, Vj = V[:, i].copy(), V[:, j].copy()
            V[:, i] = c * Vi - s * Vj
            V[:, j] = s * Vi + c * Vj
        if off <= tol:
            sig = np.sqrt(np.einsum("ij,ij->j", U, U))
            order = np.argsort(-sig, kind="stable")
            return sig[order], V[:, order]
    raise NoConvergence(f"one-sided Jacobi did not converge in {max_sweeps} sweeps")

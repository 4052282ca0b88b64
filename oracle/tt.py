"""TT-UTV, TT-SVD and masked TT evaluation in plain FP64 (test infrastructure only).

Notation follows the paper (arXiv 2501.07904): A in R^{I_1 x ... x I_d}, TT
cores G^(k) in R^{r_{k-1} x I_k x r_k} with r_0 = r_d = 1 (Eq. TT), unfoldings
A_k (Def. 2.1), ULV / URV decompositions (Eqs. ulv, urv), Algorithm 1/2
(TT-ULV, left-to-right) and Algorithm 3 (TT-URV, right-to-left) with the
prescribed-accuracy rule of Sec. 3.1 (smallest r_k with ||E||_F <= eps_k,
eps_k = w_k eps ||A||_F).

Storage is row-major (C order): the paper's reverse-lexicographic ivec only
permutes the rows and columns of every unfolding, which leaves singular
values, ranks, truncation errors and the represented tensor unchanged.

Readings where the paper is silent:

* inner UTV (the paper names the family, Sec. 2.2): a range step (identity
  when the basis side has <= l_full columns, else a Rademacher sketch
  Y = X^T Omega, W = Householder-QR(Y).Q, B = X W), then Stewart's pivoted QLP
  of B (pivoted QR of B, pivoted QR of R_1^T, L = R_2^T, Z = Pi_1 Q_2), then a
  QR of L for the URV form (T upper).  Truncation error for rank r:
  tail(r) = mu^2 + sum_{j>r} ||L(:,j)||^2, mu^2 = ||X - B W^T||_F^2.
* TT-SVD: the same range step (no random sketch) and Householder QR, then
  one-sided Jacobi on R_1.
* rank rule: smallest r >= 1 with tail(r) <= delta^2 (<= passes); fixed ranks
  are clamped to the size of the factored matrix.
"""
from __future__ import annotations

import math

import numpy as np

from .linalg import householder_qr, jacobi_svd
from .philox import rademacher

L_FULL = 256
OVERSAMPLE = 16


def _roundup(x, m):
    return ((x + m - 1) // m) * m


def sketch_size(n_basis, n_other, r_prev, p=OVERSAMPLE, fixed_r=None):
    """Number of sketch columns l (reading S9): r+p for a fixed rank, else
    roundup16(max(2 r_prev, r_prev + p, 32)); never more than either side."""
    if fixed_r is not None:
        l = fixed_r + p
    else:
        l = _roundup(max(2 * r_prev, r_prev + p, 32), 16)
    return int(min(l, n_basis, n_other))


def range_step(X, l, seed, step, q=0):
    """Range of the basis side of X (N_o x N_b): returns (W, B, mu2).

    l >= N_o uses Omega = I (the sketch then spans the whole row space, and
    power iterations change nothing); otherwise Omega is the Philox
    Rademacher matrix of this step and Y = X^T Omega is followed by q power
    (subspace) iterations Y <- X^T X Q, Q an orthonormal basis of the previous
    Y, so that span(Y) = span((X^T X)^q X^T Omega) with the weak directions
    damped by the squared singular values (the randomized range finder the
    paper's randUTV reference builds on).
    """
    n_o, n_b = X.shape
    if l >= n_o:
        Y = X.T.copy()
    else:
        Y = X.T @ rademacher(n_o, l, seed, step)
        for _ in range(q):
            Q, _, _ = householder_qr(Y)
            Y = X.T @ (X @ Q)
    W, _, _ = householder_qr(Y)
    B = X @ W
    E = X - B @ W.T
    mu2 = float(np.sum(E * E))
    return W, B, mu2


def qlp(B):
    """Pivoted QLP of B (N_o x N'): B = (Q_1 Pi_2) L (Pi_1 Q_2)^T (Stewart, cited in Sec. 2.2).

    Returns (Z, L, Q1P2) with Z = Pi_1 Q_2 (N' x N' orthogonal) and L lower
    trapezoidal (k x N', k = min(N_o, N')).
    """
    Q1, R1, p1 = householder_qr(B, pivoting=True)
    Q2, R2, p2 = householder_qr(R1.T, pivoting=True, full_q=True)
    L = R2.T                                   # k x N', L[:, j] = R2[j, :]
    Z = np.empty_like(Q2)
    Z[p1, :] = Q2
    Q1P2 = Q1[:, p2]                           # (Q_1 Pi_2)[:, j] = Q_1[:, p2[j]]
    return Z, L, Q1P2


def utv_of(X, variant="URV"):
    """Full rank-revealing UTV of a matrix via pivoted QLP (the exact path, no sketch).

    URV: X = U T V^T with T upper trapezoidal (QR of L, T = R_3).
    ULV: computed as the URV of X^T, transposed, so T is lower.
    Returns (U, T, V).
    """
    if variant == "ULV":
        U, T, V = utv_of(X.T, "URV")
        return V, T.T, U
    Z, L, Q1P2 = qlp(X)
    Q3, R3, _ = householder_qr(L)
    return Q1P2 @ Q3, R3, Z


def qlp_tails(L):
    """tail_B(r) = sum_{j>=r} ||L(:,j)||^2 for r = 0..N' (length N'+1)."""
    c = np.sum(L * L, axis=0)
    return np.concatenate([np.cumsum(c[::-1])[::-1], [0.0]])


USVP_ITERS = 8


def usv_plus(X, delta2, r_fixed, r_max, q=USVP_ITERS, mu2=0.0):
    """USV-plus-style deflation (the rank-revealing decomposition the paper
    runs as TT-ULV's inner factor in Sec. 4, with its stopping rule adapted to
    fixed ranks and to Alg. 2's accuracy rule): the right singular vectors of
    X (N_o x N_b, basis on the column side) are estimated one at a time, each
    by q power iterations on the deflated matrix D = X (I - V V^T).

    Per vector: the start is D^T D e_j for the column j of D of largest norm
    (lowest index on ties); q times v <- D^T D v / ||D^T D v||; v is
    re-orthogonalized twice against V and appended.  tail(i) = mu2 +
    ||X - X V_i V_i^T||^2 (summed directly) is the error of keeping the first
    i vectors.  Stops at the fixed rank (clamped to r_max), else at the
    first i >= 1 with tail(i) <= delta2, else at r_max.  When D vanishes
    before a fixed rank is reached, unit vectors orthogonalized against V
    (twice) complete it.  Returns (V (N_b x r), tails [tail(0) .. tail(r)]).
    """
    X = np.asarray(X, dtype=np.float64)
    n_o, n_b = X.shape
    x2 = float(np.sum(X * X))
    target = None if r_fixed is None else max(1, min(int(r_fixed), r_max))
    V = np.zeros((n_b, 0))
    tails = [mu2 + x2]
    while V.shape[1] < r_max:
        i = V.shape[1]
        if target is not None and i >= target:
            break
        if target is None and i >= 1 and tails[-1] <= delta2:
            break
        D = X - (X @ V) @ V.T
        cn = np.einsum("ij,ij->j", D, D)
        j = int(np.argmax(cn))
        v = D.T @ D[:, j] if cn[j] > 0.0 else np.zeros(n_b)
        nv = float(np.linalg.norm(v))
        if nv > 0.0:
            v = v / nv
            for _ in range(q):
                w = D.T @ (D @ v)
                nw = float(np.linalg.norm(w))
                if nw == 0.0:
                    break
                v = w / nw
            for _ in range(2):
                v = v - V @ (V.T @ v)
            nv = float(np.linalg.norm(v))
        if nv <= 0.0 or not np.isfinite(nv):
            if target is None:
                break                          # D = 0: nothing left to capture
            # complete the fixed rank with unit vectors
            for c in range(n_b):
                e = np.zeros(n_b)
                e[c] = 1.0
                for _ in range(2):
                    e = e - V @ (V.T @ e)
                ne = float(np.linalg.norm(e))
                if ne > 0.5:
                    v, nv = e / ne, 1.0
                    break
            else:
                break
        else:
            v = v / nv
        V = np.concatenate([V, v[:, None]], axis=1)
        E = X - (X @ V) @ V.T
        tails.append(mu2 + float(np.sum(E * E)))
    return V, np.asarray(tails)


LURV_ITERS = 8


def givens(a, b):
    """(c, s) with [c s; -s c] [a; b] = [rho; 0], rho = hypot(a, b) >= 0
    ((1, 0) when a = b = 0)."""
    rho = float(np.hypot(a, b))
    if rho == 0.0:
        return 1.0, 0.0
    return a / rho, b / rho


def lurv(X, delta2, r_fixed, r_max, q=LURV_ITERS, mu2=0.0, return_r=False):
    """Low-rank revealing URV with Givens rotations, warm-started from a
    pivoted QR (the family of Fierro and Hansen's low-rank UTV algorithms that
    the paper's TT-URV experiments run as the inner factor, Sec. 4):
    X (N_o x N_b, basis on the column side) = Q R V^T, started from the
    column-pivoted QR X Pi = Q R (V = Pi).  For i = 0, 1, ...:

    * the trailing block T = R[i:, i:] gets its dominant right singular
      vector estimated: start T^T T e_j for the column j of T of largest norm
      (lowest index on ties), then q power iterations v <- T^T T v / ||.||;
    * v is rotated onto the first coordinate of the block by Givens rotations
      on columns (j-1, j), j from the last down to i+1 (applied to R and V);
      each leaves a fill at R[j, j-1], removed at once by a Givens rotation on
      rows (j-1, j), which keeps R upper trapezoidal;
    * the error of keeping i + 1 basis vectors is mu2 + ||R[:, i+1:]||_F^2.

    Stops at the fixed rank (clamped to r_max) or at the first i >= 1 whose
    error is at most delta2.  Returns (V[:, :r], tails [tail(0) .. tail(r)])
    with tail(0) = mu2 + ||R||^2.
    """
    X = np.asarray(X, dtype=np.float64)
    n_o, n_b = X.shape
    _, R, p1 = householder_qr(X, pivoting=True)
    R = np.array(R, dtype=np.float64)
    k = R.shape[0]
    V = np.zeros((n_b, n_b))
    V[p1, np.arange(n_b)] = 1.0
    target = None if r_fixed is None else max(1, min(int(r_fixed), r_max))
    tails = [mu2 + float(np.sum(R * R))]
    i = 0
    while i < r_max:
        if target is not None and i >= target:
            break
        if target is None and i >= 1 and tails[-1] <= delta2:
            break
        if i < k:
            T = R[i:, i:]
            cn = np.einsum("ij,ij->j", T, T)
            j0 = int(np.argmax(cn))
            v = T.T @ T[:, j0]
            nv = float(np.linalg.norm(v))
            if nv > 0.0:
                v = v / nv
                for _ in range(q):
                    w = T.T @ (T @ v)
                    nw = float(np.linalg.norm(w))
                    if nw == 0.0:
                        break
                    v = w / nw
                # rotate v onto e_1 of the block: columns (j-1, j), bottom up
                for jj in range(n_b - i - 1, 0, -1):
                    c, s_ = givens(v[jj - 1], v[jj])
                    v[jj - 1], v[jj] = c * v[jj - 1] + s_ * v[jj], 0.0
                    a, b = i + jj - 1, i + jj
                    Ra, Rb = R[:, a].copy(), R[:, b].copy()
                    R[:, a], R[:, b] = c * Ra + s_ * Rb, -s_ * Ra + c * Rb
                    Va, Vb = V[:, a].copy(), V[:, b].copy()
                    V[:, a], V[:, b] = c * Va + s_ * Vb, -s_ * Va + c * Vb
                    if b < k:  # fill at R[b, a]: rotate rows (a, b)
                        cr, sr = givens(R[a, a], R[b, a])
                        Ra, Rb = R[a, :].copy(), R[b, :].copy()
                        R[a, :], R[b, :] = cr * Ra + sr * Rb, -sr * Ra + cr * Rb
                        R[b, a] = 0.0
        i += 1
        tails.append(mu2 + float(np.sum(R[:, i:] ** 2)))
    if return_r:
        return V[:, :i], np.asarray(tails), R, V
    return V[:, :i], np.asarray(tails)


def choose_rank(tails, delta2, r_fixed, r_max):
    """Reading S3 of the rule in Sec. 3.1: smallest r >= 1 with tail(r) <= delta^2."""
    if r_fixed is not None:
        return int(max(1, min(r_fixed, r_max)))
    for r in range(1, r_max + 1):
        if tails[r] <= delta2:
            return r
    return r_max


def factor_step(X, delta2, r_fixed, r_prev, seed, step, kind="qlp",
                l_full=L_FULL, p=OVERSAMPLE, q=0, usvp_q=USVP_ITERS):
    """One truncated UTV of X (N_o x N_b, basis on the column side).

    Returns dict(r, basis (N_b x r), carry (N_o x r) = X basis, tail, l, path).
    The truncation residual E = X - carry basis^T satisfies E basis = 0, and
    ||E||_F^2 = tail (EV_1 = 0 for URV, U_1^T E = 0 for ULV: Sec. 3.1-3.2).
    """
    n_o, n_b = X.shape
    if n_b <= l_full or (kind == "svd" and n_b <= n_o):
        W, B, mu2, l, path = None, X, 0.0, n_b, "exact"
    elif kind == "svd":
        # TT-SVD takes no random sketch: the identity range (l = N_o) is exact
        l, path = n_o, "sketch"
    else:
        l = sketch_size(n_b, n_o, r_prev, p, r_fixed)
        path = "sketch"
    while True:
        if path == "sketch":
            W, B, mu2 = range_step(X, l, seed, step, q)
        if kind in ("usvp", "lurv"):
            r_max = min(B.shape[1], n_o, n_b)
            Z, tails = (usv_plus if kind == "usvp" else lurv)(B, delta2, r_fixed, r_max, usvp_q, mu2)
            r = Z.shape[1]
            if (path == "sketch" and l < min(n_b, n_o) and r_fixed is None
                    and (r > l - p or tails[r] > delta2)):
                l = min(2 * l, n_b, n_o)
                continue
            break
        if kind == "qlp":
            Z, L, _ = qlp(B)
            tails = mu2 + qlp_tails(L)
        else:
            _, R1, _ = householder_qr(B)
            sig, Z = jacobi_svd(R1)
            s2 = sig * sig
            tails = mu2 + np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])
        r_max = min(Z.shape[1], n_o, n_b)
        tails = tails[: r_max + 1]
        r = choose_rank(tails, delta2, r_fixed, r_max)
        can_grow = (path == "sketch" and kind == "qlp" and l < min(n_b, n_o)
                    and r_fixed is None)
        if can_grow and (r > l - p or tails[r] > delta2):
            l = min(2 * l, n_b, n_o)
            continue
        break
    Z1 = Z[:, :r]
    basis = Z1 if W is None else W @ Z1
    carry = B @ Z1
    return dict(r=r, basis=basis, carry=carry, tail=float(tails[r]), l=l, path=path,
                tails=tails)


def _weights(d, weights):
    if weights is None:
        return np.full(d - 1, 1.0 / math.sqrt(d - 1))
    w = np.asarray(weights, dtype=np.float64)
    assert w.shape == (d - 1,)
    return w


def tt_sweep(A, eps=None, ranks=None, variant="URV", kind="qlp", direction=None,
             weights=None, l_full=L_FULL, p=OVERSAMPLE, seed=0, q=0, usvp_q=USVP_ITERS):
    """TT decomposition by a sweep of truncated UTVs.

    variant 'URV' -> right-to-left (Alg. 3), right-orthogonal cores;
    variant 'ULV' -> left-to-right (Alg. 1/2), left-orthogonal cores;
    kind 'svd' turns either sweep into TT-SVD (direction from ``direction``).
    Exactly one of ``eps`` (prescribed accuracy, eps_k = w_k eps ||A||_F) or
    ``ranks`` (r_1..r_{d-1}) is given.
    """
    A = np.asarray(A, dtype=np.float64)
    dims = A.shape
    d = len(dims)
    assert d >= 2
    if direction is None:
        direction = "RL" if variant == "URV" else "LR"
    assert (eps is None) != (ranks is None)
    normA2 = float(np.sum(A * A))
    w = _weights(d, weights)
    cores = [None] * d
    rk = [1] * (d + 1)
    tails = [0.0] * (d - 1)          # indexed by unfolding number k-1 (k = 1..d-1)
    steps = []
    r_prev = 0

    def delta2_of(u):                # u = unfolding number 1..d-1
        if eps is None:
            return None
        return (w[u - 1] * eps) ** 2 * normA2

    def fixed_of(u):
        return None if ranks is None else int(ranks[u - 1])

    if direction == "RL":
        C = A.reshape(-1, dims[-1])
        r_next = 1
        for k in range(d, 1, -1):
            m = int(np.prod(dims[: k - 1]))
            n = dims[k - 1] * r_next
            C = C.reshape(m, n)
            u = k - 1
            st = factor_step(C, delta2_of(u) if eps is not None else 0.0, fixed_of(u), r_prev,
                             seed, k, kind, l_full, p, q, usvp_q)
            r = st["r"]
            cores[k - 1] = st["basis"].T.reshape(r, dims[k - 1], r_next)
            C = st["carry"]
            rk[k - 1] = r
            tails[u - 1] = st["tail"]
            steps.append(dict(k=k, m=m, n=n, **{x: st[x] for x in ("r", "tail", "l", "path")}))
            r_next = r
            r_prev = r
        cores[0] = C.reshape(1, dims[0], r_next)
    else:
        C = A.reshape(dims[0], -1)
        r_left = 1
        for k in range(1, d):
            m = r_left * dims[k - 1]
            n = int(np.prod(dims[k:]))
            C = C.reshape(m, n)
            u = k
            st = factor_step(C.T, delta2_of(u) if eps is not None else 0.0, fixed_of(u), r_prev,
                             seed, k, kind, l_full, p, q, usvp_q)
            r = st["r"]
            cores[k - 1] = st["basis"].reshape(r_left, dims[k - 1], r)
            C = st["carry"].T
            rk[k] = r
            tails[u - 1] = st["tail"]
            steps.append(dict(k=k, m=m, n=n, **{x: st[x] for x in ("r", "tail", "l", "path")}))
            r_left = r
            r_prev = r
        cores[d - 1] = C.reshape(r_left, dims[d - 1], 1)
    delta2 = None if eps is None else [delta2_of(u) for u in range(1, d)]
    return dict(cores=cores, ranks=rk, tails=tails, normA2=normA2, delta2=delta2, steps=steps,
                orth="right" if direction == "RL" else "left")


def tt_utv(A, eps=None, ranks=None, variant="URV", inner="qlp", **kw):
    """TT-URV (right-to-left, Alg. 3) or TT-ULV (left-to-right, Alg. 1/2).
    inner: "qlp" (pivoted QLP, the default), "usvp" (USV-plus-style
    deflation, usv_plus) or "lurv" (Givens-based low-rank URV, lurv); the
    last two take usvp_q power iterations per basis vector."""
    assert inner in ("qlp", "usvp", "lurv")
    return tt_sweep(A, eps=eps, ranks=ranks, variant=variant, kind=inner, **kw)


def tt_svd(A, eps=None, ranks=None, direction="LR", **kw):
    """TT-SVD (Oseledets), the paper's comparison method, by the same sweep."""
    variant = "ULV" if direction == "LR" else "URV"
    return tt_sweep(A, eps=eps, ranks=ranks, variant=variant, kind="svd", direction=direction, **kw)


def tt_full(cores):
    """Contract the cores into the full tensor (Eq. TT)."""
    t = cores[0].reshape(cores[0].shape[1], cores[0].shape[2])
    for g in cores[1:]:
        r0, n, r1 = g.shape
        t = (t.reshape(-1, r0) @ g.reshape(r0, n * r1)).reshape(-1, r1)
    return t.reshape([g.shape[1] for g in cores])


def rse(A, cores):
    """Relative error ||A_hat - A||_F / ||A||_F (Sec. 4)."""
    A = np.asarray(A, dtype=np.float64)
    D = tt_full(cores) - A
    return float(np.sqrt(np.sum(D * D) / np.sum(A * A)))


def tt_eval_at(cores, lin_idx):
    """x(i) = G_1[i_1] G_2[:, i_2, :] ... G_d[:, i_d] at row-major linear indices."""
    dims = [g.shape[1] for g in cores]
    multi = np.unravel_index(np.asarray(lin_idx, dtype=np.int64), dims)
    v = np.ones((len(lin_idx), 1))
    for k, g in enumerate(cores):
        v = np.einsum("na,anb->nb", v, g[:, multi[k], :])
    return v[:, 0]


def tt_eval_grad(cores, lin_idx, gout):
    """Gradient of sum_e gout_e x(i_e) with respect to every core.

    dG_k[:, i, :] = sum_{e: i_k(e) = i} gout_e (G_1[i_1]...G_{k-1}[i_{k-1}])^T
                                         (G_{k+1}[i_{k+1}]...G_d[i_d])^T.
    """
    dims = [g.shape[1] for g in cores]
    d = len(cores)
    n = len(lin_idx)
    multi = np.unravel_index(np.asarray(lin_idx, dtype=np.int64), dims)
    left = [np.ones((n, 1))]
    for k in range(d - 1):
        left.append(np.einsum("na,anb->nb", left[-1], cores[k][:, multi[k], :]))
    right = [None] * d
    right[d - 1] = np.ones((n, 1))
    for k in range(d - 1, 0, -1):
        right[k - 1] = np.einsum("anb,nb->na", cores[k][:, multi[k], :], right[k])
    grads = []
    gout = np.asarray(gout, dtype=np.float64)
    for k in range(d):
        g = np.zeros_like(cores[k])
        contrib = gout[:, None, None] * left[k][:, :, None] * right[k][:, None, :]
        gt = np.zeros((dims[k],) + (cores[k].shape[0], cores[k].shape[2]))
        np.add.at(gt, multi[k], contrib)
        g[:] = gt.transpose(1, 0, 2)
        grads.append(g)
    return grads


def tt_ulv_rl(A, eps=None, ranks=None, lhat="l11", l_full=L_FULL, p=OVERSAMPLE, seed=0, q=0):
    """TT-ULV in a right-to-left sweep (the appendix's Alg. 4): right-orthogonal cores.

    Unfolding C_k (I_1..I_{k-1} x I_k r_k) is approximated through the ULV form
    of the pivoted QLP of its range-projected matrix, C ~ U L V^T with
    U = Q_1 Pi_2, L lower trapezoidal, V = W Z; the new core is V_1^T.
    The appendix's two choices of the kept middle block:

    * lhat = "l11" (Alg. 4 as printed): carry U_1 L_11.  Its residual
      U_2 L_21 V_1^T + U_2 L_22 V_2^T is not orthogonal to V_1, so
      ||C - U_1 L_11 V_1^T||^2 = mu^2 + ||L||^2 - ||L_11||^2 and the errors of the
      sweep add in norm (the appendix's Proposition: ||A - A_hat|| <= sum eps_k);
      a prescribed accuracy uses eps_k = eps ||A||_F / (d-1).
    * lhat = "full": carry U L(:, 1:r) = U_1 L_11 + U_2 L_21 = C V_1, residual
      U_2 L_22 V_2^T orthogonal to V_1 (error mu^2 + ||L_22||^2), for which
      results like Thm 3.1 / Cor. 3.1 hold: eps_k = eps ||A||_F / sqrt(d-1).
    """
    assert lhat in ("l11", "full")
    A = np.asarray(A, dtype=np.float64)
    dims = A.shape
    d = len(dims)
    assert d >= 2 and (eps is None) != (ranks is None)
    normA2 = float(np.sum(A * A))
    if eps is None:
        delta2 = None
    elif lhat == "l11":
        delta2 = (eps / (d - 1)) ** 2 * normA2
    else:
        delta2 = eps ** 2 / (d - 1) * normA2
    cores = [None] * d
    rk = [1] * (d + 1)
    tails = [0.0] * (d - 1)
    C = A.reshape(-1, dims[-1])
    r_next, r_prev = 1, 0
    for k in range(d, 1, -1):
        m = int(np.prod(dims[: k - 1]))
        n = dims[k - 1] * r_next
        C = C.reshape(m, n)
        r_fixed = None if ranks is None else int(ranks[k - 2])
        exact = n <= l_full
        l = n if exact else sketch_size(n, m, r_prev, p, r_fixed)
        while True:
            if exact:
                W, B, mu2 = None, C, 0.0
            else:
                W, B, mu2 = range_step(C, l, seed, k, q)
            Z, L, U = qlp(B)
            kk = L.shape[0]
            if lhat == "full":
                tl = mu2 + qlp_tails(L)
            else:
                tot = float(np.sum(L * L))
                tl = np.array([mu2 + tot - float(np.sum(L[:r, :r] ** 2))
                               for r in range(Z.shape[1] + 1)])
            r_max = min(Z.shape[1], m, n)
            tl = tl[: r_max + 1]
            r = choose_rank(tl, 0.0 if delta2 is None else delta2, r_fixed, r_max)
            grow = (not exact and l < min(n, m) and r_fixed is None
                    and (r > l - p or tl[r] > delta2))
            if grow:
                l = min(2 * l, n, m)
                continue
            break
        V1 = Z[:, :r] if W is None else W @ Z[:, :r]
        rr = min(r, kk)
        carry = np.zeros((m, r))
        if lhat == "full":
            carry[:, :] = U @ L[:, :r]
        else:
            carry[:, :rr] = U[:, :rr] @ L[:rr, :rr]
        cores[k - 1] = V1.T.reshape(r, dims[k - 1], r_next)
        rk[k - 1] = r
        tails[k - 2] = float(tl[r])
        C = carry
        r_next = r_prev = r
    cores[0] = C.reshape(1, dims[0], r_next)
    return dict(cores=cores, ranks=rk, tails=tails, normA2=normA2,
                delta2=None if delta2 is None else [delta2] * (d - 1), orth="right")

"""The reorganised Givens chase that the GPU's low-rank URV factor runs,
modelled on the CPU and held to the oracle's interleaved chase (`tt.lurv`).

Per basis vector the oracle alternates a rotation of columns (c, c+1), taken
from the estimated singular vector v, and a rotation of rows (c, c+1) that
removes the fill at R(c+1, c).  The kernel instead computes (1) every column
angle from suffix norms of v, (2) applies all column rotations first, (3)
gets every row angle from the affine recurrence rho_p^2 = y_p^2 + s_p^2
rho_{p+1}^2 (y_p: row p seen through the column rotations to its right) and
(4) applies all row rotations last, zeroing what lies below the diagonal.
Left and right multiplications commute, so both orders give the same R and
V; this model checks that algebra (and the scans' index ranges) against the
oracle on square, wide (trapezoidal R), rank-deficient, fixed-rank and
adaptive cases.
"""
import numpy as np
import pytest

from oracle import tt as otc


def _schedule_model(X, delta2, r_fixed, r_max, q=otc.LURV_ITERS):
    n = X.shape[1]
    _, R0, p1 = otc.householder_qr(X, pivoting=True)
    k1 = R0.shape[0]
    R = np.zeros((n, n))
    R[:k1] = R0
    V = np.zeros((n, n))
    V[p1, np.arange(n)] = 1.0
    fixed = r_fixed is not None
    rmax = max(1, min(r_fixed, r_max) if fixed else min(r_max, n))
    tails = [float(np.sum(R * R))]
    i = 0
    while i < rmax:
        if (i >= rmax) if fixed else (i >= 1 and tails[-1] <= delta2):
            break
        T = R[i:k1, i:]
        cn = np.sum(T * T, axis=0) if i < k1 else np.zeros(0)
        if i < k1 and cn.max() > 0:
            v = T.T @ T[:, int(np.argmax(cn))]
            for _ in range(q):
                w = T.T @ (T @ v)
                if not np.any(w):
                    break
                v = w / np.linalg.norm(w)
            lv = np.zeros(n)
            lv[i:] = v
            # (1) column angles from suffix sums of squares
            suf = np.cumsum((lv ** 2)[::-1])[::-1]
            cs, sn = np.ones(n), np.zeros(n)
            for c in range(i, n - 1):
                h = np.sqrt(suf[c])
                b = lv[n - 1] if c == n - 2 else np.sqrt(suf[c + 1])
                if h > 0:
                    cs[c], sn[c] = lv[c] / h, b / h
            # (2) all column rotations, recording y_p = the new R(p, p)
            dg, y = np.diag(R).copy(), np.zeros(n)
            for M, rows, rec in ((R, k1, True), (V, n, False)):
                for c in range(n - 2, i - 1, -1):
                    a, b = M[:rows, c].copy(), M[:rows, c + 1].copy()
                    M[:rows, c], M[:rows, c + 1] = cs[c] * a + sn[c] * b, -sn[c] * a + cs[c] * b
                    if rec and c < k1:
                        y[c] = M[c, c]
            # (3) row angles from the affine recurrence in rho^2
            P0 = min(n - 2, k1 - 2)
            if P0 >= i:
                rc0 = y[P0 + 1] if P0 + 1 <= n - 2 else dg[P0 + 1]
                rho2 = np.zeros(n + 1)
                acc = rc0 * rc0
                for p in range(P0, i - 1, -1):
                    acc = y[p] ** 2 + sn[p] ** 2 * acc
                    rho2[p] = acc
                # (4) all row rotations, then the zeros below the diagonal
                for p in range(P0, i - 1, -1):
                    rho = np.sqrt(rho2[p])
                    prev = rc0 if p == P0 else np.sqrt(rho2[p + 1])
                    cr, sr = (y[p] / rho, sn[p] * prev / rho) if rho > 0 else (1.0, 0.0)
                    a, b = R[p, i:].copy(), R[p + 1, i:].copy()
                    R[p, i:], R[p + 1, i:] = cr * a + sr * b, -sr * a + cr * b
                R[:k1, i:][np.tril_indices(k1, -1 - i, n - i)] = 0.0
        i += 1
        tails.append(float(np.sum(R[:, i:] ** 2)))
    return V[:, :i], np.asarray(tails)


CASES = [((30, 12), 5), ((8, 12), 6), ((12, 12), 12), ((5, 9), None), ((40, 20), None),
         ((3, 16), 8)]


@pytest.mark.parametrize("shape,r_fixed", CASES)
def test_schedule_equals_the_interleaved_chase(shape, r_fixed):
    rng = np.random.default_rng(sum(shape))
    no, nb = shape
    X = rng.standard_normal((no, nb)) @ np.diag(2.0 ** -np.arange(nb))
    d2 = 0.01 * np.sum(X * X)
    r_max = nb if r_fixed is not None else min(no, nb)
    Vm, tm = _schedule_model(X, d2, r_fixed, r_max)
    Vo, to = otc.lurv(X, d2, r_fixed, r_max)
    assert Vm.shape == Vo.shape
    assert np.abs(Vm - Vo).max() < 1e-12
    assert np.abs(tm - to).max() < 1e-12 * to[0]


def test_schedule_on_a_rank_deficient_matrix():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((20, 3)) @ rng.standard_normal((3, 14))
    Vm, tm = _schedule_model(X, 0.0, 6, 14)
    Vo, to = otc.lurv(X, 0.0, 6, 14)
    assert np.abs(np.abs(Vm) - np.abs(Vo))[:, :3].max() < 1e-10
    assert np.allclose(Vm.T @ Vm, np.eye(6), atol=1e-12)
    assert np.abs(tm[:4] - to[:4]).max() < 1e-10 * to[0]

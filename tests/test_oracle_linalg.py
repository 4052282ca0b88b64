"""Pins for the oracle's Householder QR and one-sided Jacobi SVD.

Each is checked against LAPACK (numpy/scipy: an independent implementation)
and against closed forms, so a dropped term, a wrong sign or a transposed
operand in the oracle fails here.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle.linalg import householder_qr, jacobi_svd


SHAPES = [(40, 7), (7, 40), (16, 16), (1, 5), (5, 1), (33, 33)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("piv", [False, True])
def test_qr_reconstructs_and_is_orthonormal(shape, piv):
    rng = np.random.default_rng(1)
    A = rng.standard_normal(shape)
    Q, R, perm = householder_qr(A, pivoting=piv)
    k = min(shape)
    assert Q.shape == (shape[0], k) and R.shape == (k, shape[1])
    np.testing.assert_allclose(A[:, perm], Q @ R, atol=1e-13)
    np.testing.assert_allclose(Q.T @ Q, np.eye(k), atol=1e-14)
    assert np.all(np.tril(R, -1) == 0.0)
    if not piv:
        assert np.array_equal(perm, np.arange(shape[1]))


@pytest.mark.parametrize("shape", SHAPES)
def test_qr_matches_lapack_up_to_signs(shape):
    rng = np.random.default_rng(2)
    A = rng.standard_normal(shape)
    _, R, _ = householder_qr(A)
    Rl = np.linalg.qr(A, mode="r")
    np.testing.assert_allclose(np.abs(R), np.abs(Rl[: R.shape[0]]), atol=1e-12)
    # pivoted: LAPACK geqp3 uses the same largest-remaining-norm rule
    _, Rp, perm = householder_qr(A, pivoting=True)
    Rs, ps = scipy.linalg.qr(A, pivoting=True, mode="r")
    assert np.array_equal(perm, ps)
    np.testing.assert_allclose(np.abs(Rp), np.abs(Rs[: Rp.shape[0]]), atol=1e-12)


def test_qr_sign_convention_and_pivot_order():
    # x = (3, 4): v = x + 5 e1, H x = -5 e1  (sign(x1) = +1)
    Q, R, _ = householder_qr(np.array([[3.0], [4.0]]))
    assert R[0, 0] == pytest.approx(-5.0)
    # sign(0) = +1: x = (0, 2) -> R = -2
    _, R, _ = householder_qr(np.array([[0.0], [2.0]]))
    assert R[0, 0] == pytest.approx(-2.0)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((30, 12)) * np.logspace(0, -6, 12)
    _, R, _ = householder_qr(A, pivoting=True)
    d = np.abs(np.diag(R))
    assert np.all(d[:-1] >= d[1:] * (1 - 1e-12))
    # ties: equal column norms keep the lowest index first
    _, _, perm = householder_qr(np.eye(4), pivoting=True)
    assert np.array_equal(perm, np.arange(4))


def test_qr_full_q_completion():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((9, 4))
    Q, R, perm = householder_qr(A, full_q=True)
    assert Q.shape == (9, 9) and R.shape == (9, 4)
    np.testing.assert_allclose(Q.T @ Q, np.eye(9), atol=1e-14)
    np.testing.assert_allclose(Q @ R, A, atol=1e-13)


def test_qr_rank_deficient():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((20, 3)) @ rng.standard_normal((3, 8))
    Q, R, perm = householder_qr(A, pivoting=True)
    np.testing.assert_allclose(A[:, perm], Q @ R, atol=1e-12)
    assert np.abs(R[3:, 3:]).max() < 1e-12 * np.abs(R).max()


@pytest.mark.parametrize("shape", [(40, 7), (7, 40), (16, 16), (3, 1), (50, 50)])
def test_jacobi_matches_lapack(shape):
    rng = np.random.default_rng(6)
    A = rng.standard_normal(shape)
    sig, V = jacobi_svd(A)
    s_ref = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(sig[: len(s_ref)], s_ref, rtol=1e-12, atol=1e-12 * s_ref[0])
    assert np.all(sig[len(s_ref):] < 1e-12 * s_ref[0])
    np.testing.assert_allclose(V.T @ V, np.eye(shape[1]), atol=1e-13)
    AV = A @ V
    G = AV.T @ AV
    np.testing.assert_allclose(G - np.diag(np.diag(G)), 0, atol=1e-12 * s_ref[0] ** 2)
    np.testing.assert_allclose(np.sqrt(np.diag(G)), sig, atol=1e-12 * s_ref[0])


def test_jacobi_closed_forms():
    # diagonal
    sig, _ = jacobi_svd(np.diag([1.0, -5.0, 3.0]))
    np.testing.assert_allclose(sig, [5.0, 3.0, 1.0], rtol=1e-15)
    # rank one u v^T: sigma_1 = |u||v|, the rest zero
    u, v = np.arange(1.0, 6.0), np.array([2.0, -1.0, 0.5])
    sig, V = jacobi_svd(np.outer(u, v))
    assert sig[0] == pytest.approx(np.linalg.norm(u) * np.linalg.norm(v), rel=1e-14)
    assert np.all(sig[1:] < 1e-13)
    np.testing.assert_allclose(np.abs(V[:, 0]), np.abs(v) / np.linalg.norm(v), atol=1e-13)
    # 2x2 upper triangular [[a, b], [0, c]]: sigma_1 sigma_2 = |ac|, s1^2 + s2^2 = a^2+b^2+c^2
    a, b, c = 3.0, 4.0, 2.0
    sig, _ = jacobi_svd(np.array([[a, b], [0.0, c]]))
    assert sig[0] * sig[1] == pytest.approx(abs(a * c), rel=1e-14)
    assert sig[0] ** 2 + sig[1] ** 2 == pytest.approx(a * a + b * b + c * c, rel=1e-14)
    # orthogonal matrix: all singular values 1
    Q, _ = np.linalg.qr(np.random.default_rng(7).standard_normal((12, 12)))
    sig, _ = jacobi_svd(Q)
    np.testing.assert_allclose(sig, 1.0, atol=1e-14)

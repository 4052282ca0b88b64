"""Pins of the oracle's Givens-based low-rank URV (`tt.lurv`, the family of
warm-started low-rank UTV algorithms the paper's TT-URV experiments run as
the inner factor, Sec. 4) against facts that do not come from its own code:

* a Givens rotation maps (a, b) to (hypot(a, b), 0) and is orthogonal;
* a diagonal matrix worked by hand (q = 0: the warm start is already the
  decomposition; tails 14, 5, 1, 0);
* the factorisation holds throughout: X Pi-start = Q R V^T with R upper
  trapezoidal and V orthogonal, so X V = Q R (checked as ||X V||_F per
  column against ||R||_F per column, and X V V^T = X);
* the error of keeping i basis vectors is the directly computed residual
  ||X - X V_i V_i^T||^2 (plus the range miss), for any q;
* with many power iterations on a gapped spectrum the basis is LAPACK's top
  singular vectors and the errors are Eckart-Young's;
* in the sweep: RSE <= eps, the equality inside the proof of Thm 3.1, exact
  recovery of TT-structured tensors, and the sketched fixed-rank path.
"""
import numpy as np
import pytest

import synth
from oracle import tt as otc


def test_givens_rotation():
    for a, b in ((3.0, 4.0), (-2.0, 1.0), (0.0, -5.0), (1e-300, 1e-300)):
        c, s = otc.givens(a, b)
        assert abs(c * c + s * s - 1.0) < 1e-15
        assert abs(c * a + s * b - np.hypot(a, b)) < 1e-15 * max(1.0, np.hypot(a, b))
        assert abs(-s * a + c * b) < 1e-15 * max(1.0, np.hypot(a, b))
    assert otc.givens(0.0, 0.0) == (1.0, 0.0)


def test_diagonal_by_hand():
    X = np.zeros((4, 3))
    X[0, 0], X[1, 1], X[2, 2] = 3.0, 2.0, 1.0
    V, tails = otc.lurv(X, 0.0, 3, 3, q=0)
    assert np.allclose(np.abs(V), np.eye(3))
    assert np.allclose(tails, [14.0, 5.0, 1.0, 0.0])
    V2, t2 = otc.lurv(X, 1.5, None, 3, q=0)
    assert V2.shape[1] == 2 and np.allclose(t2, [14.0, 5.0, 1.0])


@pytest.mark.parametrize("q", [0, 2, 8])
def test_factorisation_invariants_and_exact_tails(q):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((40, 12)) @ np.diag(np.linspace(3, 0.05, 12)) @ rng.standard_normal((12, 12))
    V1, tails, R, V = otc.lurv(X, 0.0, 9, 12, q=q, mu2=0.5, return_r=True)
    assert np.allclose(V.T @ V, np.eye(12), atol=1e-13)
    assert np.allclose(np.tril(R, -1), 0.0, atol=1e-12 * np.abs(R).max())
    # X V = Q R with Q orthonormal: column norms agree, and X V V^T = X
    assert np.allclose(np.linalg.norm(X @ V, axis=0), np.linalg.norm(R, axis=0), rtol=1e-11)
    assert np.allclose(X @ V @ V.T, X, atol=1e-12 * np.abs(X).max())
    for i in range(10):
        Vi = V1[:, :i]
        E = X - X @ Vi @ Vi.T
        assert tails[i] == pytest.approx(0.5 + float(np.sum(E * E)), rel=1e-10, abs=1e-12)


def test_many_iterations_give_the_singular_vectors():
    rng = np.random.default_rng(2)
    U, _ = np.linalg.qr(rng.standard_normal((50, 10)))
    W, _ = np.linalg.qr(rng.standard_normal((10, 10)))
    s = 2.0 ** -np.arange(10)
    X = (U * s) @ W.T
    V, tails = otc.lurv(X, 0.0, 5, 10, q=200)
    _, sv, vt = np.linalg.svd(X)
    for i in range(5):
        assert abs(abs(float(vt[i] @ V[:, i])) - 1.0) < 1e-10
    for r in range(6):
        assert tails[r] == pytest.approx(float(np.sum(sv[r:] ** 2)), rel=1e-9, abs=1e-14)


def test_adaptive_stop_and_rank_deficiency():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((20, 3)) @ rng.standard_normal((3, 15))
    V, tails = otc.lurv(X, 1e-20 * np.sum(X * X), None, 15, q=4)
    assert V.shape[1] == 3
    Y = rng.standard_normal((30, 12)) @ np.diag(2.0 ** -np.arange(12))
    d2 = 0.01 * np.sum(Y * Y)
    Vy, ty = otc.lurv(Y, d2, None, 12, q=2)
    r = Vy.shape[1]
    assert ty[r] <= d2 and (r == 1 or ty[r - 1] > d2)


@pytest.mark.parametrize("variant", ["URV", "ULV"])
def test_sweep_with_lurv_meets_the_theorems(variant):
    A = synth.gaussian_tt((6, 7, 8, 5), (1, 3, 4, 2, 1), 1e-3, seed=5, dtype=np.float64)
    for eps in (1e-2, 1e-4):
        res = otc.tt_utv(A, eps=eps, variant=variant, inner="lurv")
        rse = otc.rse(A, res["cores"])
        assert rse <= eps
        assert abs(rse ** 2 * res["normA2"] - sum(res["tails"])) <= 1e-10 * res["normA2"]
    B = synth.gaussian_tt((5, 6, 7, 4), (1, 2, 3, 2, 1), 0.0, seed=6, dtype=np.float64)
    res = otc.tt_utv(B, eps=1e-10, variant=variant, inner="lurv")
    assert res["ranks"] == [1, 2, 3, 2, 1]
    assert otc.rse(B, res["cores"]) < 1e-12


def test_sketch_path_and_fixed_ranks():
    A = synth.gaussian_tt((4, 5, 300), (1, 3, 4, 1), 1e-4, seed=7, dtype=np.float64)
    res = otc.tt_utv(A, ranks=[3, 4], variant="URV", inner="lurv")
    assert res["ranks"] == [1, 3, 4, 1]
    assert res["steps"][0]["path"] == "sketch"
    assert otc.rse(A, res["cores"]) < 1e-3


def test_start_vector_with_no_iterations():
    # q = 0: the first basis vector is X^T X e_j / ||.|| for the column j of X
    # of largest norm (the warm start's first pivot)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((25, 8)) @ rng.standard_normal((8, 8))
    V, _ = otc.lurv(X, 0.0, 2, 8, q=0)
    j = int(np.argmax(np.sum(X * X, axis=0)))
    v = X.T @ X[:, j]
    v /= np.linalg.norm(v)
    assert abs(abs(float(v @ V[:, 0])) - 1.0) < 1e-12

"""Pins of the oracle's USV-plus-style inner factor (the deflation the paper
runs inside TT-ULV in Sec. 4, stopping rule adapted to fixed ranks and to
Alg. 2) against facts that do not come from its own code:

* a diagonal matrix worked by hand (q = 0: start vectors and tails);
* each vector is the normalised (D^T D)^(q+1) e_j of the deflated matrix,
  recomputed with a matrix power;
* with many power iterations on a spectrum with gaps, the basis is LAPACK's
  top-r right singular vectors (up to sign) and the tails are Eckart-Young's
  sums of the dropped squared singular values;
* for any q the basis is orthonormal and tail(i) is the directly computed
  residual ||X - X V_i V_i^T||^2 (plus the range miss);
* the adaptive stop is the first i with tail(i) <= delta^2; an exactly
  rank-k matrix stops at k, and a fixed rank above k is completed with
  orthonormal unit vectors;
* in the sweep, TT-ULV / TT-URV with this inner factor satisfy the equality
  inside the proof of Thm 3.1 (RSE^2 ||A||^2 = sum of the step errors), the
  bound RSE <= eps of Alg. 2, and recover TT-structured tensors exactly.
"""
import numpy as np
import pytest

import synth
from oracle import tt as otc


def test_diagonal_by_hand():
    X = np.zeros((4, 3))
    X[0, 0], X[1, 1], X[2, 2] = 3.0, 2.0, 1.0
    V, tails = otc.usv_plus(X, 0.0, 3, 3, q=0)
    # column norms 9, 4, 1: starts e_0, e_1, e_2 in turn
    assert np.allclose(np.abs(V), np.eye(3))
    assert np.allclose(tails, [14.0, 5.0, 1.0, 0.0])
    # the adaptive rule with delta^2 = 1.5 keeps two vectors
    V2, t2 = otc.usv_plus(X, 1.5, None, 3, q=0)
    assert V2.shape[1] == 2 and np.allclose(t2, [14.0, 5.0, 1.0])


def test_vectors_are_matrix_powers_of_the_deflated_gram():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((30, 12))
    q = 3
    V, _ = otc.usv_plus(X, 0.0, 4, 12, q=q)
    P = np.eye(12)
    for i in range(4):
        D = X @ P
        G = D.T @ D
        j = int(np.argmax(np.diag(G)))
        v = np.linalg.matrix_power(G, q + 1)[:, j]
        v = P @ v
        v /= np.linalg.norm(v)
        assert abs(abs(float(v @ V[:, i])) - 1.0) < 1e-10, i
        P = P - np.outer(V[:, i], V[:, i])


def test_many_iterations_give_the_singular_vectors():
    rng = np.random.default_rng(2)
    U, _ = np.linalg.qr(rng.standard_normal((40, 10)))
    W, _ = np.linalg.qr(rng.standard_normal((10, 10)))
    s = 2.0 ** -np.arange(10)
    X = (U * s) @ W.T
    V, tails = otc.usv_plus(X, 0.0, 5, 10, q=200)
    _, sv, vt = np.linalg.svd(X)
    for i in range(5):
        assert abs(abs(float(vt[i] @ V[:, i])) - 1.0) < 1e-10
    for r in range(6):
        assert tails[r] == pytest.approx(float(np.sum(sv[r:] ** 2)), rel=1e-9, abs=1e-14)


@pytest.mark.parametrize("q", [0, 1, 8])
def test_orthonormal_basis_and_exact_tails(q):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((25, 9)) @ np.diag(np.linspace(3, 0.1, 9))
    V, tails = otc.usv_plus(X, 0.0, 9, 9, q=q, mu2=0.25)
    assert np.allclose(V.T @ V, np.eye(9), atol=1e-12)
    for i in range(10):
        Vi = V[:, :i]
        E = X - X @ Vi @ Vi.T
        assert tails[i] == pytest.approx(0.25 + float(np.sum(E * E)), rel=1e-10, abs=1e-12)


def test_adaptive_stop_and_exact_rank():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((20, 3)) @ rng.standard_normal((3, 15))
    V, tails = otc.usv_plus(X, 1e-20 * np.sum(X * X), None, 15, q=4)
    assert V.shape[1] == 3 and tails[-1] <= 1e-20 * np.sum(X * X) + 1e-18
    # a fixed rank above the matrix rank is completed with orthonormal vectors
    V5, t5 = otc.usv_plus(X, 0.0, 5, 15, q=4)
    assert V5.shape[1] == 5 and np.allclose(V5.T @ V5, np.eye(5), atol=1e-12)
    assert abs(t5[-1]) < 1e-9 * np.sum(X * X)
    # the adaptive rank is the first that meets the tolerance
    Y = rng.standard_normal((30, 12)) @ np.diag(2.0 ** -np.arange(12))
    d2 = 0.01 * np.sum(Y * Y)
    Vy, ty = otc.usv_plus(Y, d2, None, 12, q=2)
    r = Vy.shape[1]
    assert ty[r] <= d2 and (r == 1 or ty[r - 1] > d2)


@pytest.mark.parametrize("variant", ["ULV", "URV"])
def test_sweep_with_usvp_meets_the_theorems(variant):
    A = synth.gaussian_tt((6, 7, 8, 5), (1, 3, 4, 2, 1), 1e-3, seed=5, dtype=np.float64)
    for eps in (1e-2, 1e-4):
        res = otc.tt_utv(A, eps=eps, variant=variant, inner="usvp")
        rse = otc.rse(A, res["cores"])
        assert rse <= eps
        assert abs(rse ** 2 * res["normA2"] - sum(res["tails"])) <= 1e-10 * res["normA2"]
    # exact recovery of a TT-structured tensor
    B = synth.gaussian_tt((5, 6, 7, 4), (1, 2, 3, 2, 1), 0.0, seed=6, dtype=np.float64)
    res = otc.tt_utv(B, eps=1e-10, variant=variant, inner="usvp")
    assert res["ranks"] == [1, 2, 3, 2, 1]
    assert otc.rse(B, res["cores"]) < 1e-12


def test_sketch_path_and_fixed_ranks():
    A = synth.gaussian_tt((4, 5, 300), (1, 3, 4, 1), 1e-4, seed=7, dtype=np.float64)
    res = otc.tt_utv(A, ranks=[3, 4], variant="URV", inner="usvp")
    assert res["ranks"] == [1, 3, 4, 1]
    assert res["steps"][0]["path"] == "sketch"
    assert otc.rse(A, res["cores"]) < 1e-3

"""Pins of the Riemannian-gradient oracle (Sec. 4.2.2) against facts that do
not come from its own code:

* the tangent-space projection is an orthogonal projector (idempotent and
  self-adjoint) whose rank is the dimension of the manifold of TT tensors of
  fixed ranks, sum_k r_{k-1} I_k r_k - sum_{k<d} r_k^2 (Holtz, Rohwedder and
  Schneider 2012); it fixes the point itself and every velocity of a curve of
  TT tensors; its increments satisfy the gauge U_k^T dU_k = 0;
* for d = 2 it is the textbook projection onto the tangent space of the
  fixed-rank matrices, U U^T Z + Z V V^T - U U^T Z V V^T (U, V from LAPACK's
  SVD);
* the entry-by-entry mixed-interface gradient equals the oracle's vectorised
  masked gradient when both interface sets are the same cores, and after the
  gauge it equals the dense projection of the zero-filled observations;
* the step is the minimiser of the quadratic along the direction;
* the descent recovers an exactly low-rank tensor from a fraction of its
  entries, with either retraction.
"""
import numpy as np
import pytest

import synth
from oracle import rgrad as org
from oracle import tt as otc


def _tt(dims, ranks, seed):
    return [np.asarray(c, np.float64) for c in synth.gaussian_cores(dims, ranks, seed=seed)]


def _proj(U, V, Z):
    return otc.tt_full(org.tangent_cores(U, V, org.tangent_project(U, V, Z)))


def _frames(dims, ranks, seed):
    X = _tt(dims, ranks, seed)
    return X, org.left_orthogonal(X), org.right_orthogonal(X)


def test_orthogonal_frames_represent_the_same_tensor():
    X, U, V = _frames((4, 5, 6, 3), (1, 2, 3, 2, 1), 1)
    full = otc.tt_full(X)
    assert np.allclose(otc.tt_full(U), full, atol=1e-12 * np.abs(full).max())
    assert np.allclose(otc.tt_full(V), full, atol=1e-12 * np.abs(full).max())
    for g in U[:-1]:
        m = g.reshape(-1, g.shape[2])
        assert np.allclose(m.T @ m, np.eye(m.shape[1]), atol=1e-13)
    for g in V[1:]:
        m = g.reshape(g.shape[0], -1)
        assert np.allclose(m @ m.T, np.eye(m.shape[0]), atol=1e-13)


@pytest.mark.parametrize("dims,ranks", [((3, 4, 5), (1, 2, 3, 1)),
                                        ((2, 3, 2, 3), (1, 2, 3, 2, 1)),
                                        ((6, 5), (1, 2, 1))])
def test_projector_rank_is_the_manifold_dimension(dims, ranks):
    X, U, V = _frames(dims, ranks, 2)
    N = int(np.prod(dims))
    P = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        P[:, j] = _proj(U, V, e.reshape(dims)).reshape(-1)
    assert np.allclose(P, P.T, atol=1e-12)            # self-adjoint
    assert np.allclose(P @ P, P, atol=1e-12)          # idempotent
    dim = sum(ranks[k] * dims[k] * ranks[k + 1] for k in range(len(dims))) \
        - sum(r * r for r in ranks[1:-1])
    ev = np.linalg.eigvalsh(P)
    assert np.all((np.abs(ev) < 1e-10) | (np.abs(ev - 1) < 1e-10))
    assert int(np.sum(ev > 0.5)) == dim
    assert abs(np.trace(P) - dim) < 1e-9


def test_projector_fixes_the_point_and_curve_velocities():
    dims, ranks = (4, 5, 3, 4), (1, 2, 3, 2, 1)
    X, U, V = _frames(dims, ranks, 3)
    full = otc.tt_full(X)
    assert np.allclose(_proj(U, V, full), full, atol=1e-12 * np.abs(full).max())
    rng = np.random.default_rng(4)
    dX = [rng.standard_normal(g.shape) for g in X]
    # the velocity of t -> TT(X + t dX) at t = 0 (multilinear in the cores)
    vel = sum(otc.tt_full([dX[j] if j == k else X[j] for j in range(len(X))])
              for k in range(len(X)))
    assert np.allclose(_proj(U, V, vel), vel, atol=1e-11 * np.abs(vel).max())
    # and a generic tensor is moved
    Z = rng.standard_normal(dims)
    assert np.linalg.norm(_proj(U, V, Z) - Z) > 0.5 * np.linalg.norm(Z)


def test_gauge_and_residual_orthogonality():
    dims, ranks = (5, 4, 6), (1, 3, 2, 1)
    X, U, V = _frames(dims, ranks, 5)
    rng = np.random.default_rng(6)
    Z = rng.standard_normal(dims)
    dU = org.tangent_project(U, V, Z)
    for k in range(len(dims) - 1):
        ul = U[k].reshape(-1, U[k].shape[2])
        assert np.abs(ul.T @ dU[k].reshape(ul.shape[0], -1)).max() < 1e-12
    # Z - P Z is orthogonal to every tangent vector (one from random increments)
    W = org.tangent_project(U, V, rng.standard_normal(dims))
    t = otc.tt_full(org.tangent_cores(U, V, W))
    res = Z - otc.tt_full(org.tangent_cores(U, V, dU))
    assert abs(np.sum(res * t)) < 1e-11 * np.linalg.norm(res) * np.linalg.norm(t)


def test_matrix_case_is_the_textbook_projection():
    X, U, V = _frames((7, 9), (1, 3, 1), 7)
    Z = np.random.default_rng(8).standard_normal((7, 9))
    u, s, vt = np.linalg.svd(otc.tt_full(X))
    Pu, Pv = u[:, :3] @ u[:, :3].T, vt[:3].T @ vt[:3]
    ref = Pu @ Z + Z @ Pv - Pu @ Z @ Pv
    assert np.allclose(_proj(U, V, Z), ref, atol=1e-12)


def test_mixed_gradient_matches_the_vectorised_and_dense_forms():
    dims, ranks = (4, 3, 5, 3), (1, 2, 3, 2, 1)
    X, U, V = _frames(dims, ranks, 9)
    rng = np.random.default_rng(10)
    idx = rng.choice(int(np.prod(dims)), 70, replace=False)
    g = rng.standard_normal(len(idx))
    same = org.mixed_eval_grad(X, X, idx, g)
    for a, b in zip(same, otc.tt_eval_grad(X, idx, g)):
        assert np.allclose(a, b, atol=1e-12)
    Y = org.mixed_eval_grad(U, V, idx, g)
    for k in range(len(dims) - 1):
        ul = U[k].reshape(-1, U[k].shape[2])
        yl = Y[k].reshape(ul.shape[0], -1)
        Y[k] = (yl - ul @ (ul.T @ yl)).reshape(Y[k].shape)
    Z = np.zeros(int(np.prod(dims)))
    np.add.at(Z, idx, g)
    for a, b in zip(Y, org.tangent_project(U, V, Z.reshape(dims))):
        assert np.allclose(a, b, atol=1e-12)


def test_step_size_is_the_line_minimiser():
    rng = np.random.default_rng(11)
    xi, z = rng.standard_normal(50), rng.standard_normal(50)
    a = org.step_size(xi, z)
    f = lambda t: float(np.sum((z - t * xi) ** 2))  # noqa: E731
    assert abs(float(np.dot(xi, z - a * xi))) < 1e-12   # zero derivative
    for h in (1e-3, -1e-3, 0.5, -0.5):
        assert f(a) <= f(a + h)
    assert org.step_size(np.zeros(5), np.ones(5)) == 0.0


@pytest.mark.parametrize("variant", ["URV", "SVD"])
def test_rgrad_recovers_a_low_rank_tensor(variant):
    dims, ranks = (10, 11, 9), (1, 2, 3, 1)
    T = otc.tt_full(_tt(dims, ranks, 12))
    idx = np.sort(np.random.default_rng(13).choice(T.size, T.size // 2, replace=False))
    cores, losses = org.rgrad(T.reshape(-1)[idx], idx, dims, ranks, steps=60, variant=variant)
    assert losses[-1] < 1e-8 * losses[0]
    assert otc.rse(T, cores) < 1e-5

"""Pins for the oracle's TT algorithms (TT format, TT-ULV/TT-URV sweeps, TT-SVD,
masked evaluation), against what the paper and the mathematics fix:

* Eq. TT written out as an explicit sum (brute force on tiny tensors);
* the UTV identity and triangular structure (Eqs. ulv, urv) and the residual
  orthogonality EV_1 = 0 / U_1^T E = 0 the error analysis relies on (Sec. 3);
* the equality inside the proof of Thm 3.1 (and its URV analogue, Thm 3.2):
  ||A - A_hat||_F^2 = sum_k ||E_k||_F^2 when every residual is orthogonal to
  the kept basis;  the bound of Alg. 2: ||A - A_hat|| <= eps ||A||;
* left/right orthogonality of the cores (Def. 2.2, outputs of Alg. 1-3);
* Eckart-Young for d = 2 and brute-force sequential truncated SVD of full
  unfoldings with LAPACK (an independent implementation) for TT-SVD;
* exact recovery of tensors built from known TT cores.
"""
import itertools

import numpy as np
import pytest

import synth
from oracle import tt


def brute_full(cores):
    dims = [g.shape[1] for g in cores]
    out = np.zeros(dims)
    for idx in itertools.product(*[range(n) for n in dims]):
        v = np.ones((1, 1))
        for g, i in zip(cores, idx):
            v = v @ g[:, i, :]
        out[idx] = v[0, 0]
    return out


def brute_tt_svd_lr(A, eps):
    """Sequential truncated SVD of the full unfoldings with LAPACK (left-to-right)."""
    dims = A.shape
    d = len(dims)
    delta2 = eps ** 2 * np.sum(A * A) / (d - 1)
    C = A.reshape(dims[0], -1)
    rp, ranks, cores = 1, [1], []
    for k in range(d - 1):
        C = C.reshape(rp * dims[k], -1)
        U, s, Vt = np.linalg.svd(C, full_matrices=False)
        tails = np.concatenate([np.cumsum((s * s)[::-1])[::-1], [0.0]])
        r = next((q for q in range(1, len(s) + 1) if tails[q] <= delta2), len(s))
        cores.append(U[:, :r].reshape(rp, dims[k], r))
        C = s[:r, None] * Vt[:r]
        rp = r
        ranks.append(r)
    cores.append(C.reshape(rp, dims[-1], 1))
    return ranks + [1], cores


def right_orth_err(g):
    G1 = g.reshape(g.shape[0], -1)
    return np.abs(G1 @ G1.T - np.eye(g.shape[0])).max()


def left_orth_err(g):
    G2 = g.reshape(-1, g.shape[2])
    return np.abs(G2.T @ G2 - np.eye(g.shape[2])).max()


def test_tt_full_is_eq_tt():
    cores = synth.gaussian_cores((3, 4, 2, 3), (1, 2, 3, 2, 1), seed=11)
    np.testing.assert_allclose(tt.tt_full(cores), brute_full(cores), atol=1e-12)
    np.testing.assert_allclose(synth.contract_cores(cores), brute_full(cores), atol=1e-12)


@pytest.mark.parametrize("shape", [(30, 8), (8, 30), (12, 12)])
@pytest.mark.parametrize("variant", ["URV", "ULV"])
def test_utv_identity_structure_and_residual_orthogonality(shape, variant):
    rng = np.random.default_rng(12)
    X = rng.standard_normal(shape) * np.logspace(0, -4, shape[1])
    U, T, V = tt.utv_of(X, variant)
    np.testing.assert_allclose(U @ T @ V.T, X, atol=1e-13)
    np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-13)
    if variant == "URV":
        assert np.all(np.tril(T, -1) == 0)
    else:
        assert np.all(np.triu(T, 1) == 0)
    for r in range(1, min(shape)):
        if variant == "URV":
            V1 = V[:, :r]
            E = X - X @ V1 @ V1.T
            np.testing.assert_allclose(E @ V1, 0, atol=1e-12)
            tail_T = np.sum(T[:, r:] ** 2)          # ||[R12; R22]||^2
        else:
            U1 = U[:, :r]
            E = X - U1 @ U1.T @ X
            np.testing.assert_allclose(U1.T @ E, 0, atol=1e-12)
            tail_T = np.sum(T[r:, :] ** 2)          # ||[L21 L22]||^2
        assert np.sum(E * E) == pytest.approx(tail_T, rel=1e-10, abs=1e-24)


def test_qlp_tails_are_truncation_errors_and_track_svd():
    rng = np.random.default_rng(13)
    X = rng.standard_normal((40, 10)) @ np.diag(np.logspace(0, -5, 10)) @ np.linalg.qr(
        rng.standard_normal((10, 10)))[0]
    Z, L, _ = tt.qlp(X)
    tails = tt.qlp_tails(L)
    s = np.linalg.svd(X, compute_uv=False)
    ey = np.concatenate([np.cumsum((s * s)[::-1])[::-1], [0.0]])
    for r in range(0, 11):
        E = X - X @ Z[:, :r] @ Z[:, :r].T
        assert np.sum(E * E) == pytest.approx(tails[r], rel=1e-9, abs=1e-28)
        assert tails[r] >= ey[r] * (1 - 1e-10)        # never better than Eckart-Young
        assert tails[r] <= 20 * ey[r] + 1e-28          # pivoted QLP tracks the SVD closely


@pytest.mark.parametrize("r", [1, 3, 6])
def test_tt_svd_d2_is_eckart_young(r):
    rng = np.random.default_rng(14)
    A = rng.standard_normal((25, 17))
    s = np.linalg.svd(A, compute_uv=False)
    res = tt.tt_svd(A, ranks=[r])
    assert res["ranks"] == [1, r, 1]
    assert res["tails"][0] == pytest.approx(np.sum(s[r:] ** 2), rel=1e-12)
    assert tt.rse(A, res["cores"]) ** 2 * np.sum(A * A) == pytest.approx(np.sum(s[r:] ** 2), rel=1e-10)


@pytest.mark.parametrize("shape", [(3, 4, 5), (4, 4, 4, 4), (5, 3, 4, 2)])
@pytest.mark.parametrize("eps", [0.3, 0.05])
def test_tt_svd_matches_brute_force_lapack(shape, eps):
    rng = np.random.default_rng(15)
    A = rng.standard_normal(shape)
    ranks, cores = brute_tt_svd_lr(A, eps)
    res = tt.tt_svd(A, eps=eps)
    assert res["ranks"] == ranks
    assert tt.rse(A, res["cores"]) == pytest.approx(tt.rse(A, cores), rel=1e-9)
    np.testing.assert_allclose(tt.tt_full(res["cores"]), tt.tt_full(cores), atol=1e-10)


def test_utv_first_step_never_beats_svd():
    rng = np.random.default_rng(16)
    A = rng.standard_normal((6, 5, 4, 3))
    for eps in (0.5, 0.2, 0.05):
        u = tt.tt_utv(A, eps=eps, variant="ULV")
        s = tt.tt_svd(A, eps=eps)
        assert u["ranks"][1] >= s["ranks"][1]


@pytest.mark.parametrize("variant", ["URV", "ULV", "SVD"])
def test_exact_recovery(variant):
    cores = synth.gaussian_cores((6, 6, 6, 6), (1, 2, 3, 2, 1), seed=17)
    A = synth.contract_cores(cores)
    run = (lambda **k: tt.tt_svd(A, **k)) if variant == "SVD" else (
        lambda **k: tt.tt_utv(A, variant=variant, **k))
    res = run(eps=1e-10)
    assert res["ranks"] == [1, 2, 3, 2, 1]
    assert tt.rse(A, res["cores"]) < 1e-13
    res = run(eps=1e-10, l_full=4)               # forces the sketch path
    assert res["ranks"] == [1, 2, 3, 2, 1]
    assert tt.rse(A, res["cores"]) < 1e-13


def _run(A, variant, **kw):
    if variant == "SVD":
        return tt.tt_svd(A, **kw)
    return tt.tt_utv(A, variant=variant, **kw)


@pytest.mark.parametrize("variant", ["URV", "ULV", "SVD"])
@pytest.mark.parametrize("mode", ["eps", "ranks", "eps-sketch", "ranks-sketch"])
def test_error_equality_bound_and_orthogonality(variant, mode):
    A = synth.gaussian_tt((7, 6, 9, 5), (1, 3, 4, 3, 1), rel_noise=0.05, seed=18, dtype=np.float64)
    kw = dict(l_full=8) if "sketch" in mode else {}
    eps = 0.03
    res = _run(A, variant, **(dict(eps=eps) if mode.startswith("eps") else dict(ranks=[2, 3, 2])), **kw)
    err2 = tt.rse(A, res["cores"]) ** 2 * res["normA2"]
    # equality in the proof of Thm 3.1 / Thm 3.2
    assert err2 == pytest.approx(sum(res["tails"]), rel=1e-10)
    if mode.startswith("eps"):
        assert np.sqrt(err2 / res["normA2"]) <= eps
        for t, d2 in zip(res["tails"], res["delta2"]):
            assert t <= d2
    cores = res["cores"]
    if res["orth"] == "right":
        assert max(right_orth_err(g) for g in cores[1:]) < 1e-13
    else:
        assert max(left_orth_err(g) for g in cores[:-1]) < 1e-13


def test_sketch_path_is_exact_when_l_covers_rank():
    A = synth.gaussian_tt((8, 8, 8, 8), (1, 3, 5, 3, 1), rel_noise=1e-9, seed=19, dtype=np.float64)
    a = tt.tt_utv(A, eps=1e-6, variant="URV")
    b = tt.tt_utv(A, eps=1e-6, variant="URV", l_full=4)
    assert a["ranks"] == b["ranks"] == [1, 3, 5, 3, 1]
    assert any(s["path"] == "sketch" for s in b["steps"])
    np.testing.assert_allclose(tt.tt_full(a["cores"]), tt.tt_full(b["cores"]), atol=1e-7)


@pytest.mark.parametrize("q", [1, 2])
def test_power_iterations_span_the_closed_form(q):
    # span(Y) after q power iterations = span(V S^{2q+1} U^T Omega) for
    # X = U S V^T: the re-orthonormalizations between them change no span.
    # X has a slowly decaying spectrum (1 .. 0.05), where iterations matter.
    rng = np.random.default_rng(31)
    n_o, n_b, l = 90, 70, 12
    U, _ = np.linalg.qr(rng.standard_normal((n_o, n_b)))
    V, _ = np.linalg.qr(rng.standard_normal((n_b, n_b)))
    s = np.geomspace(1.0, 0.05, n_b)
    X = (U * s) @ V.T
    W, B, mu2 = tt.range_step(X, l, seed=3, step=2, q=q)
    from oracle.philox import rademacher
    Om = rademacher(n_o, l, 3, 2)
    Q_ref, _ = np.linalg.qr((V * s ** (2 * q + 1)) @ (U.T @ Om))
    cosines = np.linalg.svd(W.T @ Q_ref, compute_uv=False)
    assert np.all(cosines > 1 - 1e-10), cosines.min()
    np.testing.assert_allclose(W.T @ W, np.eye(l), atol=1e-13)
    np.testing.assert_allclose(B, X @ W, atol=1e-13)
    assert mu2 == pytest.approx(np.sum((X - B @ W.T) ** 2), rel=1e-12)
    # q = 0 is the plain sketch, which misses more of X on this spectrum
    _, _, mu2_0 = tt.range_step(X, l, seed=3, step=2, q=0)
    assert mu2 < mu2_0


def test_power_iterations_keep_exactness_and_identity():
    # l >= rank: every q gives the exact-path ranks and tensor; Omega = I: q ignored
    A = synth.gaussian_tt((8, 8, 8, 8), (1, 3, 5, 3, 1), rel_noise=1e-9, seed=19, dtype=np.float64)
    a = tt.tt_utv(A, eps=1e-6, variant="URV")
    for q in (1, 2):
        b = tt.tt_utv(A, eps=1e-6, variant="URV", l_full=4, q=q)
        assert b["ranks"] == a["ranks"] == [1, 3, 5, 3, 1]
        np.testing.assert_allclose(tt.tt_full(a["cores"]), tt.tt_full(b["cores"]), atol=1e-7)
    X = np.random.default_rng(5).standard_normal((6, 40))
    W0, _, m0 = tt.range_step(X, 6, seed=0, step=1, q=0)
    W2, _, m2 = tt.range_step(X, 6, seed=0, step=1, q=2)
    np.testing.assert_array_equal(W0, W2)
    assert m0 == m2


def test_sketch_grows_when_too_small():
    # rank 40 at the sketched step but the first sketch has l = 32 columns
    A = synth.gaussian_tt((50, 50, 50), (1, 40, 40, 1), rel_noise=1e-10, seed=20, dtype=np.float64)
    res = tt.tt_utv(A, eps=1e-6, variant="URV", l_full=16)
    assert res["ranks"] == [1, 40, 40, 1]
    assert res["steps"][0]["l"] >= 40 + 16 or res["steps"][0]["l"] == 50


def test_config_c1_ranks():
    A = synth.make_config("c1")
    for res in (tt.tt_utv(A, eps=1e-6, variant="URV"), tt.tt_utv(A, eps=1e-6, variant="ULV"),
                tt.tt_svd(A, eps=1e-6)):
        assert res["ranks"] == [1, 4, 4, 4, 1]
        assert tt.rse(A, res["cores"]) < 1e-6


def test_edge_cases():
    rng = np.random.default_rng(21)
    # a mode of size 1, d = 2, fixed rank above the matrix size is clamped
    A = rng.standard_normal((5, 1, 7))
    res = tt.tt_utv(A, ranks=[9, 9], variant="URV")
    # unfoldings are 5 x 7 and 5 x 5: both ranks clamp to 5
    assert res["ranks"] == [1, 5, 5, 1]
    assert tt.rse(A, res["cores"]) < 1e-12
    M = rng.standard_normal((6, 4))
    res = tt.tt_utv(M, ranks=[10], variant="ULV")
    assert res["ranks"] == [1, 4, 1]
    assert tt.rse(M, res["cores"]) < 1e-13
    # zero tensor: ||C|| <= delta at once, rank 1
    Z = np.zeros((3, 4, 5))
    res = tt.tt_utv(Z, eps=0.1, variant="URV")
    assert res["ranks"] == [1, 1, 1, 1]
    assert np.all(tt.tt_full(res["cores"]) == 0)


def test_masked_eval_and_gradient():
    cores = synth.gaussian_cores((5, 4, 6), (1, 3, 2, 1), seed=22)
    full = tt.tt_full(cores)
    idx = synth.random_indices((5, 4, 6), 50, seed=23)
    np.testing.assert_allclose(tt.tt_eval_at(cores, idx), full.ravel()[idx], atol=1e-13)
    gout = np.random.default_rng(24).standard_normal(50)
    grads = tt.tt_eval_grad(cores, idx, gout)
    # brute force: d/dG of sum_e g_e x(i_e) is linear -> exact central differences
    h = 1e-6
    rng = np.random.default_rng(25)
    for k, g in enumerate(cores):
        for _ in range(6):
            pos = tuple(rng.integers(0, s) for s in g.shape)
            cp = [c.copy() for c in cores]
            cm = [c.copy() for c in cores]
            cp[k][pos] += h
            cm[k][pos] -= h
            fd = (gout @ tt.tt_eval_at(cp, idx) - gout @ tt.tt_eval_at(cm, idx)) / (2 * h)
            assert grads[k][pos] == pytest.approx(fd, rel=1e-6, abs=1e-8)


# ------------------------------------------- TT-ULV right-to-left (appendix, Alg. 4)

@pytest.mark.parametrize("l_full", [256, 6])
def test_alg4_full_block_equals_urv_rl(l_full):
    # the appendix's first case (keep U_1 L_11 + U_2 L_21, i.e. C V_1) computed
    # from the ULV factors gives the right-to-left TT-URV of Alg. 3 exactly
    A = synth.gaussian_tt((9, 10, 11, 8), (1, 3, 4, 3, 1), rel_noise=1e-3, seed=2, dtype=np.float64)
    u = tt.tt_utv(A, eps=1e-2, variant="URV", l_full=l_full)
    f = tt.tt_ulv_rl(A, eps=1e-2, lhat="full", l_full=l_full)
    assert f["ranks"] == u["ranks"]
    nA = np.sqrt(u["normA2"])
    assert np.abs(tt.tt_full(u["cores"]) - tt.tt_full(f["cores"])).max() <= 1e-12 * nA
    np.testing.assert_allclose(f["tails"], u["tails"], rtol=1e-9, atol=1e-14 * u["normA2"])


def test_alg4_l11_error_is_its_residual_and_exceeds_the_projection():
    # d = 2: one truncation, A_hat = U_1 L_11 V_1^T; its squared error is the
    # reported tail ||L||^2 - ||L_11||^2 and is no smaller than that of the
    # orthogonal projection C V_1 V_1^T with the same V_1
    rng = np.random.default_rng(8)
    A = rng.standard_normal((30, 6)) @ rng.standard_normal((6, 25)) + 0.05 * rng.standard_normal((30, 25))
    for r in (2, 4, 6):
        l = tt.tt_ulv_rl(A, ranks=[r], lhat="l11")
        f = tt.tt_ulv_rl(A, ranks=[r], lhat="full")
        e_l = float(np.sum((A - tt.tt_full(l["cores"])) ** 2))
        e_f = float(np.sum((A - tt.tt_full(f["cores"])) ** 2))
        assert e_l == pytest.approx(l["tails"][0], rel=1e-10)
        assert e_f == pytest.approx(f["tails"][0], rel=1e-10)
        assert e_l >= e_f * (1 - 1e-12)


@pytest.mark.parametrize("l_full", [256, 6])
def test_alg4_l11_proposition_bound(l_full):
    # ||A - A_hat|| <= sum_k ||E_k|| <= eps ||A|| with eps_k = eps ||A|| / (d-1)
    A = synth.gaussian_tt((9, 10, 11, 8), (1, 3, 4, 3, 1), rel_noise=1e-2, seed=4, dtype=np.float64)
    for eps in (3e-2, 1e-1):
        l = tt.tt_ulv_rl(A, eps=eps, lhat="l11", l_full=l_full)
        nA = np.sqrt(l["normA2"])
        err = tt.rse(A, l["cores"]) * nA
        bound = sum(np.sqrt(l["tails"]))
        assert err <= bound * (1 + 1e-10)
        assert all(t <= dl * (1 + 1e-12) for t, dl in zip(l["tails"], l["delta2"]))
        assert bound <= eps * nA * (1 + 1e-12)
        assert max(right_orth_err(g) for g in l["cores"][1:]) < 1e-12


def test_alg4_l11_exact_recovery():
    A = synth.gaussian_tt((6, 7, 5, 6), (1, 2, 3, 2, 1), rel_noise=0.0, seed=12, dtype=np.float64)
    l = tt.tt_ulv_rl(A, eps=1e-8, lhat="l11")
    assert l["ranks"] == [1, 2, 3, 2, 1]
    assert tt.rse(A, l["cores"]) < 1e-12

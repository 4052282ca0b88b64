"""Riemannian gradient completion (Sec. 4.2.2) on the GPU against the FP64
oracle: the two-frame masked backward, the tangent-space projection with its
gauge, the block TT of the tangent vector, and whole descents (an exactly
low-rank tensor, whose iterates follow the oracle's, and the completion
workload's 256 x 256 x 64 blob volume with 70% of its entries removed, with
TT-URV, TT-ULV and TT-SVD retractions).

Error bounds: an FP32 sum of m products errs by at most about m u times the
same sum of absolute values (u = 2^-24), so the backward is checked against
depth * u * (the oracle on |cores| and |z|), depth the longest reduction on
the path; the gauge adds one FP32 rounding of each entry of U (U^T Y), so the
projection's bound adds (r + 2) u |U| |U^T Y| (computed by the oracle).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import rgrad as org
from oracle import tt as otc
from test_gpu_parity import tu  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _frames32(dims, ranks, seed):
    X = [np.asarray(c, np.float64) / np.sqrt(c.shape[0]) for c in
         synth.gaussian_cores(dims, ranks, seed=seed)]
    L = [c.astype(np.float32) for c in org.left_orthogonal(X)]
    R = [c.astype(np.float32) for c in org.right_orthogonal(X)]
    return L, R


def _dev(cs):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cs]


MIXED_CASES = {
    "d3_stored_rows": ((9, 11, 13), (1, 3, 5, 1), 1283),
    "d3_chained": ((9, 6, 41), (1, 8, 40, 1), 900),
    "d4": ((7, 5, 9, 4), (1, 3, 4, 2, 1), 700),
    "d2": ((40, 30), (1, 6, 1), 500),
    "d4_rank64": ((8, 8, 8, 8), (1, 8, 64, 8, 1), 600),
}


@pytest.mark.parametrize("name", sorted(MIXED_CASES))
def test_mixed_backward_matches_oracle(tu, name):
    dims, ranks, n = MIXED_CASES[name]
    idx = synth.random_indices(dims, n, seed=71 + len(name))
    L, R = _frames32(dims, ranks, 72)
    g = np.random.default_rng(73).standard_normal(n).astype(np.float32)
    plan = tu.EvalPlan(dims, ranks, torch.from_numpy(idx).cuda())
    got = plan.backward(_dev(L), torch.from_numpy(g).cuda(), right=_dev(R))
    L64, R64 = [c.astype(np.float64) for c in L], [c.astype(np.float64) for c in R]
    ref = org.mixed_eval_grad(L64, R64, idx, g.astype(np.float64))
    mag = org.mixed_eval_grad([np.abs(c) for c in L64], [np.abs(c) for c in R64], idx,
                              np.abs(g).astype(np.float64))
    multi = np.unravel_index(idx, dims)
    depth = sum(ranks) + 8
    for k, (a, r, m) in enumerate(zip(got, ref, mag)):
        most = int(np.bincount(multi[k], minlength=dims[k]).max())
        bound = (depth + most) * U32 * m + 1e-30
        assert np.all(np.abs(a.double().cpu().numpy() - r) <= bound), (name, k)
    # the same set on both sides is the plain backward, bit for bit
    same = plan.backward(_dev(L), torch.from_numpy(g).cuda(), right=_dev(L))
    for a, b in zip(same, plan.backward(_dev(L), torch.from_numpy(g).cuda())):
        assert torch.equal(a, b)


@pytest.mark.parametrize("name", ["d3_stored_rows", "d4", "d2", "d4_rank64"])
def test_tangent_projection_matches_oracle(tu, name):
    dims, ranks, n = MIXED_CASES[name]
    idx = synth.random_indices(dims, n, seed=81 + len(name))
    L, R = _frames32(dims, ranks, 82)
    z = np.random.default_rng(83).standard_normal(n).astype(np.float32)
    plan = tu.EvalPlan(dims, ranks, torch.from_numpy(idx).cuda())
    stale = [torch.full_like(c, 7.0) for c in _dev(L)]
    dU = plan.tangent_project(_dev(L), _dev(R), torch.from_numpy(z).cuda(), out=stale)
    assert dU[0].data_ptr() == stale[0].data_ptr()          # overwritten in place
    L64, R64 = [c.astype(np.float64) for c in L], [c.astype(np.float64) for c in R]
    Z = np.zeros(int(np.prod(dims)))
    np.add.at(Z, idx, z.astype(np.float64))
    ref = org.tangent_project(L64, R64, Z.reshape(dims))
    Y = org.mixed_eval_grad(L64, R64, idx, z.astype(np.float64))
    mag = org.mixed_eval_grad([np.abs(c) for c in L64], [np.abs(c) for c in R64], idx,
                              np.abs(z).astype(np.float64))
    multi = np.unravel_index(idx, dims)
    depth = sum(ranks) + 8
    for k in range(len(dims)):
        most = int(np.bincount(multi[k], minlength=dims[k]).max())
        bound = (depth + most) * U32 * mag[k]
        if k < len(dims) - 1:
            ul = np.abs(L64[k].reshape(-1, ranks[k + 1]))
            s_abs = np.abs(L64[k].reshape(-1, ranks[k + 1]).T @ Y[k].reshape(ul.shape[0], -1))
            s_mag = ul.T @ mag[k].reshape(ul.shape[0], -1)
            gauge = (ranks[k + 1] + 2) * U32 * (ul @ s_abs) + (depth + most) * U32 * (ul @ s_mag)
            bound = bound + gauge.reshape(bound.shape)
        got = dU[k].double().cpu().numpy()
        assert np.all(np.abs(got - ref[k]) <= bound + 1e-30), (name, k)
        if k < len(dims) - 1:
            # the gauge, on the scale of Y_k (dU_k itself vanishes when the
            # left unfolding is square: U_k U_k^T = I)
            m = L64[k].reshape(-1, ranks[k + 1])
            gk = got.reshape(m.shape[0], -1)
            assert np.abs(m.T @ gk).max() <= 1e-5 * np.abs(Y[k]).max()


def _interfaces(cores, side):
    """Gauge-invariant spans: the projectors onto the column spaces of the
    left interfaces G_1..G_k ((I_1..I_k) x r_k) or onto the row spaces of the
    right interfaces G_k..G_d (r_{k-1} x (I_k..I_d))."""
    out = []
    d = len(cores)
    if side == "left":
        L = np.ones((1, 1))
        for k in range(d - 1):
            g = cores[k]
            L = (L @ g.reshape(g.shape[0], -1)).reshape(-1, g.shape[2])
            out.append(L)
    else:
        R = np.ones((1, 1))
        for k in range(d - 1, 0, -1):
            g = cores[k]
            R = (g.reshape(-1, g.shape[2]) @ R).reshape(g.shape[0], -1)
            out.append(R.T)
    return out


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_orthogonalize_matches_oracle(tu, dtype):
    """Both sides, against the oracle's Householder frames: the same tensor,
    orthonormal unfoldings, and the same nested interface spans (a
    left-orthogonal TT is unique up to an orthogonal change of basis between
    neighbouring cores, so the spans are what is unique); the shape has a
    rank-64 core whose left unfolding is square."""
    dims, ranks = (8, 8, 8, 8), (1, 8, 64, 8, 1)
    X = [np.asarray(c, np.float64) / np.sqrt(c.shape[0]) for c in
         synth.gaussian_cores(dims, ranks, seed=90)]
    Xd = [c.astype(dtype) for c in X]
    X64 = [c.astype(np.float64) for c in Xd]
    full = otc.tt_full(X64)
    tol = 1e-5 if dtype == np.float32 else 1e-12
    for side, ref in (("left", org.left_orthogonal(X64)), ("right", org.right_orthogonal(X64))):
        got = [g.double().cpu().numpy() for g in tu.tt_orthogonalize(_dev(Xd), side)]
        assert np.abs(otc.tt_full(got) - full).max() <= tol * np.abs(full).max(), side
        ks = range(len(dims) - 1) if side == "left" else range(1, len(dims))
        for k in ks:
            if side == "left":
                a = got[k].reshape(-1, ranks[k + 1])
            else:
                a = got[k].reshape(ranks[k], -1).T
            assert np.abs(a.T @ a - np.eye(a.shape[1])).max() <= tol, (side, k)
        for a, b in zip(_interfaces(got, side), _interfaces(ref, side)):
            assert np.abs(a @ a.T - b @ b.T).max() <= 10 * tol, side


def test_orthogonalize_rejects_bad_arguments(tu):
    g = [torch.zeros(1, 3, 5, device="cuda"), torch.zeros(5, 2, 1, device="cuda")]
    with pytest.raises(tu.TTError) as ei:      # r_1 = 5 > r_0 I_1 = 3
        tu.tt_orthogonalize(g, "left")
    assert ei.value.status == tu.TT_EINVAL
    with pytest.raises(tu.TTError) as ei:      # r_1 = 5 > I_2 r_2 = 2
        tu.tt_orthogonalize(g, "right")
    assert ei.value.status == tu.TT_EINVAL


@pytest.mark.parametrize("name", sorted(MIXED_CASES))
def test_tangent_eval_matches_oracle(tu, name):
    """P_Omega of the tangent vector sum_k U_<k dU_k V_>k against the oracle's
    block TT of it contracted in full (FP64)."""
    dims, ranks, n = MIXED_CASES[name]
    idx = synth.random_indices(dims, n, seed=91 + len(name))
    L, R = _frames32(dims, ranks, 92)
    dU = [np.random.default_rng(93 + k).standard_normal(c.shape).astype(np.float32)
          for k, c in enumerate(L)]
    plan = tu.EvalPlan(dims, ranks, torch.from_numpy(idx).cuda())
    got = plan.tangent_eval(_dev(L), _dev(R), _dev(dU)).double().cpu().numpy()
    L64, R64, d64 = ([c.astype(np.float64) for c in x] for x in (L, R, dU))
    ref = otc.tt_full(org.tangent_cores(L64, R64, d64)).reshape(-1)[idx]
    mag = otc.tt_full(org.tangent_cores([np.abs(c) for c in L64], [np.abs(c) for c in R64],
                                        [np.abs(c) for c in d64])).reshape(-1)[idx]
    depth = sum(ranks) + 8 + len(dims)
    assert np.all(np.abs(got - ref) <= depth * U32 * mag + 1e-30), name


def test_rgrad_ranks_above_32(tu):
    """Ranks the rank-2r block TT could not take (r_1 = 40 > 32): the first
    iterations follow the oracle's, and the loss falls."""
    from paper_2501_07904_gb300.completion import rgrad

    dims, ranks = (48, 40, 30), (1, 40, 12, 1)
    T = otc.tt_full([np.asarray(c, np.float64) for c in synth.gaussian_cores(dims, ranks, seed=94)])
    T = (T / np.abs(T).max()).astype(np.float32)
    idx = np.sort(np.random.default_rng(95).choice(T.size, T.size // 2, replace=False))
    vals = T.reshape(-1)[idx]
    _, losses, _ = rgrad(torch.from_numpy(vals).cuda(), torch.from_numpy(idx).cuda(), dims,
                         ranks[1:-1], steps=8, retraction="URV")
    _, ref = org.rgrad(vals.astype(np.float64), idx, dims, ranks, steps=3, variant="URV")
    for t in range(4):
        assert losses[t] == pytest.approx(ref[t], rel=2e-3), t
    assert losses[-1] < 0.1 * losses[0]


def test_tangent_projection_empty_index_set(tu):
    dims, ranks = (4, 5, 3), (1, 2, 3, 1)
    L, R = _frames32(dims, ranks, 84)
    plan = tu.EvalPlan(dims, ranks, torch.zeros(0, dtype=torch.int64, device="cuda"))
    dU = plan.tangent_project(_dev(L), _dev(R), torch.zeros(0, device="cuda"),
                              out=[torch.full_like(c, 3.0) for c in _dev(L)])
    assert all(float(g.abs().sum()) == 0.0 for g in dU)


def test_block_cores_represent_the_tangent_vector(tu):
    from paper_2501_07904_gb300.completion import tangent_block_cores

    dims, ranks = (6, 5, 7, 4), (1, 3, 4, 2, 1)
    L, R = _frames32(dims, ranks, 85)
    L64, R64 = [c.astype(np.float64) for c in L], [c.astype(np.float64) for c in R]
    dU = [np.random.default_rng(86 + k).standard_normal(c.shape) for k, c in enumerate(L)]
    for alpha in (None, 0.25):
        got = tu.tt_full(tangent_block_cores(_dev(L), _dev(R), _dev([d.astype(np.float32) for d in dU]),
                                             alpha)).double().cpu().numpy()
        ref = otc.tt_full(org.tangent_cores(L64, R64, [d.astype(np.float32).astype(np.float64)
                                                        for d in dU],
                                            alpha=alpha or 0.0, with_point=alpha is not None))
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_rgrad_follows_the_oracle_on_a_low_rank_tensor(tu):
    from paper_2501_07904_gb300.completion import rgrad

    dims, ranks = (20, 24, 16), (1, 3, 4, 1)
    T = otc.tt_full([np.asarray(c, np.float64) for c in synth.gaussian_cores(dims, ranks, seed=87)])
    T = (T / np.abs(T).max()).astype(np.float32)
    idx = np.sort(np.random.default_rng(88).choice(T.size, T.size // 2, replace=False))
    vals = T.reshape(-1)[idx]
    cores, losses, alphas = rgrad(torch.from_numpy(vals).cuda(), torch.from_numpy(idx).cuda(),
                                  dims, ranks[1:-1], steps=30, retraction="URV")
    _, ref_losses = org.rgrad(vals.astype(np.float64), idx, dims, ranks, steps=30, variant="URV")
    # the first iterates follow the oracle's; later ones reach the FP32 floor
    for t in range(6):
        assert losses[t] == pytest.approx(ref_losses[t], rel=2e-3), t
    assert losses[-1] <= 1e-8 * losses[0]
    assert all(a > 0 for a in alphas)
    c64 = [c.double().cpu().numpy() for c in cores]
    assert otc.rse(T.astype(np.float64), c64) < 1e-4


def _psnr(x, truth):
    mse = float(((x - truth) ** 2).mean())
    return 10.0 * np.log10(float(truth.abs().max()) ** 2 / mse)


def test_rgrad_c4_retractions(tu):
    """The completion workload with each retraction: 40 iterations from the
    spectral initialisation.  The loss falls, the error on the full volume
    falls, and both TT-UTV retractions end at an RSE no worse than the TT-SVD
    retraction's (Sec. 4.2.2 finds them as effective; on this volume TT-URV
    reached 0.043, TT-ULV 0.046 and TT-SVD 0.070 after 40 iterations)."""
    from paper_2501_07904_gb300.completion import rgrad

    cfg = synth.CONFIGS["c4"]
    shape = cfg["shape"]
    M = synth.make_config("c4")
    idx = synth.observation_mask(shape, cfg["p_obs"], cfg["mask_seed"])
    v_t = torch.from_numpy(np.ascontiguousarray(M.reshape(-1)[idx])).cuda()
    i_t = torch.from_numpy(idx).cuda()
    truth = torch.from_numpy(M).cuda().double()
    ranks = cfg["ranks"][1:-1]
    final = {}
    for method in ("URV", "ULV", "SVD"):
        rses = []

        def record(t, cores):
            x = tu.tt_full(cores).double()
            rses.append(float(torch.linalg.vector_norm(x - truth) / torch.linalg.vector_norm(truth)))

        cores, losses, alphas = rgrad(v_t, i_t, shape, ranks, steps=40, retraction=method,
                                      callback=record)
        assert losses[-1] <= 0.5 * losses[0], method
        assert rses[-1] <= 0.8 * rses[0], method
        x = tu.tt_full(cores).double()
        final[method] = (rses[-1], _psnr(x, truth))
        print(method, "RSE", rses[0], "->", rses[-1], "PSNR", final[method][1],
              "loss", losses[0], "->", losses[-1])
    for method in ("URV", "ULV"):
        assert final[method][0] <= 1.05 * final["SVD"][0], final


def test_rgrad_c4_first_iterations_match_the_oracle(tu):
    """At the completion workload's full size: the losses of the spectral
    initialisation and of the first two TT-URV iterations equal the FP64
    oracle's run of the same iteration (dense tangent projection, oracle
    TT-URV retraction; about 20 s on the host)."""
    from paper_2501_07904_gb300.completion import rgrad

    cfg = synth.CONFIGS["c4"]
    shape = cfg["shape"]
    M = synth.make_config("c4")
    idx = synth.observation_mask(shape, cfg["p_obs"], cfg["mask_seed"])
    vals = np.ascontiguousarray(M.reshape(-1)[idx])
    _, losses, _ = rgrad(torch.from_numpy(vals).cuda(), torch.from_numpy(idx).cuda(), shape,
                         cfg["ranks"][1:-1], steps=2, retraction="URV")
    _, ref = org.rgrad(vals.astype(np.float64), idx, shape, cfg["ranks"], steps=2, variant="URV")
    for a, b in zip(losses, ref):
        assert a == pytest.approx(b, rel=1e-4)

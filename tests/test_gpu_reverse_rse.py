"""The index-reversed sweep (tt_opts.reverse, Remark after Thm 3.2) and the
streamed reconstruction error tt_rse (Sec. 4's RSE), through the C ABI,
against the FP64 oracle.

Reverse: the oracle factors the index-reversed tensor itself and its cores
are read back as cores of A here (core k of A = core d+1-k of the reversed
tensor with its rank axes swapped); the GPU result must match that in ranks,
represented tensor, per-unfolding errors and orthogonality (a right-to-left
TT-URV of the reversed tensor is left-orthogonal for A).

tt_rse: compared with ||A - A_TT||^2 and ||A||^2 formed in FP64 by the
oracle's contraction of the same cores, on shapes that take one slab, several
slabs with a ragged last one, and a single first-mode slice larger than a slab.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import tt as otc
from test_gpu_parity import np_cores, orth_err, rel_diff, tu  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

RAGGED = synth.gaussian_tt((37, 29, 41, 23), (1, 5, 7, 4, 1), rel_noise=1e-6, seed=5,
                           dtype=np.float64)


def reversed_oracle(A, method, **kw):
    d = A.ndim
    Ar = np.ascontiguousarray(np.transpose(A, tuple(range(d - 1, -1, -1))))
    ref = otc.tt_utv(Ar, variant=method, **kw)
    cores = [np.ascontiguousarray(np.transpose(ref["cores"][d - 1 - k], (2, 1, 0)))
             for k in range(d)]
    return dict(cores=cores, ranks=ref["ranks"][::-1], tails=ref["tails"][::-1],
                normA2=ref["normA2"])


@pytest.mark.parametrize("precision, tol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("method", ["URV", "ULV"])
@pytest.mark.parametrize("l_full", [256, 24])
def test_reverse_adaptive(tu, precision, tol, method, l_full):
    A = RAGGED if precision == "fp64" else RAGGED.astype(np.float32)
    res = tu.tt_utv(torch.from_numpy(A).cuda(), eps=1e-3, variant=method, precision=precision,
                    l_full=l_full, reverse=True)
    ref = reversed_oracle(np.asarray(A, np.float64), method, eps=1e-3, l_full=l_full)
    normA2 = ref["normA2"]
    assert res.ranks == ref["ranks"], (res.ranks, ref["ranks"])
    assert [tuple(g.shape) for g in res.cores] == [g.shape for g in ref["cores"]]
    diff = rel_diff(np_cores(res), ref["cores"], normA2)
    assert diff <= tol, diff
    for t, tr in zip(res.tail_sq, ref["tails"]):
        assert abs(t - tr) <= 50 * tol * normA2 + 1e-3 * tr
    assert res.orth == ("left" if method == "URV" else "right")
    assert orth_err(res) <= 100 * tol
    assert abs(res.norm_sq - normA2) <= 1e-6 * normA2


def test_reverse_fixed_ranks_and_weights(tu):
    A = RAGGED.astype(np.float32)
    # fixed ranks refer to the unfoldings of A, not of the reversed tensor
    res = tu.tt_utv(torch.from_numpy(A).cuda(), ranks=[3, 6, 2], reverse=True, l_full=24)
    assert res.ranks == [1, 3, 6, 2, 1]
    ref = reversed_oracle(np.asarray(A, np.float64), "URV", ranks=[2, 6, 3], l_full=24)
    assert ref["ranks"] == [1, 3, 6, 2, 1]
    assert rel_diff(np_cores(res), ref["cores"], ref["normA2"]) <= 1e-5
    # weights refer to the unfoldings of A too: the tolerances match the forward sweep's
    w = np.array([0.2, 0.9, 0.0])
    w[2] = np.sqrt(1.0 - w[0] ** 2 - w[1] ** 2)
    res = tu.tt_utv(torch.from_numpy(A).cuda(), eps=1e-2, weights=list(w), reverse=True)
    fwd = tu.tt_utv(torch.from_numpy(A).cuda(), eps=1e-2, weights=list(w))
    assert res.ranks == fwd.ranks
    for a, b, wk in zip(res.delta_sq, fwd.delta_sq, w):
        assert a == pytest.approx(b, rel=1e-6)
        assert a == pytest.approx((wk * 1e-2) ** 2 * fwd.norm_sq, rel=1e-6)


def test_reverse_host_input(tu):
    A = RAGGED.astype(np.float32)
    dev = tu.tt_utv(torch.from_numpy(A).cuda(), eps=1e-3, reverse=True)
    host = tu.tt_utv(torch.from_numpy(A).pin_memory(), eps=1e-3, reverse=True)
    assert dev.ranks == host.ranks
    for a, b in zip(dev.cores, host.cores):
        assert torch.equal(a, b)


def _rse_case(tu, dims, ranks, dtype, seed):
    cores = synth.gaussian_cores(dims, ranks, seed)
    rng = np.random.default_rng(seed + 1)
    A = synth.contract_cores(cores) + 1e-3 * rng.standard_normal(dims)
    npdt = np.float64 if dtype == torch.float64 else np.float32
    A = A.astype(npdt)
    cores = [c.astype(npdt) for c in cores]
    A_t = torch.from_numpy(A).cuda()
    err2, norm2 = tu.tt_rse(A_t, [torch.from_numpy(c).cuda() for c in cores])
    D = otc.tt_full([c.astype(np.float64) for c in cores]) - A.astype(np.float64)
    return err2, norm2, float(np.sum(D * D)), float(np.sum(A.astype(np.float64) ** 2))


@pytest.mark.parametrize("dims, ranks", [
    ((37, 29, 41, 23), (1, 5, 7, 4, 1)),           # one slab
    ((300, 256, 256), (1, 6, 5, 1)),               # slabs of 256 slices, the last one of 44
    ((2, 4096, 4200), (1, 2, 2, 1)),               # one slice (17.2M entries) larger than a slab
])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_rse_streamed(tu, dims, ranks, dtype):
    err2, norm2, err2_ref, norm2_ref = _rse_case(tu, dims, ranks, dtype, seed=11)
    tol = 1e-12 if dtype == torch.float64 else 1e-6
    assert abs(norm2 - norm2_ref) <= tol * norm2_ref
    # the FP32 contraction rounds each entry of A_TT once (~6e-8 relative)
    assert abs(err2 - err2_ref) <= 1e-4 * err2_ref
    assert err2_ref > 0


def test_rse_matches_sweep_tails(tu):
    A = torch.from_numpy(RAGGED).cuda()
    res = tu.tt_utv(A, eps=1e-3, precision="fp64")
    err2, norm2 = tu.tt_rse(A, res.cores)
    # Thm 3.1 / 3.2: ||A - A_TT||^2 = sum of the per-unfolding errors
    assert abs(err2 - sum(res.tail_sq)) <= 1e-8 * norm2
    assert norm2 == pytest.approx(res.norm_sq, rel=1e-12)

"""TT-URV / TT-ULV with the Givens-based low-rank URV inner factor (the
Fierro-Hansen family the paper runs inside TT-URV in Sec. 4), warm-started
from a pivoted QR, on the GPU against the FP64 oracle's `lurv`: ranks equal,
the represented tensors equal to the data's precision, the bound RSE <= eps of
Alg. 2 and the equality inside the proof of Thm 3.1 (RSE^2 ||A||^2 = sum of
the step errors), on exact, sketched, fixed-rank and rank-deficient steps, in
FP64 and FP32, and for several power-iteration counts.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import tt as otc
from test_gpu_parity import tu  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _gpu(tu, A, **kw):
    res = tu.tt_utv(torch.from_numpy(A).cuda(), inner="lurv", **kw)
    return res, [g.double().cpu().numpy() for g in res.cores]


def _diff(c1, c2, A):
    return np.linalg.norm(otc.tt_full(c1) - otc.tt_full(c2)) / np.linalg.norm(A)


@pytest.mark.parametrize("variant", ["URV", "ULV"])
@pytest.mark.parametrize("eps", [1e-2, 1e-4])
def test_lurv_fp64_matches_oracle(tu, variant, eps):
    A = synth.gaussian_tt((6, 7, 8, 5), (1, 3, 4, 2, 1), 1e-3, seed=21, dtype=np.float64)
    res, cores = _gpu(tu, A, eps=eps, variant=variant, precision="fp64")
    ref = otc.tt_utv(A, eps=eps, variant=variant, inner="lurv")
    assert res.ranks == ref["ranks"]
    assert _diff(cores, ref["cores"], A) <= 1e-10
    rse = otc.rse(A, cores)
    assert rse <= eps
    assert abs(rse ** 2 * res.norm_sq - sum(res.tail_sq)) <= 1e-9 * res.norm_sq
    for a, b in zip(res.tail_sq, ref["tails"]):
        assert abs(a - b) <= 1e-10 * res.norm_sq


@pytest.mark.parametrize("variant", ["URV", "ULV"])
def test_lurv_fp32_matches_oracle(tu, variant):
    A = synth.gaussian_tt((16, 16, 16, 16), (1, 4, 4, 4, 1), 1e-3, seed=22, dtype=np.float32)
    A64 = A.astype(np.float64)
    res, cores = _gpu(tu, A, eps=1e-2, variant=variant, precision="fp32")
    ref = otc.tt_utv(A64, eps=1e-2, variant=variant, inner="lurv")
    assert res.ranks == ref["ranks"] == [1, 4, 4, 4, 1]
    assert _diff(cores, ref["cores"], A64) <= 1e-5
    assert otc.rse(A64, cores) <= 1e-2


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_lurv_sketched_fixed_ranks(tu, precision):
    dt = np.float64 if precision == "fp64" else np.float32
    A = synth.gaussian_tt((4, 5, 300), (1, 3, 4, 1), 1e-4, seed=23, dtype=dt)
    A64 = A.astype(np.float64)
    res, cores = _gpu(tu, A, ranks=[3, 4], variant="URV", precision=precision)
    ref = otc.tt_utv(A64, ranks=[3, 4], variant="URV", inner="lurv")
    assert res.ranks == ref["ranks"] == [1, 3, 4, 1]
    assert res.sketch_l[1] > 0                      # the 300-wide step is sketched
    assert _diff(cores, ref["cores"], A64) <= (1e-10 if precision == "fp64" else 1e-5)


def test_lurv_wide_trapezoidal_step(tu):
    # the first step factors the 120 x 200 unfolding exactly (a 200-wide Gram
    # of rank 120: R upper trapezoidal, more columns than rows); the second is
    # sketched
    A = synth.gaussian_tt((3, 40, 200), (1, 3, 10, 1), 1e-3, seed=24, dtype=np.float64)
    for variant in ("URV", "ULV"):
        res, cores = _gpu(tu, A, eps=2e-3, variant=variant, precision="fp64")
        ref = otc.tt_utv(A, eps=2e-3, variant=variant, inner="lurv")
        assert res.ranks == ref["ranks"], variant
        assert _diff(cores, ref["cores"], A) <= 1e-10, variant
        assert otc.rse(A, cores) <= 2e-3


def test_lurv_rank_deficient_and_fixed_rank_above_it(tu):
    # an exactly TT-structured tensor: the pivoted Cholesky stops early, and a
    # fixed rank above the unfolding's rank is completed from the pivot columns.
    # (eps stays above the Gram's rounding floor, ~1e-8 in norm in FP64.)
    A = synth.gaussian_tt((5, 6, 7, 4), (1, 2, 3, 2, 1), 0.0, seed=25, dtype=np.float64)
    res, cores = _gpu(tu, A, eps=1e-6, variant="URV", precision="fp64")
    assert res.ranks == [1, 2, 3, 2, 1]
    assert otc.rse(A, cores) < 1e-7
    res, cores = _gpu(tu, A, ranks=[4, 5, 3], variant="ULV", precision="fp64")
    assert res.ranks == [1, 4, 5, 3, 1]
    assert otc.rse(A, cores) < 1e-7


def test_lurv_iteration_count_changes_the_basis_not_the_bounds(tu):
    A = synth.gaussian_tt((8, 9, 10), (1, 5, 6, 1), 3e-2, seed=26, dtype=np.float64)
    for q in (0, 2, 16):
        res = tu.tt_utv(torch.from_numpy(A).cuda(), eps=5e-2, variant="URV", inner="lurv",
                        usvp_iters=q, precision="fp64")
        ref = otc.tt_utv(A, eps=5e-2, variant="URV", inner="lurv", usvp_q=q)
        cores = [g.double().cpu().numpy() for g in res.cores]
        assert res.ranks == ref["ranks"], q
        assert _diff(cores, ref["cores"], A) <= 1e-10, q
        assert otc.rse(A, cores) <= 5e-2


def test_lurv_rejects_bad_options(tu):
    A = torch.ones(4, 5, 6, device="cuda")
    with pytest.raises(tu.TTError) as ei:
        tu.tt_utv(A, eps=1e-2, inner="lurv", usvp_iters=-1)
    assert ei.value.status == tu.TT_EINVAL
    with pytest.raises(tu.TTError) as ei:
        tu.tt_utv(A, eps=1e-2, variant="ULV", direction="RL", inner="lurv", lhat="l11")
    assert ei.value.status == tu.TT_EINVAL

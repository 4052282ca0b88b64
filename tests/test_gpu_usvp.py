"""TT-ULV / TT-URV with the USV-plus-style inner factor (the deflation the
paper runs inside TT-ULV in Sec. 4) on the GPU against the FP64 oracle's
`usv_plus`: ranks equal, the represented tensors equal to the data's
precision, the bound RSE <= eps of Alg. 2 and the equality inside the proof
of Thm 3.1 (RSE^2 ||A||^2 = sum of the step errors), on exact, sketched and
fixed-rank steps, in FP64 and FP32.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import tt as otc
from test_gpu_parity import tu  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _gpu(tu, A, **kw):
    res = tu.tt_utv(torch.from_numpy(A).cuda(), inner="usvp", **kw)
    return res, [g.double().cpu().numpy() for g in res.cores]


def _diff(c1, c2, A):
    return np.linalg.norm(otc.tt_full(c1) - otc.tt_full(c2)) / np.linalg.norm(A)


@pytest.mark.parametrize("variant", ["ULV", "URV"])
@pytest.mark.parametrize("eps", [1e-2, 1e-4])
def test_usvp_fp64_matches_oracle(tu, variant, eps):
    A = synth.gaussian_tt((6, 7, 8, 5), (1, 3, 4, 2, 1), 1e-3, seed=11, dtype=np.float64)
    res, cores = _gpu(tu, A, eps=eps, variant=variant, precision="fp64")
    ref = otc.tt_utv(A, eps=eps, variant=variant, inner="usvp")
    assert res.ranks == ref["ranks"]
    assert _diff(cores, ref["cores"], A) <= 1e-10
    rse = otc.rse(A, cores)
    assert rse <= eps
    assert abs(rse ** 2 * res.norm_sq - sum(res.tail_sq)) <= 1e-9 * res.norm_sq


@pytest.mark.parametrize("variant", ["ULV", "URV"])
def test_usvp_fp32_matches_oracle(tu, variant):
    A = synth.gaussian_tt((16, 16, 16, 16), (1, 4, 4, 4, 1), 1e-3, seed=12, dtype=np.float32)
    A64 = A.astype(np.float64)
    res, cores = _gpu(tu, A, eps=1e-2, variant=variant, precision="fp32")
    ref = otc.tt_utv(A64, eps=1e-2, variant=variant, inner="usvp")
    assert res.ranks == ref["ranks"] == [1, 4, 4, 4, 1]
    assert _diff(cores, ref["cores"], A64) <= 1e-5
    assert otc.rse(A64, cores) <= 1e-2


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_usvp_sketched_fixed_ranks(tu, precision):
    dt = np.float64 if precision == "fp64" else np.float32
    A = synth.gaussian_tt((4, 5, 300), (1, 3, 4, 1), 1e-4, seed=13, dtype=dt)
    A64 = A.astype(np.float64)
    res, cores = _gpu(tu, A, ranks=[3, 4], variant="URV", precision=precision)
    ref = otc.tt_utv(A64, ranks=[3, 4], variant="URV", inner="usvp")
    assert res.ranks == ref["ranks"] == [1, 3, 4, 1]
    assert res.sketch_l[1] > 0                      # the 300-wide step is sketched
    assert _diff(cores, ref["cores"], A64) <= (1e-10 if precision == "fp64" else 1e-5)


def test_usvp_iteration_count_changes_the_basis_not_the_bounds(tu):
    A = synth.gaussian_tt((8, 9, 10), (1, 5, 6, 1), 3e-2, seed=14, dtype=np.float64)
    for q in (0, 2, 16):
        res = tu.tt_utv(torch.from_numpy(A).cuda(), eps=5e-2, variant="ULV", inner="usvp",
                        usvp_iters=q, precision="fp64")
        ref = otc.tt_utv(A, eps=5e-2, variant="ULV", inner="usvp", usvp_q=q)
        cores = [g.double().cpu().numpy() for g in res.cores]
        assert res.ranks == ref["ranks"], q
        assert _diff(cores, ref["cores"], A) <= 1e-10, q
        assert otc.rse(A, cores) <= 5e-2


def test_usvp_rejects_bad_options(tu):
    A = torch.ones(4, 5, 6, device="cuda")
    with pytest.raises(tu.TTError) as ei:
        tu.tt_utv(A, eps=1e-2, inner="usvp", usvp_iters=65)
    assert ei.value.status == tu.TT_EINVAL

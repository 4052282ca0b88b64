"""Table (tab: Beps), Example 2 of Sec. 4.1, on the GPU: the 160^4 tensor
B(i) = sin(sqrt(sum_k ((i_k - 1)/(I - 1))^2)) decomposed at eps = 1e-2 .. 1e-5
by TT-SVD left-to-right, TT-ULV left-to-right and TT-URV right-to-left must
give the printed ranks (tests/golden/beps_ranks.txt) with a relative error
below eps.  After the first step the basis side is r_{k-1} 160 (left to
right) or 160 r_k (right to left), above 256 once r >= 2, so those steps take
the sketch path (TT-SVD included: a Jacobi SVD of the projected block)."""
import pytest
import torch

import synth
from test_gpu_parity import tu  # noqa: F401  (fixture)
from test_oracle_beps import load_gold

pytestmark = pytest.mark.gpu
EPS = (1e-2, 1e-3, 1e-4, 1e-5)


@pytest.fixture(scope="module")
def B32():
    return synth.example2_torch(160, 4, "cuda", torch.float32).contiguous()


def _check(tu, B, res, eps, want):
    assert tuple(res.ranks[1:-1]) == want, (eps, res.ranks, want)
    err2, norm2 = tu.tt_rse(B, res.cores)
    assert (err2 / norm2) ** 0.5 < eps


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("method", ["TT-SVD", "TT-ULV(lulv)", "TT-URV(lurv)"])
def test_table_beps_on_gpu(tu, B32, method, precision):
    gold = load_gold()
    for eps in EPS:
        if method == "TT-SVD":
            res = tu.tt_svd(B32, eps=eps, direction="LR", precision=precision)
        else:
            res = tu.tt_utv(B32, eps=eps, variant="ULV" if "ULV" in method else "URV",
                            precision=precision)
        _check(tu, B32, res, eps, gold[(eps, method)])


def test_table_beps_tt_svd_fp64(tu):
    gold = load_gold()
    B = synth.example2_torch(160, 4, "cuda", torch.float64).contiguous()
    for eps in EPS:
        res = tu.tt_svd(B, eps=eps, direction="LR", precision="fp64")
        _check(tu, B, res, eps, gold[(eps, "TT-SVD")])

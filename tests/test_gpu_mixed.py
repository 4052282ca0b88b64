"""Mixed precision (TT_P_MIXED: tcgen05 tensor cores, TF32 operands) against
the FP64 oracle.

What is unique is compared as in test_gpu_parity: ranks, the represented
tensor, RSE, the error equality of Thm 3.1/3.2 and the orthogonality of the
cores.  Tolerance 5e-5 relative to ||A||_F: the range-finding products
(Gram of an exact step, Cholesky-QR Grams, Gram of the projection) round
their operands to TF32 (2^-11), which tilts the kept subspace by a few 1e-6
on these spectra; every product that becomes part of the result carries its
operands as two TF32 terms (~2^-22).  Tight steps (eps^2 w_k^2 below
2 n u_fp32) find their range on the FP32 path and form their carries and
cores on the tensor cores; they are held to the FP32 tolerance.
"""
import os

import numpy as np
import pytest
import torch

import synth
from test_gpu_parity import (check_against_oracle, check_gold, check_tight_tails, np_cores,
                             run_gpu)

pytestmark = pytest.mark.gpu

TOL = 5e-5

# Unfoldings with leading dimensions that are multiples of 4 (tensor-core
# eligible), ragged against the 128-row tiles and 32-wide k-blocks; the
# sweep takes exact steps and sketched steps with a non-identity Omega.
ALIGNED = synth.gaussian_tt((36, 28, 41, 24), (1, 8, 12, 4, 1), 1e-3, seed=51, dtype=np.float32)


@pytest.fixture(scope="module")
def tu():
    import paper_2501_07904_gb300 as m
    if not os.path.exists(m.LIB_PATH):
        from paper_2501_07904_gb300 import build
        build.build()
    assert torch.cuda.is_available()
    m.lib()
    return m


@pytest.mark.parametrize("method", ["URV", "ULV"])
@pytest.mark.parametrize("l_full", [256, 24])
def test_mixed_aligned_adaptive(tu, method, l_full):
    res, ref = check_against_oracle(tu, ALIGNED, method, TOL, eps=1e-2, precision="mixed",
                                    l_full=l_full)
    assert res.ranks == [1, 8, 12, 4, 1]


@pytest.mark.parametrize("method", ["URV", "ULV"])
def test_mixed_fixed_ranks(tu, method):
    check_against_oracle(tu, ALIGNED, method, TOL, ranks=[6, 8, 4], precision="mixed", l_full=24)


def test_mixed_deterministic(tu):
    A = torch.from_numpy(ALIGNED).cuda()
    a = tu.tt_utv(A, eps=1e-2, precision="mixed", l_full=24)
    b = tu.tt_utv(A, eps=1e-2, precision="mixed", l_full=24)
    for x, y in zip(a.cores, b.cores):
        assert torch.equal(x, y)
    assert a.tail_sq == b.tail_sq


@pytest.mark.parametrize("method", ["URV", "ULV"])
def test_mixed_c3_tight_steps(tu, method):
    # eps = 1e-3 on 32^5 makes every step tight: Grams, sketches and
    # projections run on the SIMT path, carries and cores on the tensor cores
    # with split operands; held to the FP32 tolerance
    A = synth.make_config("c3")
    res = check_gold(tu, A, method, f"c3_{method}", 1e-5, 1e-3, precision="mixed")
    assert res.ranks == [1, 20, 20, 20, 20, 1]
    check_tight_tails(tu, A, res, method, "c3")


def test_mixed_c5_128pow4(tu):
    A = synth.make_config("c5")
    res = check_gold(tu, A, "URV", "c5_URV", 2e-5, 1e-2, precision="mixed")
    assert res.ranks == [1, 64, 64, 64, 1]

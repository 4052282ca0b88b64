"""Opt-in direct step errors (tt_opts.direct_tails): every non-tight step
reports ||E_k||_F^2 summed from its residual instead of ||C||^2 - ||carry||^2.
Checked on exact and sketched steps in FP32 and mixed precision, both sweeps:
ranks and cores unchanged (bitwise); the equality inside the proof of Thm 3.1 (and Thm
3.2), ||A - A_TT||^2 = sum of the step errors, to 3%; each step error against
the FP64 oracle's; and the 128^4 workload in mixed precision against its
stored oracle errors.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import tt as otc
from test_gpu_parity import load_gold, tu  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

# exact and sketched (non-identity Omega) steps at l_full = 24
ALIGNED = synth.gaussian_tt((36, 28, 41, 24), (1, 8, 12, 4, 1), 1e-3, seed=51, dtype=np.float32)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("method", ["URV", "ULV"])
def test_direct_tails_sum_to_the_error(tu, method, precision):
    A = torch.from_numpy(ALIGNED).cuda()
    kw = dict(eps=1e-2, variant=method, precision=precision, l_full=24)
    base = tu.tt_utv(A, **kw)
    res = tu.tt_utv(A, direct_tails=True, **kw)
    assert res.ranks == base.ranks
    assert any(l > 0 for l in res.sketch_l)
    for a, b in zip(res.cores, base.cores):
        assert torch.equal(a, b)
    err2, normA2 = tu.tt_rse(A, res.cores)
    assert abs(sum(res.tail_sq) - err2) <= 0.03 * err2, (res.tail_sq, err2)
    ref = otc.tt_utv(ALIGNED.astype(np.float64), eps=1e-2, variant=method, l_full=24)
    assert res.ranks == ref["ranks"]
    for t, t_ref in zip(res.tail_sq, ref["tails"]):
        assert abs(t - t_ref) <= 0.1 * t_ref + 1e-9 * normA2, (res.tail_sq, ref["tails"])


def test_direct_tails_c5_mixed(tu):
    A = torch.from_numpy(synth.make_config("c5")).cuda()
    res = tu.tt_utv(A, eps=1e-2, variant="URV", precision="mixed", direct_tails=True)
    g = load_gold("c5_URV")
    assert res.ranks == [int(x) for x in g["ranks"]]
    err2, normA2 = tu.tt_rse(A, res.cores)
    ratio = sum(res.tail_sq) / err2
    print(f"DIRECT c5 mixed tails/err2={ratio:.4f} tails={[t / normA2 for t in res.tail_sq]}")
    assert 0.95 <= ratio <= 1.05, ratio
    for t, t_ref in zip(res.tail_sq, g["tails"]):
        assert abs(t - float(t_ref)) <= 0.1 * float(t_ref) + 1e-10 * normA2

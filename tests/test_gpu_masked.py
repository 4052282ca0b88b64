"""Masked TT evaluation and its backward (the observation operator P_Omega of
Sec. 4.2.2 and its core gradients) against the FP64 oracle, on shapes that
exercise every path of the plan: d = 1, 2, 3 (stored per-entry rows for the
outer cores, and the chained path when r_2 > 32), 4 and 5, a mode of more than 256 slices
(two radix digits), ranks that are not multiples of 4, a 64 x 64 core (two
accumulation tiles per thread), one index repeated across every chunk (the
fix-up chain), all-distinct slices, ragged chunk tails and the empty set.

Error bounds: an FP32 sum of m products errs by at most about m u times the
same sum of absolute values (u = 2^-24), so each check compares
|gpu - oracle| with depth * u * (the oracle evaluated on |cores| and |gout|),
where depth is the longest reduction on the path (the chain's ranks plus,
for a gradient, the most entries summed into one slice).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import tt as otc
from test_gpu_parity import tu  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _cores(dims, ranks, seed):
    cs = synth.gaussian_cores(dims, ranks, seed=seed)
    return [(c / np.sqrt(c.shape[0])).astype(np.float32) for c in cs]


def _check_case(tu, dims, ranks, idx, seed):
    c32 = _cores(dims, ranks, seed)
    c64 = [c.astype(np.float64) for c in c32]
    cabs = [np.abs(c) for c in c64]
    gout = np.random.default_rng(seed + 1).standard_normal(len(idx)).astype(np.float32)
    tc = [torch.from_numpy(c).cuda() for c in c32]
    ti = torch.from_numpy(np.asarray(idx, np.int64)).cuda()
    plan = tu.EvalPlan(dims, ranks, ti)
    x = plan.at(tc).double().cpu().numpy()
    depth = sum(ranks) + 8
    if len(idx):
        ref = otc.tt_eval_at(c64, idx)
        mag = otc.tt_eval_at(cabs, idx)
        assert np.all(np.abs(x - ref) <= depth * U * mag + 1e-30)
    grads = plan.backward(tc, torch.from_numpy(gout).cuda())
    ref_g = otc.tt_eval_grad(c64, idx, gout.astype(np.float64)) if len(idx) else \
        [np.zeros_like(c) for c in c64]
    mag_g = otc.tt_eval_grad(cabs, idx, np.abs(gout).astype(np.float64)) if len(idx) else \
        [np.zeros_like(c) for c in c64]
    multi = np.unravel_index(np.asarray(idx, np.int64), dims) if len(idx) else None
    for k, (g, r, m) in enumerate(zip(grads, ref_g, mag_g)):
        most = int(np.bincount(multi[k], minlength=dims[k]).max()) if len(idx) else 0
        bound = (depth + most) * U * m + 1e-30
        assert np.all(np.abs(g.double().cpu().numpy() - r) <= bound), k
    return plan, tc, ti, gout


CASES = {
    "d4": ((7, 5, 9, 4), (1, 3, 4, 2, 1), 700),
    "d1": ((37,), (1, 1), 1000),
    "d2_two_digit_mode": ((300, 9), (1, 5, 1), 3000),
    "rank64": ((6, 5, 4, 3, 7), (1, 6, 64, 64, 7, 1), 2000),
    "ragged_ranks": ((9, 11, 13), (1, 3, 5, 1), 1283),
    "d3_wide_last_rank": ((5, 6, 7), (1, 8, 40, 1), 1500),   # d = 3 on the chained path
    "distinct_slices": ((1000, 3), (1, 7, 1), 2500),
    "long_modes": ((70000, 2, 3), (1, 4, 2, 1), 5000),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_masked_matches_oracle(tu, name):
    dims, ranks, n = CASES[name]
    idx = synth.random_indices(dims, n, seed=41 + len(name))
    _check_case(tu, dims, ranks, idx, seed=51)


def test_one_index_repeated_everywhere(tu):
    # one slice per core spans every chunk: its partials are summed by the fix-up pass
    dims, ranks = (5, 6), (1, 2, 1)
    _check_case(tu, dims, ranks, np.full(1000, 17, np.int64), seed=52)


def test_empty_index_set(tu):
    dims, ranks = (4, 5), (1, 3, 1)
    plan, tc, ti, _ = _check_case(tu, dims, ranks, np.zeros(0, np.int64), seed=53)
    assert plan.at(tc).numel() == 0
    grads = plan.backward(tc, torch.zeros(0, device="cuda"))
    assert all(float(g.abs().sum()) == 0.0 for g in grads)


def test_out_of_range_index_is_rejected(tu):
    dims, ranks = (4, 5, 6), (1, 2, 3, 1)
    tc = [torch.from_numpy(c).cuda() for c in _cores(dims, ranks, 54)]
    for bad in (120, -1, 1 << 40):
        idx = torch.tensor([0, 7, bad, 3], dtype=torch.int64, device="cuda")
        with pytest.raises(tu.TTError) as ei:
            tu.EvalPlan(dims, ranks, idx)
        assert ei.value.status == tu.TT_EINVAL
        with pytest.raises(tu.TTError) as ei:
            tu.tt_eval_at(tc, idx)
        assert ei.value.status == tu.TT_EINVAL
    # the context stays usable
    good = torch.tensor([0, 7, 119, 3], dtype=torch.int64, device="cuda")
    full = tu.tt_full(tc).reshape(-1)
    assert torch.allclose(tu.tt_eval_at(tc, good), full[good], rtol=1e-6, atol=1e-7)


def test_backward_is_bitwise_reproducible(tu):
    dims, ranks = (256, 256, 64), (1, 32, 16, 1)
    idx = synth.random_indices(dims, 300_000, seed=55)
    tc = [torch.from_numpy(c).cuda() for c in _cores(dims, ranks, 56)]
    ti = torch.from_numpy(idx).cuda()
    gout = torch.from_numpy(np.random.default_rng(57).standard_normal(len(idx)).astype(np.float32)).cuda()
    p1 = tu.EvalPlan(dims, ranks, ti)
    p2 = tu.EvalPlan(dims, ranks, ti)
    x1, x2 = p1.at(tc), p2.at(tc)
    assert torch.equal(x1, x2) and torch.equal(x1, tu.tt_eval_at(tc, ti))
    g1 = p1.backward(tc, gout)
    for g in (p1.backward(tc, gout), p2.backward(tc, gout), tu.tt_eval_at_backward(tc, ti, gout)):
        for a, b in zip(g1, g):
            assert torch.equal(a, b)


def test_strided_operands(tu):
    dims, ranks = (9, 8, 7), (1, 4, 3, 1)
    idx = synth.random_indices(dims, 2000, seed=58)
    tc = [torch.from_numpy(c).cuda() for c in _cores(dims, ranks, 59)]
    big = torch.zeros(2 * len(idx), dtype=torch.int64, device="cuda")
    big[::2] = torch.from_numpy(idx).cuda()
    ti = big[::2]
    assert not ti.is_contiguous()
    gbig = torch.from_numpy(np.random.default_rng(60).standard_normal(3 * len(idx)).astype(np.float32)).cuda()
    gout = gbig[::3]
    x = tu.tt_eval_at(tc, ti)
    g = tu.tt_eval_at_backward(tc, ti, gout)
    tic, goc = ti.contiguous(), gout.contiguous()
    assert torch.equal(x, tu.tt_eval_at(tc, tic))
    for a, b in zip(g, tu.tt_eval_at_backward(tc, tic, goc)):
        assert torch.equal(a, b)


def test_backward_accumulates_into_out(tu):
    dims, ranks = (6, 7, 5), (1, 3, 2, 1)
    idx = torch.from_numpy(synth.random_indices(dims, 900, seed=61)).cuda()
    tc = [torch.from_numpy(c).cuda() for c in _cores(dims, ranks, 62)]
    gout = torch.randn(900, device="cuda")
    plan = tu.EvalPlan(dims, ranks, idx)
    g = plan.backward(tc, gout)
    base = [torch.full_like(c, 0.5) for c in tc]
    acc = plan.backward(tc, gout, out=[b.clone() for b in base])
    for a, b, gg in zip(acc, base, g):
        assert torch.allclose(a, b + gg, rtol=1e-6, atol=1e-6)


def test_autograd_function_with_plan(tu):
    dims, ranks = (6, 8, 5), (1, 4, 3, 1)
    idx = torch.from_numpy(synth.random_indices(dims, 150, seed=63)).cuda()
    cores = [torch.from_numpy(c).cuda().requires_grad_() for c in _cores(dims, ranks, 64)]
    plan = tu.EvalPlan(dims, ranks, idx)
    x = tu.TTEvalMasked.apply(plan, *cores)
    (x * x).sum().backward()
    with torch.no_grad():
        cd = [c.detach().double().cpu().numpy() for c in cores]
        ref = otc.tt_eval_grad(cd, idx.cpu().numpy(), 2 * x.detach().double().cpu().numpy())
    for c, r in zip(cores, ref):
        np.testing.assert_allclose(c.grad.double().cpu().numpy(), r, rtol=1e-4, atol=1e-5 * np.abs(r).max())


def test_c4_full_size(tu):
    """The completion workload's own shapes: 256 x 256 x 64, ranks (1, 32, 16, 1),
    the Bernoulli(0.3) observation set (about 1.26M entries).  Sampled entries
    against the oracle, and at full size the identity that holds because x is
    linear in each core: <dG_k, G_k> = sum_e gout_e x_e for every k."""
    cfg = synth.CONFIGS["c4"]
    dims, ranks = cfg["shape"], cfg["ranks"]
    idx = synth.observation_mask(dims, cfg["p_obs"], cfg["mask_seed"])
    c32 = _cores(dims, ranks, 65)
    tc = [torch.from_numpy(c).cuda() for c in c32]
    ti = torch.from_numpy(idx).cuda()
    gout = torch.from_numpy(np.random.default_rng(66).standard_normal(len(idx)).astype(np.float32)).cuda()
    plan = tu.EvalPlan(dims, ranks, ti)
    x = plan.at(tc)
    grads = plan.backward(tc, gout)
    xs = x.double().cpu().numpy()
    sub = np.random.default_rng(67).choice(len(idx), 20000, replace=False)
    c64 = [c.astype(np.float64) for c in c32]
    ref = otc.tt_eval_at(c64, idx[sub])
    mag = otc.tt_eval_at([np.abs(c) for c in c64], idx[sub])
    assert np.all(np.abs(xs[sub] - ref) <= (sum(ranks) + 8) * U * mag)
    s = float((gout.double() * x.double()).sum())
    # scale of the rounding: sum_e |gout_e| (the TT of |G_k| at e)
    xa = plan.at([c.abs() for c in tc])
    sabs = float((gout.double().abs() * xa.double()).sum())
    for g, c in zip(grads, tc):
        e = float((g.double() * c.double()).sum())
        assert abs(e - s) <= 1e-4 * sabs, (e, s)

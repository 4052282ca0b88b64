"""Parity of the CUDA sweep (through the C ABI) with the FP64 oracle.

Cores are unique only up to a gauge (rotations between neighbouring cores),
so parity compares what is unique: the ranks, the represented tensor
(||A_gpu - A_oracle||_F / ||A||_F), the error RSE, the error equality of
Thm 3.1/3.2 (RSE^2 ||A||^2 = sum_k ||E_k||^2) and the orthogonality of the
cores (Def. 2.2).  Tolerances: FP64 arithmetic 1e-10; FP32 1e-5 (relative to
||A||_F) with identical ranks and RSE <= eps (1 + 1e-3).
"""
import os

import numpy as np
import pytest
import torch

import synth
from oracle import tt as otc
from oracle.philox import rademacher

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tu():
    import paper_2501_07904_gb300 as m
    if not os.path.exists(m.LIB_PATH):
        from paper_2501_07904_gb300 import build
        build.build()
    assert torch.cuda.is_available()
    m.lib()
    return m


def np_cores(res):
    return [g.detach().double().cpu().numpy() for g in res.cores]


def rel_diff(cores_a, cores_b, normA2):
    D = otc.tt_full(cores_a) - otc.tt_full(cores_b)
    return float(np.sqrt(np.sum(D * D) / normA2))


def tt_inner(a, b):
    """<X, Y> of two tensors in TT format (FP64), contracting core by core:
    O(d I r^3), the full tensors are never formed."""
    Z = np.ones((1, 1))
    for ga, gb in zip(a, b):
        T = np.einsum("xy,xip->yip", Z, np.asarray(ga, np.float64))
        Z = np.einsum("yip,yiq->pq", T, np.asarray(gb, np.float64))
    return float(Z[0, 0])


def rel_diff_tt(cores_a, cores_b, normA2):
    """||X - Y||_F / ||A||_F from TT inner products, ||X||^2 - 2<X,Y> + ||Y||^2:
    gauge invariant (does not depend on how the cores split the tensor).  The
    FP64 inner products carry ~1e-14 of ||X||^2, so differences below ~1e-7
    of ||A|| are not resolved; the tolerances here are 1e-5 and above."""
    d2 = tt_inner(cores_a, cores_a) - 2.0 * tt_inner(cores_a, cores_b) + tt_inner(cores_b, cores_b)
    return float(np.sqrt(max(d2, 0.0) / normA2))


def orth_err(res):
    errs = []
    if res.orth == "right":
        for g in res.cores[1:]:
            G1 = g.double().reshape(g.shape[0], -1)
            errs.append((G1 @ G1.T - torch.eye(g.shape[0], dtype=torch.float64, device=g.device)).abs().max().item())
    else:
        for g in res.cores[:-1]:
            G2 = g.double().reshape(-1, g.shape[2])
            errs.append((G2.T @ G2 - torch.eye(g.shape[2], dtype=torch.float64, device=g.device)).abs().max().item())
    return max(errs) if errs else 0.0


def gpu_rse(tu, A_t, res):
    full = tu.tt_full([g.double() for g in res.cores])
    D = full - A_t.double()
    return float(torch.sqrt((D * D).sum() / (A_t.double() ** 2).sum()).item())


def run_gpu(tu, A, method, **kw):
    A_t = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    if method == "SVD":
        return A_t, tu.tt_svd(A_t, **kw)
    return A_t, tu.tt_utv(A_t, variant=method, **kw)


def run_oracle(A, method, **kw):
    kw = {k: v for k, v in kw.items() if k in ("eps", "ranks", "l_full", "oversample", "seed")}
    if "oversample" in kw:
        kw["p"] = kw.pop("oversample")
    if method == "SVD":
        kw.pop("seed", None)
        kw.pop("p", None)
        return otc.tt_svd(A, direction="LR", **kw)
    return otc.tt_utv(A, variant=method, **kw)


def tail_floor(precision, d):
    """Resolution of the library's per-step errors, as a fraction of ||A||^2,
    summed over the d - 1 unfoldings: a non-tight step's error is a
    difference of two squared norms of size ~||A||^2, which FP64 holds to
    ~1e-14, FP32 to about one unit roundoff (6e-8) and the tensor cores'
    FP32 accumulation to ~2^-21 (its carry norms are biased low by the
    accumulation's truncation).  Tight steps use compensated sums and FP64
    factors and resolve far below this."""
    per = {"fp64": 1e-14, "fp32": 1e-7, "mixed": 5e-7}[precision]
    return per * (d - 1)


def check_thm_equality(res, err2, normA2, precision):
    """Thm 3.1 / 3.2: ||A - A_TT||^2 = sum of the per-step errors, to 10% plus
    the precision floor."""
    d = len(res.cores)
    floor = tail_floor(precision, d) * normA2
    assert abs(sum(res.tail_sq) - err2) <= 0.1 * err2 + floor, (res.tail_sq, err2, floor)


def check_against_oracle(tu, A, method, tol, eps=None, **kw):
    A_t, res = run_gpu(tu, A, method, eps=eps, **kw)
    ref = run_oracle(np.asarray(A, np.float64), method, eps=eps, **kw)
    normA2 = ref["normA2"]
    diff = rel_diff(np_cores(res), ref["cores"], normA2)
    rse = gpu_rse(tu, A_t, res)
    rse_ref = otc.rse(A, ref["cores"])
    print(f"PARITY {method} {kw} eps={eps} ranks={res.ranks}/{ref['ranks']} diff={diff:.3e} "
          f"rse={rse:.3e} rse_ref={rse_ref:.3e} orth={orth_err(res):.2e} "
          f"tails={sum(res.tail_sq)/normA2:.3e}")
    assert res.ranks == ref["ranks"], (res.ranks, ref["ranks"])
    assert diff <= tol, diff
    assert abs(rse - rse_ref) <= tol + 1e-3 * rse_ref
    if eps is not None:
        assert rse <= eps * (1 + 1e-3)
    # Thm 3.1 / 3.2 equality with the library's own per-step errors
    check_thm_equality(res, rse * rse * normA2, normA2, kw.get("precision", "fp32"))
    assert orth_err(res) <= 100 * tol
    assert abs(res.norm_sq - normA2) <= 1e-6 * normA2
    return res, ref


# ---------------------------------------------------------------- sketch stream

@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_sketch_matrix_bit_identical(tu, dtype):
    for rows, cols, seed, step in [(300, 200, 7, 3), (17, 129, (1 << 40) + 5, 1), (1, 1, 0, 0)]:
        g = tu.sketch_matrix(rows, cols, seed=seed, step=step, dtype=dtype).cpu().double().numpy()
        o = rademacher(rows, cols, seed, step)
        assert np.array_equal(g, o)


# ------------------------------------------------------------------ c1: 16^4 FP64

@pytest.mark.parametrize("method", ["URV", "ULV", "SVD"])
def test_c1_fp64(tu, method):
    A = synth.make_config("c1")
    res, ref = check_against_oracle(tu, A, method, 1e-10, eps=1e-6, precision="fp64")
    assert res.ranks == [1, 4, 4, 4, 1]


# ---------------------------------------------- ragged sizes, several tiles, paths

RAGGED = synth.gaussian_tt((37, 29, 41, 23), (1, 5, 7, 4, 1), rel_noise=1e-6, seed=5,
                           dtype=np.float64)


@pytest.mark.parametrize("precision, tol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("method", ["URV", "ULV"])
@pytest.mark.parametrize("l_full", [256, 24])
def test_ragged_adaptive(tu, precision, tol, method, l_full):
    A = RAGGED if precision == "fp64" else RAGGED.astype(np.float32)
    res, ref = check_against_oracle(tu, A, method, tol, eps=1e-3, precision=precision,
                                    l_full=l_full)
    if l_full == 24:
        assert any(l > 0 for l in res.sketch_l)


@pytest.mark.parametrize("method", ["URV", "ULV"])
@pytest.mark.parametrize("l_full", [256, 24])
def test_ragged_fixed_ranks(tu, method, l_full):
    A = RAGGED.astype(np.float32)
    check_against_oracle(tu, A, method, 1e-5, ranks=[4, 6, 3], precision="fp32", l_full=l_full)


def test_ragged_tt_svd(tu):
    A = RAGGED.astype(np.float32)
    check_against_oracle(tu, A, "SVD", 1e-5, eps=1e-3, precision="fp32")


def test_sketch_growth(tu):
    # rank 40 at the sketched step; the first sketch has 32 columns
    A = synth.gaussian_tt((50, 50, 50), (1, 40, 40, 1), rel_noise=1e-9, seed=20, dtype=np.float64)
    res, ref = check_against_oracle(tu, A, "URV", 1e-9, eps=1e-6, precision="fp64", l_full=16)
    assert res.ranks == [1, 40, 40, 1]


def test_matrix_d2(tu):
    rng = np.random.default_rng(3)
    A = (rng.standard_normal((300, 12)) @ rng.standard_normal((12, 200))
         + 1e-5 * rng.standard_normal((300, 200))).astype(np.float32)
    for m in ("URV", "ULV", "SVD"):
        res, _ = check_against_oracle(tu, A, m, 1e-5, eps=1e-4, precision="fp32")
        assert res.ranks == [1, 12, 1]


# -------------------------------------------------------------- edge cases

def test_edge_dims_of_one_and_clamp(tu):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((5, 1, 7)).astype(np.float32)
    res, _ = check_against_oracle(tu, A, "URV", 1e-5, ranks=[9, 9], precision="fp32")
    assert res.ranks == [1, 5, 5, 1]


def test_zero_tensor(tu):
    A = torch.zeros((6, 7, 8), device="cuda")
    res = tu.tt_utv(A, eps=0.1)
    assert res.ranks == [1, 1, 1, 1]
    assert torch.count_nonzero(tu.tt_full(res.cores)).item() == 0


def test_nonfinite_rejected(tu):
    A = torch.randn((8, 9, 10), device="cuda")
    A[3, 4, 5] = float("nan")
    with pytest.raises(tu.TTError, match="ENONFINITE"):
        tu.tt_utv(A, eps=0.1)
    A[3, 4, 5] = float("inf")
    with pytest.raises(tu.TTError, match="ENONFINITE"):
        tu.tt_utv(A, eps=0.1, variant="ULV")


def test_host_input_and_cast(tu):
    A = RAGGED.astype(np.float32)
    dev = tu.tt_utv(torch.from_numpy(A).cuda(), eps=1e-3)
    host = tu.tt_utv(torch.from_numpy(A).pin_memory(), eps=1e-3)
    assert dev.ranks == host.ranks
    for a, b in zip(dev.cores, host.cores):
        assert torch.equal(a, b)
    # FP64 data decomposed in FP32 arithmetic: the input is narrowed first
    r64 = tu.tt_utv(torch.from_numpy(RAGGED).cuda(), eps=1e-3, precision="fp32")
    assert r64.ranks == dev.ranks and r64.cores[0].dtype == torch.float32


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_svd_sketched_when_both_sides_large(tu, precision):
    # both sides of the first unfolding above l_full: the Jacobi SVD runs on
    # the projection onto the sketch's range, which holds the tensor's whole
    # low-rank range here, so ranks match the exact TT-SVD's and the cores
    # agree to the level of the 1e-7 noise that the two treat differently;
    # FP32 resolves the range miss (a difference of squared norms) only to
    # ~1e-8 of ||A||^2, which bounds its tail estimate
    A = synth.gaussian_tt((300, 300, 2), (1, 5, 2, 1), 1e-7, seed=71, dtype=np.float64)
    if precision == "fp32":
        A = A.astype(np.float32)
    res = tu.tt_svd(torch.from_numpy(A).cuda(), eps=1e-3, l_full=16, direction="LR",
                    precision=precision)
    ref = otc.tt_svd(np.asarray(A, np.float64), eps=1e-3, direction="LR")
    assert res.ranks == ref["ranks"]
    assert res.sketch_l[0] > 0
    d = rel_diff_tt([c.double().cpu().numpy() for c in res.cores], ref["cores"], ref["normA2"])
    assert d <= (1e-6 if precision == "fp64" else 1e-5), d
    err2 = float(np.sum((otc.tt_full([c.double().cpu().numpy() for c in res.cores]) - A) ** 2))
    floor = (1e-12 if precision == "fp64" else 1e-7) * ref["normA2"]
    assert abs(sum(res.tail_sq) - err2) <= 0.1 * err2 + floor


@pytest.mark.parametrize("precision, tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_alg4_pairings(tu, precision, tol):
    # TT-ULV right-to-left keeping [L_11; L_21] (the appendix's Alg. 4, first
    # case) against the oracle's Alg. 4, which forms it from the ULV factors;
    # it runs the URV right-to-left sweep, and URV left-to-right the ULV
    # left-to-right one, bit for bit
    A = RAGGED if precision == "fp64" else RAGGED.astype(np.float32)
    A_t = torch.from_numpy(A).cuda()
    res = tu.tt_utv(A_t, eps=1e-3, variant="ULV", direction="RL", precision=precision, l_full=24)
    ref = otc.tt_ulv_rl(np.asarray(A, np.float64), eps=1e-3, lhat="full", l_full=24)
    assert res.ranks == ref["ranks"]
    assert res.orth == "right"
    assert rel_diff(np_cores(res), ref["cores"], ref["normA2"]) <= tol
    for v, direction, same in (("ULV", "RL", "URV"), ("URV", "LR", "ULV")):
        a = tu.tt_utv(A_t, eps=1e-3, variant=v, direction=direction, precision=precision, l_full=24)
        b = tu.tt_utv(A_t, eps=1e-3, variant=same, precision=precision, l_full=24)
        assert a.ranks == b.ranks and a.orth == b.orth and a.tail_sq == b.tail_sq
        for x, y in zip(a.cores, b.cores):
            assert torch.equal(x, y)


@pytest.mark.parametrize("precision, tol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("l_full", [256, 24])
def test_alg4_l11_matches_oracle(tu, precision, tol, l_full):
    # the appendix's Alg. 4 as printed (L_11 kept alone) against the oracle's,
    # which forms U_1 L_11 from Householder factors: same ranks, tensors and
    # step errors, the Proposition's bound RSE <= sum eps_k = eps (weights
    # 1/(d-1)), and its error = the sum of the step errors no longer an
    # equality (the errors add in norm); exact and sketched steps
    A = RAGGED if precision == "fp64" else RAGGED.astype(np.float32)
    A64 = np.asarray(A, np.float64)
    A_t = torch.from_numpy(A).cuda()
    for eps in (1e-2, 1e-5):
        res = tu.tt_utv(A_t, eps=eps, variant="ULV", direction="RL", lhat="l11",
                        precision=precision, l_full=l_full)
        ref = otc.tt_ulv_rl(A64, eps=eps, lhat="l11", l_full=l_full)
        assert res.ranks == ref["ranks"], (eps, res.ranks, ref["ranks"])
        assert res.orth == "right"
        cores = np_cores(res)
        assert rel_diff(cores, ref["cores"], ref["normA2"]) <= tol
        rse = otc.rse(A64, cores)
        assert rse <= eps
        if precision == "fp64":  # FP32 step errors this small sit below FP32 rounding of ||C||^2
            for t, tr in zip(res.tail_sq, ref["tails"]):
                assert abs(t - tr) <= max(1e-6 * tr, 1e-12 * ref["normA2"])
    # fixed ranks: the same cores as the oracle's
    res = tu.tt_utv(A_t, ranks=[4, 6, 3], variant="ULV", direction="RL", lhat="l11",
                    precision=precision, l_full=l_full)
    ref = otc.tt_ulv_rl(A64, ranks=[4, 6, 3], lhat="l11", l_full=l_full)
    assert res.ranks == ref["ranks"]
    assert rel_diff(np_cores(res), ref["cores"], ref["normA2"]) <= tol


def test_alg4_l11_argument_checks(tu):
    A = torch.from_numpy(RAGGED.astype(np.float32)).cuda()
    for kw in (dict(variant="URV", direction="RL"), dict(variant="ULV", direction="LR"),
               dict(variant="ULV", direction="RL", inner="usvp"),
               dict(variant="ULV", direction="RL", inner="lurv")):
        with pytest.raises(tu.TTError) as ei:
            tu.tt_utv(A, eps=1e-2, lhat="l11", **kw)
        assert ei.value.status == tu.TT_EINVAL
    with pytest.raises(tu.TTError) as ei:      # L_11 weights must sum to 1
        tu.tt_utv(A, eps=1e-2, variant="ULV", direction="RL", lhat="l11",
                  weights=[3 ** -0.5] * 3)
    assert ei.value.status == tu.TT_EINVAL


def test_deterministic(tu):
    A = torch.from_numpy(RAGGED.astype(np.float32)).cuda()
    a = tu.tt_utv(A, eps=1e-3, l_full=24)
    b = tu.tt_utv(A, eps=1e-3, l_full=24)
    for x, y in zip(a.cores, b.cores):
        assert torch.equal(x, y)


# -------------------------------------------------- full-size configs (golden)

def load_gold(name):
    path = os.path.join(GOLD, name + ".npz")
    if not os.path.exists(path):
        pytest.fail(f"missing golden file {path}: run tests/golden/make_golden.py")
    return np.load(path)


def check_gold(tu, A, method, name, tol, eps, **kw):
    g = load_gold(name)
    A_t, res = run_gpu(tu, A, method, eps=eps, **kw)
    assert res.ranks == [int(x) for x in g["ranks"]], (res.ranks, g["ranks"])
    normA2 = float(g["normA2"])
    vals = tu.tt_eval_at([c.float() for c in res.cores],
                         torch.from_numpy(g["sample_idx"]).cuda()).double().cpu().numpy()
    ref = g["sample_val"]
    samp = np.sqrt(np.sum((vals - ref) ** 2) / np.sum(g["sample_ref"] ** 2))
    assert samp <= 10 * tol, samp
    # the whole represented tensor against the oracle's (S13's criterion)
    ocores = [g[f"core{k}"].astype(np.float64) for k in range(len(res.cores))]
    full = rel_diff_tt(np_cores(res), ocores, normA2)
    print(f"GOLD {name} {kw} ranks={res.ranks} full_diff={full:.3e} sampled={samp:.3e}")
    assert full <= tol, full
    rse = gpu_rse(tu, A_t, res)
    assert abs(rse - float(g["rse"])) <= tol + 1e-3 * float(g["rse"])
    assert rse <= eps * (1 + 1e-3)
    check_thm_equality(res, rse * rse * normA2, normA2, kw.get("precision", "fp32"))
    assert orth_err(res) <= 1e-4
    return res


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("method", ["URV", "ULV", "SVD"])
def test_c2_hilbert_256(tu, method, precision):
    # the FP32 input of 1/(i+j+k+1).  FP64 arithmetic widens it; FP32 and
    # mixed arithmetic meet eps = 1e-6 (eps_k^2 = 5e-13 ||A||^2, every step
    # tight, kept singular values down to ~1e-6 of ||C||) through compensated
    # Grams, FP64 small factors and compensated sketches, projections, carries
    # and cores
    A = synth.make_config("c2")
    check_gold(tu, A, method, f"c2_{method}", 1e-5, 1e-6, precision=precision)


@pytest.mark.parametrize("method", ["URV", "ULV"])
def test_c3_32pow5(tu, method):
    A = synth.make_config("c3")
    res = check_gold(tu, A, method, f"c3_{method}", 1e-5, 1e-3, precision="fp32")
    assert res.ranks == [1, 20, 20, 20, 20, 1]
    check_tight_tails(tu, A, res, method, "c3")


def check_tight_tails(tu, A, res, method, name):
    """Every step of c3 is tight: its reported errors come from compensated
    Grams and FP64 factorizations.  The first step's (an exact Gram step)
    matches the oracle's to 1e-3 relative, far below FP32 rounding of ||A||^2.
    The sum matches ||A - A_TT||^2 (Thm 3.1/3.2) to 25% plus the floor of the
    sketched steps' estimates: their range miss ||C||^2 - ||C W||^2 carries
    the FP32 rounding of B = C W, about u_fp32 sqrt(2 / entries of B) of
    ||C||^2 (4e-9 of ||A||^2 for the 32 x 32 B of the last step), against
    tolerances delta_k^2 of 2.5e-7 ||A||^2."""
    g = load_gold(f"{name}_{method}")
    normA2 = float(g["normA2"])
    first = len(res.tail_sq) - 1 if method == "URV" else 0
    t, t_ref = res.tail_sq[first], float(g["tails"][first])
    assert abs(t - t_ref) <= 1e-3 * t_ref + 1e-13 * normA2, (t, t_ref)
    err2, _ = tu.tt_rse(torch.from_numpy(np.ascontiguousarray(A)).cuda(), res.cores)
    assert abs(sum(res.tail_sq) - err2) <= 0.25 * err2 + 1e-8 * normA2, (res.tail_sq, err2)


def test_c5_128pow4(tu):
    A = synth.make_config("c5")
    res = check_gold(tu, A, "URV", "c5_URV", 1e-5, 1e-2, precision="fp32")
    assert res.ranks == [1, 64, 64, 64, 1]


# ------------------------------------------------ masked evaluation and gradient

def test_masked_eval_and_grad_small(tu):
    cores = synth.gaussian_cores((7, 5, 9, 4), (1, 3, 4, 2, 1), seed=31)
    idx = synth.random_indices((7, 5, 9, 4), 700, seed=32)
    gout = np.random.default_rng(33).standard_normal(700)
    tc = [torch.from_numpy(c).float().cuda() for c in cores]
    ti = torch.from_numpy(idx).cuda()
    x = tu.tt_eval_at(tc, ti).double().cpu().numpy()
    c32 = [c.astype(np.float32).astype(np.float64) for c in cores]
    np.testing.assert_allclose(x, otc.tt_eval_at(c32, idx), rtol=1e-5, atol=1e-5)
    grads = tu.tt_eval_at_backward(tc, ti, torch.from_numpy(gout).float().cuda())
    ref = otc.tt_eval_grad(c32, idx, gout.astype(np.float32).astype(np.float64))
    for g, r in zip(grads, ref):
        np.testing.assert_allclose(g.double().cpu().numpy(), r, rtol=1e-4, atol=1e-4 * np.abs(r).max())
    # FP64 central differences of the oracle (the map is linear in each core)
    h = 1e-6
    rng = np.random.default_rng(34)
    for k in range(4):
        for _ in range(5):
            pos = tuple(rng.integers(0, s) for s in cores[k].shape)
            cp = [c.copy() for c in c32]
            cm = [c.copy() for c in c32]
            cp[k][pos] += h
            cm[k][pos] -= h
            fd = (gout @ otc.tt_eval_at(cp, idx) - gout @ otc.tt_eval_at(cm, idx)) / (2 * h)
            assert abs(grads[k][pos].item() - fd) <= 1e-3 * max(1.0, abs(fd))


def test_masked_autograd_function(tu):
    cores = [torch.from_numpy(c).float().cuda().requires_grad_() for c in
             synth.gaussian_cores((6, 8, 5), (1, 4, 3, 1), seed=35)]
    idx = torch.from_numpy(synth.random_indices((6, 8, 5), 100, seed=36)).cuda()
    x = tu.TTEvalMasked.apply(idx, *cores)
    (x * x).sum().backward()
    full = tu.tt_full([c.detach() for c in cores]).reshape(-1)
    assert torch.allclose(x, full[idx], rtol=1e-5, atol=1e-6)
    with torch.no_grad():
        cd = [c.detach().double().cpu().numpy() for c in cores]
        ref = otc.tt_eval_grad(cd, idx.cpu().numpy(), 2 * x.detach().double().cpu().numpy())
    for c, r in zip(cores, ref):
        np.testing.assert_allclose(c.grad.double().cpu().numpy(), r, rtol=1e-4, atol=1e-4 * np.abs(r).max())


def test_masked_eval_c4_shapes(tu):
    cfg = synth.CONFIGS["c4"]
    shape = cfg["shape"]
    idx = synth.observation_mask(shape, cfg["p_obs"], cfg["mask_seed"])
    cores = synth.gaussian_cores(shape, cfg["ranks"], seed=37)
    cores = [c / np.sqrt(c.shape[0]) for c in cores]
    tc = [torch.from_numpy(c).float().cuda() for c in cores]
    ti = torch.from_numpy(idx).cuda()
    x = tu.tt_eval_at(tc, ti).double().cpu().numpy()
    c32 = [c.astype(np.float32).astype(np.float64) for c in cores]
    sub = np.random.default_rng(38).choice(len(idx), 20000, replace=False)
    np.testing.assert_allclose(x[sub], otc.tt_eval_at(c32, idx[sub]), rtol=1e-4, atol=1e-5)
    gsub = np.sort(sub)
    gout = np.random.default_rng(39).standard_normal(len(gsub))
    grads = tu.tt_eval_at_backward(tc, torch.from_numpy(idx[gsub]).cuda(),
                                   torch.from_numpy(gout).float().cuda())
    ref = otc.tt_eval_grad(c32, idx[gsub], gout.astype(np.float32).astype(np.float64))
    for g, r in zip(grads, ref):
        np.testing.assert_allclose(g.double().cpu().numpy(), r, rtol=1e-3, atol=1e-4 * np.abs(r).max())

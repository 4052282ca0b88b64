"""The bounds-checked build (-DTT_BOUNDS_CHECK, libttutv_bc.so), the stand-in
for a memory checker: every checked access (the masked evaluation's decoded
indices, permutations and positions, core slices, tensor-map coordinates and
their 16-byte alignment, gathered copies) is verified before it is made, and
a violation is counted and skipped instead of performed.  The whole API is
driven through that build in a child process on small cases of every path --
exact, sketched, mixed-precision and FP64 sweeps, TT-SVD, reversed sweeps,
USV-plus and the Givens URV, contraction and RSE, orthogonalization, the masked evaluation, its
two-frame backward and the tangent projection -- and the results are checked
against the FP64 oracle and the counters must read zero.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

from test_gpu_parity import tu  # noqa: F401,E402  (fixture)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
import paper_2501_07904_gb300 as tu
import synth
from oracle import tt as otc
assert tu.LIB_PATH.endswith("libttutv_bc.so")
assert tu.bounds_violations(reset=True)[0] == 0
dev = "cuda"
A64 = synth.gaussian_tt((12, 10, 300, 8), (1, 4, 6, 3, 1), 1e-6, seed=1, dtype=np.float64)
A = torch.from_numpy(A64).to(dev)
ref = otc.tt_utv(A64, eps=1e-4, variant="URV")
for prec in ("fp64", "fp32", "mixed"):
    X = A if prec == "fp64" else A.float()
    for variant in ("URV", "ULV"):
        res = tu.tt_utv(X, eps=1e-4, variant=variant, precision=prec)
        assert res.ranks == ref["ranks"], (prec, variant, res.ranks)
        cores = [c.double().cpu().numpy() for c in res.cores]
        assert otc.rse(A64, cores) <= 1e-4, (prec, variant)
    res = tu.tt_utv(X, eps=1e-4, variant="URV", precision=prec, reverse=True)
    assert res.ranks == ref["ranks"]
res = tu.tt_svd(A, eps=1e-4)
assert res.ranks == ref["ranks"]
for inner in ("lurv", "usvp"):
    res = tu.tt_utv(A, eps=1e-4, variant="ULV", precision="fp64", inner=inner)
    assert res.ranks == ref["ranks"], inner
full = tu.tt_full(res.cores)
assert float((full - A).norm() / A.norm()) <= 1e-4
err2, n2 = tu.tt_rse(A, res.cores)
assert (err2 / n2) ** 0.5 <= 1e-4
for side in ("left", "right"):
    oc = tu.tt_orthogonalize(res.cores, side)
    assert float((tu.tt_full(oc) - full).norm() / full.norm()) <= 1e-12
# masked evaluation, two-frame backward, tangent projection (d = 3 stored rows)
dims, ranks = (40, 30, 20), (1, 6, 5, 1)
cs = [torch.from_numpy(c).float().to(dev) for c in synth.gaussian_cores(dims, ranks, seed=2)]
idx = torch.from_numpy(synth.random_indices(dims, 5000, seed=3)).to(dev)
plan = tu.EvalPlan(dims, ranks, idx)
x = plan.at(cs)
c64 = [c.double().cpu().numpy() for c in cs]
xr = otc.tt_eval_at(c64, idx.cpu().numpy())
assert np.abs(x.double().cpu().numpy() - xr).max() <= 1e-4 * np.abs(xr).max()
g = plan.backward(cs, x)
U = tu.tt_orthogonalize(cs, "left")
V = tu.tt_orthogonalize(cs, "right")
dU = plan.tangent_project(U, V, x)
gb = plan.backward(U, x, right=V)
n, line = tu.bounds_violations()
assert n == 0, (n, line)
print("bounds-checked run: 0 violations")
"""


def test_bounds_checked_build_runs_clean():
    from paper_2501_07904_gb300 import build

    lib = build.build(checked=True)
    assert os.path.exists(lib)
    env = dict(os.environ, TTUTV_CHECKED="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    res = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=900)
    assert res.returncode == 0, res.stdout[-3000:] + res.stderr[-3000:]
    assert "0 violations" in res.stdout


def test_normal_build_reports_no_counters(tu):
    assert tu.bounds_violations() == (-1, 0)

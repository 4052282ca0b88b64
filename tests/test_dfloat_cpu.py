"""Host checks of the double-float arithmetic in csrc/dfloat.cuh (an FP32 pair
h + l carrying ~48 bits), compiled for the CPU with g++ and compared with
exact rational arithmetic: the error-free transformations are exact, and the
compound operations stay within small multiples of u^2 (u = 2^-24) of the
exact result, the bounds of Joldes, Muller and Popescu (2017) for the sum and
product, and the same order for the fused product-sum under cancellation.
"""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2501_07904_gb300", "csrc")
U = Fraction(1, 2 ** 24)

HARNESS = r"""
#include <cmath>
#include <cstdio>
#include "dfloat.cuh"
using ttk::df32;
int main() {
  int n;
  if (scanf("%d", &n) != 1) return 1;
  for (int i = 0; i < n; ++i) {
    float ah, al, bh, bl, ch, cl;
    if (scanf("%a %a %a %a %a %a", &ah, &al, &bh, &bl, &ch, &cl) != 6) return 2;
    df32 a(ah, al), b(bh, bl), c(ch, cl);
    float s, e, p, q;
    ttk::two_sum(ah, bh, s, e);
    ttk::two_prod(ah, bh, p, q);
    df32 x = a + b, y = a * b, z = ttk::fma_df(a, b, c), w = a - b;
    df32 aa = ah > 0 ? a : -a;
    df32 r = ttk::rsqrt_df(aa, 1.0f / std::sqrt(aa.h));
    df32 m = ttk::fmax_df(a, b);
    printf("%a %a %a %a %a %a %a %a %a %a %a %a %a %a %a %a %d %d\n", s, e, p, q, x.h, x.l, y.h,
           y.l, z.h, z.l, w.h, w.l, r.h, r.l, m.h, m.l, (int)(a > b), (int)(a <= b));
  }
  return 0;
}
"""


def _split(x):
    h = np.float32(x)
    return h, np.float32(x - np.float64(h))


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        ea, eb = rng.integers(-20, 20, size=2)
        a = rng.standard_normal() * 2.0 ** ea
        b = rng.standard_normal() * 2.0 ** eb
        kind = i % 4
        if kind == 1:          # near-cancellation in a + b and a b + c
            b = -a * (1 + rng.standard_normal() * 2.0 ** -int(rng.integers(10, 40)))
        c = rng.standard_normal() * abs(a * b) * 2.0 ** int(rng.integers(-5, 5))
        if kind == 2:          # a b + c cancels
            c = -a * b * (1 + rng.standard_normal() * 2.0 ** -int(rng.integers(10, 40)))
        rows.append((*_split(a), *_split(b), *_split(c)))
    return rows


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("dfloat")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o",
                    str(exe)], check=True)
    rows = _inputs(4000, seed=7)
    text = f"{len(rows)}\n" + "\n".join(" ".join(float(v).hex() for v in r) for r in rows)
    out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout
    res = []
    for r, line in zip(rows, out.splitlines()):
        f = line.split()
        res.append((r, [float.fromhex(v) for v in f[:16]], int(f[16]), int(f[17])))
    assert len(res) == len(rows)
    return res


def F(x):
    return Fraction(float(x))


def _normalized(h, l):
    return float(np.float32(np.float32(h) + np.float32(l))) == h


def test_error_free_transformations(results):
    for r, v, _, _ in results:
        ah, bh = F(r[0]), F(r[2])
        assert F(v[0]) + F(v[1]) == ah + bh
        # the product of two FP32 words is exact in FP64, so p + e must match it
        # unless the exact error underflows FP32 (not the case for these inputs)
        assert F(v[2]) + F(v[3]) == ah * bh


def test_sum_difference_product_bounds(results):
    for r, v, _, _ in results:
        a = F(r[0]) + F(r[1])
        b = F(r[2]) + F(r[3])
        x, y, w = F(v[4]) + F(v[5]), F(v[6]) + F(v[7]), F(v[10]) + F(v[11])
        assert abs(x - (a + b)) <= 4 * U * U * abs(a + b)
        assert abs(w - (a - b)) <= 4 * U * U * abs(a - b)
        assert abs(y - a * b) <= 6 * U * U * abs(a * b)
        for h, l in ((v[4], v[5]), (v[6], v[7]), (v[10], v[11])):
            assert _normalized(h, l)


def test_fused_product_sum_under_cancellation(results):
    worst = Fraction(0)
    for r, v, _, _ in results:
        a, b, c = (F(r[0]) + F(r[1])), (F(r[2]) + F(r[3])), (F(r[4]) + F(r[5]))
        z = F(v[8]) + F(v[9])
        err = abs(z - (a * b + c)) / (abs(a * b) + abs(c))
        worst = max(worst, err)
        assert _normalized(v[8], v[9])
    assert worst <= 8 * U * U, float(worst / (U * U))


def test_reciprocal_square_root(results):
    for r, v, _, _ in results:
        a = abs(F(r[0]) + F(r[1]) if r[0] > 0 else -(F(r[0]) + F(r[1])))
        x = F(v[12]) + F(v[13])
        # x^2 a = 1 within 2^-40 (one Newton step from an FP32 estimate)
        assert abs(x * x * a - 1) <= Fraction(1, 2 ** 40)


def test_comparisons_and_max(results):
    for r, v, gt, le in results:
        a = F(r[0]) + F(r[1])
        b = F(r[2]) + F(r[3])
        assert gt == int(a > b) and le == int(a <= b)
        assert F(v[14]) + F(v[15]) == max(a, b)

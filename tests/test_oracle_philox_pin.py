"""Pin of the oracle's Philox4x32-10 stream against an independent implementation.

PyTorch ships a Philox4x32-10 engine as C++ source (ATen/core/PhiloxRNGEngine.h,
written from the same SC'11 definition by other authors).  A small host
program compiled against that header prints raw 4 x 32-bit output blocks;
the oracle (oracle/philox.py) must reproduce them bit for bit.

The engine's state maps onto the oracle's counter as
    key     = (seed lo, seed hi)
    counter = (offset lo, offset hi, subsequence lo, subsequence hi)
so the sketch's counter (row i, column block j // 128, sweep step, purpose) is
offset = i | (j // 128) << 32, subsequence = step | purpose << 32.  The second
test rebuilds the Rademacher sketch matrix (the range step of randUTV, Sec. 2.2
and 3.3) from the engine's words and compares it with oracle.philox.rademacher.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.philox import philox4x32_10, rademacher

HARNESS = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
int main() {
  unsigned long long seed, sub, off;
  while (std::scanf("%llu %llu %llu", &seed, &sub, &off) == 3) {
    at::philox_engine e(seed, sub, off);
    const unsigned a = e(), b = e(), c = e(), d = e();
    std::printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


def _torch_include():
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("torch's PhiloxRNGEngine.h is not installed")
    return inc


@pytest.fixture(scope="module")
def engine(tmp_path_factory):
    """Path of the compiled harness."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    inc = _torch_include()
    d = tmp_path_factory.mktemp("philox")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I" + inc, str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    return str(exe)


def _run(exe, triples):
    """Engine output blocks for (seed, subsequence, offset) triples."""
    inp = "\n".join(f"{s} {u} {o}" for s, u, o in triples) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    return np.array([[int(x) for x in ln.split()] for ln in out.strip().splitlines()],
                    dtype=np.uint64)


def _cases():
    rng = np.random.default_rng(20250107)
    seeds = [0, 1, 7, 0xFFFFFFFF, 1 << 32, (1 << 32) + 5, 0x0123456789ABCDEF,
             (1 << 64) - 1] + [int(x) for x in rng.integers(0, 2**63, 8, dtype=np.int64)]
    triples = []
    # the sketch's own counters: rows, both column blocks, steps 1..16, purpose 0
    for s in seeds[:8]:
        for step in range(1, 17):
            for i in (0, 1, 2, 127, 4095, 65535, 1 << 20):
                for jb in (0, 1):
                    triples.append((s, step, i | (jb << 32)))
    # arbitrary 64-bit offsets and subsequences (every counter word exercised)
    for s in seeds:
        for _ in range(16):
            triples.append((s, int(rng.integers(0, 2**63)) * 2 + 1, int(rng.integers(0, 2**63)) * 2))
    return triples


def test_blocks_equal_torch_engine(engine):
    triples = _cases()
    assert len(triples) >= 1000
    ref = _run(engine, triples)
    s = np.array([t[0] for t in triples], dtype=np.uint64)
    u = np.array([t[1] for t in triples], dtype=np.uint64)
    o = np.array([t[2] for t in triples], dtype=np.uint64)
    m = np.uint64(0xFFFFFFFF)
    got = np.empty_like(ref)
    for e in range(len(triples)):
        w = philox4x32_10(o[e] & m, o[e] >> np.uint64(32), u[e] & m, u[e] >> np.uint64(32),
                          int(s[e] & m), int(s[e] >> np.uint64(32)))
        got[e] = [int(x) for x in w]
    bad = np.nonzero(np.any(got != ref, axis=1))[0]
    assert bad.size == 0, f"{bad.size} of {len(triples)} blocks differ; first {triples[bad[0]]}"


@pytest.mark.parametrize("seed,step", [(0, 1), (3, 4), ((1 << 40) + 17, 16)])
def test_sketch_matrix_from_torch_engine(engine, seed, step):
    rows, cols = 40, 200  # two column blocks, the second ragged
    om = rademacher(rows, cols, seed=seed, step=step)
    triples = [(seed, step, i | (jb << 32)) for i in range(rows) for jb in range(2)]
    words = _run(engine, triples).reshape(rows, 2, 4)
    ref = np.empty((rows, cols))
    for j in range(cols):
        b = j % 128
        bit = (words[:, j // 128, b // 32] >> np.uint64(b % 32)) & np.uint64(1)
        ref[:, j] = 1.0 - 2.0 * bit.astype(np.float64)
    assert np.array_equal(om, ref)

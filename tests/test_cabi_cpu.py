"""The C-ABI library loads and exports every entry point include/ttutv.h
declares; argument validation answers without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2501_07904_gb300 as tu

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "ttutv.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(tt_[a-z_]+)\s*\(", src, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(tu.LIB_PATH):
        from paper_2501_07904_gb300 import build
        build.build()
    return tu.lib()


def test_header_and_binding_agree():
    assert declared_functions() == sorted(tu.EXPORTS)


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_version_and_defaults(L):
    assert b"sm_103a" in L.tt_version()
    o = tu.tt_opts()
    L.tt_opts_default(ctypes.byref(o))
    assert (o.precision, o.small_precision, o.oversample, o.l_full, o.seed, o.orth_precision) == \
        (1, 0, 16, 256, 0, 0)


def _call(L, A=1, dtype=0, d=3, dims=(4, 5, 6), eps=0.1, fixed=None, variant=0, direction=0, opts=None):
    res = tu.tt_result()
    fr = tu._i64(fixed) if fixed is not None else None
    return L.tt_utv(ctypes.c_void_p(A) if A else None, dtype, d, tu._i64(dims) if dims else None,
                    eps, fr, variant, direction, opts, tu.ALLOC_FN(0), tu.FREE_FN(0), None, None,
                    ctypes.byref(res))


@pytest.mark.parametrize("kw, status", [
    (dict(A=0), 1), (dict(dims=None), 1), (dict(d=1), 1), (dict(d=17, dims=[2] * 17), 1),
    (dict(dims=(4, 0, 6)), 1), (dict(eps=0.0), 1), (dict(eps=-1.0), 1), (dict(eps=float("nan")), 1),
    (dict(fixed=(2, 0)), 1), (dict(dtype=7), 1), (dict(direction=5), 1),
    (dict(variant=-1), 1), (dict(variant=5), 1),
])
def test_invalid_arguments_rejected(L, kw, status):
    assert _call(L, **kw) == status
    assert L.tt_last_error() != b""


def test_invalid_options_rejected(L):
    o = tu.tt_opts()
    L.tt_opts_default(ctypes.byref(o))
    o.l_full = 300
    assert _call(L, opts=ctypes.byref(o)) == 1
    L.tt_opts_default(ctypes.byref(o))
    o.small_precision = 4                        # AUTO, FP32, FP64, DF are 0..3
    assert _call(L, opts=ctypes.byref(o)) == 1
    L.tt_opts_default(ctypes.byref(o))
    o.orth_precision = -1
    assert _call(L, opts=ctypes.byref(o)) == 1
    L.tt_opts_default(ctypes.byref(o))
    w = (ctypes.c_double * 2)(0.5, 0.5)          # sum w^2 != 1
    o.weights = ctypes.cast(w, ctypes.POINTER(ctypes.c_double))
    assert _call(L, opts=ctypes.byref(o)) == 1


def test_eval_rejects_bad_ranks(L):
    dims, ranks = tu._i64([3, 3]), tu._i64([1, 65, 1])
    ptrs = (ctypes.c_void_p * 2)(1, 1)
    assert L.tt_eval_at(2, dims, ranks, ptrs, ctypes.c_void_p(1), 4, ctypes.c_void_p(1), None) == 1
    ranks = tu._i64([2, 3, 1])
    assert L.tt_eval_at(2, dims, ranks, ptrs, ctypes.c_void_p(1), 4, ctypes.c_void_p(1), None) == 1


def test_full_work_bytes(L):
    n = L.tt_full_work_bytes(3, tu._i64([4, 5, 6]), tu._i64([1, 2, 3, 1]), 0)
    assert n >= 2 * 4 * 5 * 3 * 4
    assert L.tt_full_work_bytes(1, tu._i64([4]), tu._i64([1, 1]), 0) == 0


def test_reverse_option(L):
    o = tu.tt_opts()
    L.tt_opts_default(ctypes.byref(o))
    assert o.reverse == 0
    o.reverse = 2
    assert _call(L, opts=ctypes.byref(o)) == 1


def test_rse_arguments_and_work_bytes(L):
    dims, ranks = tu._i64([300, 256, 256]), tu._i64([1, 6, 5, 1])
    ptrs = (ctypes.c_void_p * 3)(1, 1, 1)
    out = ctypes.c_void_p(1)
    # NULL A, NULL work, NULL out, d = 1, r_0 != 1: rejected before any device work
    assert L.tt_rse(3, dims, ranks, ptrs, 0, None, ctypes.c_void_p(1), out, None) == 1
    assert L.tt_rse(3, dims, ranks, ptrs, 0, ctypes.c_void_p(1), None, out, None) == 1
    assert L.tt_rse(3, dims, ranks, ptrs, 0, ctypes.c_void_p(1), ctypes.c_void_p(1), None, None) == 1
    assert L.tt_rse(1, dims, ranks, ptrs, 0, ctypes.c_void_p(1), ctypes.c_void_p(1), out, None) == 1
    assert L.tt_rse(3, dims, tu._i64([2, 6, 5, 1]), ptrs, 0, ctypes.c_void_p(1),
                    ctypes.c_void_p(1), out, None) == 1
    # scratch: a slab of 256 first-mode slices (2^24 entries) plus the contraction's scratch
    n32 = L.tt_rse_work_bytes(3, dims, ranks, 0)
    n64 = L.tt_rse_work_bytes(3, dims, ranks, 1)
    assert n32 >= 256 * 256 * 256 * 4 and n64 >= 256 * 256 * 256 * 8
    assert n32 < 3 * 256 * 256 * 256 * 4
    # one slice of the first mode larger than a slab: the slab is that slice
    big = L.tt_rse_work_bytes(3, tu._i64([2, 4096, 4200]), tu._i64([1, 2, 2, 1]), 0)
    assert 4096 * 4200 * 4 <= big < 2 * 4096 * 4200 * 4
    assert L.tt_rse_work_bytes(1, tu._i64([4]), tu._i64([1, 1]), 0) == 0


def test_rse_work_covers_the_ragged_slab(L):
    # slabs of 1024 first-mode slices and a last one of 276: a smaller
    # contraction may split its inner dimension, so both sizes must fit
    dims, ranks = [1300, 128, 128], [1, 256, 128, 1]
    w = L.tt_rse_work_bytes(3, tu._i64(dims), tu._i64(ranks), 0)
    slab = 1024 * 128 * 128 * 4
    for rows in (1024, 276):
        need = L.tt_full_work_bytes(3, tu._i64([rows, 128, 128]), tu._i64(ranks), 0)
        assert w >= slab + need


@pytest.mark.parametrize("reverse", [0, 1])
def test_allocator_failure_reports_enomem(L, reverse):
    # a host input is staged through the caller's allocator first; an
    # allocator that returns NULL ends the call with TT_ENOMEM before any
    # device work (no GPU needed)
    calls = []

    def alloc(nbytes, stream, ctx):
        calls.append(nbytes)
        return None

    def free(p, stream, ctx):
        raise AssertionError("nothing was allocated")

    af, ff = tu.ALLOC_FN(alloc), tu.FREE_FN(free)
    A = np.ones((4, 5, 6), np.float32)
    o = tu.tt_opts()
    L.tt_opts_default(ctypes.byref(o))
    o.reverse = reverse
    res = tu.tt_result()
    st = L.tt_utv(ctypes.c_void_p(A.ctypes.data), 0, 3, tu._i64(A.shape), 0.1, None, 0, 0,
                  ctypes.byref(o), af, ff, None, None, ctypes.byref(res))
    assert st == 3                                   # TT_ENOMEM
    assert b"allocator returned NULL" in L.tt_last_error()
    assert calls and calls[0] >= A.nbytes
    assert all(res.cores[k] is None for k in range(3))


def test_power_iters_option(L):
    o = tu.tt_opts()
    L.tt_opts_default(ctypes.byref(o))
    assert o.power_iters == 0
    for bad in (-1, 9):
        o.power_iters = bad
        assert _call(L, opts=ctypes.byref(o)) == 1


def test_direct_tails_option(L):
    o = tu.tt_opts()
    L.tt_opts_default(ctypes.byref(o))
    assert o.direct_tails == 0
    for bad in (-1, 2):
        o.direct_tails = bad
        assert _call(L, opts=ctypes.byref(o)) == 1


def test_binding_structs_match_the_header(tmp_path):
    # every field offset and the size of tt_opts and tt_result, from the C
    # compiler's view of include/ttutv.h, against the ctypes declarations
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ttutv.h"', "int main(void) {"]
    for st in (tu.tt_opts, tu.tt_result, tu.tt_shard):
        name = st.__name__
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    inc = os.path.join(os.path.dirname(__file__), "..", "include")
    subprocess.run([gcc, "-I", inc, str(src), "-o", str(tmp_path / "layout")], check=True)
    out = subprocess.run([str(tmp_path / "layout")], capture_output=True, text=True, check=True).stdout
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}
    for st in (tu.tt_opts, tu.tt_result, tu.tt_shard):
        name = st.__name__
        assert got[(name, "size")] == ctypes.sizeof(st)
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, (name, f)


def test_sharded_arguments_rejected(L):
    # the partition is validated before any device work
    dims = tu._i64([8, 6, 5])
    res = tu.tt_result()

    def call(shard, direction=tu.TT_RL, opts=None, variant=tu.TT_URV):
        return L.tt_utv_sharded(ctypes.c_void_p(16), tu.TT_F32, 3, dims, 1e-2, None, variant,
                                direction, opts, tu.ALLOC_FN(), tu.FREE_FN(), None, None,
                                ctypes.byref(shard) if shard is not None else None, ctypes.byref(res))

    assert call(None) == 1                                   # no shard
    noop_r = tu.ALLREDUCE_FN(lambda *a: 0)
    noop_g = tu.ALLGATHER_FN(lambda *a: 0)
    assert call(tu.tt_shard(2, 2, noop_r, noop_g, None)) == 1    # rank out of range
    assert call(tu.tt_shard(3, 0, noop_r, noop_g, None)) == 1    # mode 1 (8) not a multiple of 3
    assert call(tu.tt_shard(2, 0, noop_r, noop_g, None), direction=tu.TT_LR, variant=tu.TT_ULV) == 1  # mode 3 (5)
    assert call(tu.tt_shard(2, 0, tu.ALLREDUCE_FN(), tu.ALLGATHER_FN(), None)) == 1  # no callbacks
    o = tu.tt_opts()
    L.tt_opts_default(ctypes.byref(o))
    o.reverse = 1
    assert call(tu.tt_shard(2, 0, noop_r, noop_g, None), opts=ctypes.byref(o)) == 7   # reversed: unsupported


def test_eval_plan_arguments_rejected(L):
    """Plan creation validates its shape before any device work; the plan
    calls reject a NULL plan; destroying NULL is a no-op."""
    dims, ranks = tu._i64([3, 4]), tu._i64([1, 2, 1])
    out = ctypes.c_void_p()
    idx = ctypes.c_void_p(1)

    def create(d=2, dm=dims, rk=ranks, n=4, alloc=None, free=None, o=True):
        return L.tt_eval_plan_create(d, dm, rk, idx, n, alloc or tu.ALLOC_FN(0),
                                     free or tu.FREE_FN(0), None, None,
                                     ctypes.byref(out) if o else None)

    assert create(o=False) == 1
    assert create(d=0) == 1 and create(d=17, dm=tu._i64([2] * 17), rk=tu._i64([1] * 18)) == 1
    assert create(rk=tu._i64([1, 65, 1])) == 1 and create(rk=tu._i64([2, 2, 1])) == 1
    assert create(dm=tu._i64([3, 0])) == 1 and create(dm=tu._i64([3, 1 << 31])) == 1
    assert create(n=-1) == 1 and create(n=1 << 31) == 1
    assert create(alloc=tu.ALLOC_FN(lambda b, s, c: None)) == 1      # alloc without free
    assert out.value is None
    assert L.tt_last_error() != b""
    ptrs = (ctypes.c_void_p * 2)(1, 1)
    assert L.tt_eval_plan_at(None, ptrs, ctypes.c_void_p(1), None) == 1
    assert L.tt_eval_plan_backward(None, ptrs, ctypes.c_void_p(1), ptrs, None) == 1
    assert L.tt_eval_plan_backward_mixed(None, ptrs, ptrs, ctypes.c_void_p(1), ptrs, None) == 1
    assert L.tt_tangent_project(None, ptrs, ptrs, ctypes.c_void_p(1), ptrs, None) == 1
    # orthogonalization: d, dtype, side, rank and aliasing checks (no kernel runs)
    D, R = tu._i64([3, 4]), tu._i64([1, 2, 1])
    w = ctypes.c_void_p(1)
    assert L.tt_orthogonalize(1, D, R, ptrs, 0, 1, ptrs, w, None) == 1
    assert L.tt_orthogonalize(2, D, R, ptrs, 5, 1, ptrs, w, None) == 1
    assert L.tt_orthogonalize(2, D, R, ptrs, 0, 2, ptrs, w, None) == 1
    assert L.tt_orthogonalize(2, D, tu._i64([1, 4, 1]), ptrs, 0, 1, ptrs, w, None) == 1
    assert L.tt_orthogonalize(2, D, R, ptrs, 0, 1, ptrs, w, None) == 1   # out aliases cores
    assert L.tt_orthogonalize_work_bytes(2, D, R, 0) > 0
    L.tt_eval_plan_destroy(None, None)
    assert L.tt_eval_plan_device_bytes(None) == 0


def test_wait_selftest_arguments_rejected(L):
    assert L.tt_wait_selftest(0, 0, None) == 1
    assert L.tt_wait_selftest(1, -5, None) == 1
    assert L.tt_wait_selftest(0, 20_000_000_000, None) == 1

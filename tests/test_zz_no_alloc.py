"""tt_full_noalloc: the contraction of TT cores into a full tensor without any
device allocation.

Some callers cannot allocate device memory while they run -- for example code
whose device memory is entirely held by another allocator's pool, or a
latency-critical loop that must not pay cudaMalloc's implicit device
synchronization.  tt_full_noalloc serves them with a fixed 32 MiB scratch array
in the library's static device memory.  This test calls it through the C ABI
and checks its result against tt_full (which takes a caller-allocated work
buffer), on calls in a row with different shapes -- one of them with inner
ranks large enough that the contraction splits its inner dimension and keeps
FP64 partial sums in the scratch -- so stale contents left in the shared
scratch by one call cannot leak into the next.  A second test checks that,
once the first call on the device has loaded the array, further calls change
neither the device's free memory nor torch's reserved bytes.  It lives in a
file collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tu():
    import paper_2501_07904_gb300 as m
    if not os.path.exists(m.LIB_PATH):
        from paper_2501_07904_gb300 import build
        build.build()
    assert torch.cuda.is_available()
    m.lib()
    return m


def _meta(cores):
    dims = [int(g.shape[1]) for g in cores]
    ranks = [1] + [int(g.shape[2]) for g in cores]
    return dims, ranks


def full_with_work(tu, cores, dtype_code):
    """tt_full with a work buffer allocated by the caller (torch)."""
    L = tu.lib()
    dims, ranks = _meta(cores)
    D, R = tu._i64(dims), tu._i64(ranks)
    out = torch.empty(dims, dtype=cores[0].dtype, device="cuda")
    work = torch.empty(int(L.tt_full_work_bytes(len(cores), D, R, dtype_code)), dtype=torch.uint8,
                       device="cuda")
    ptrs = (ctypes.c_void_p * len(cores))(*[c.data_ptr() for c in cores])
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.tt_full(len(cores), D, R, ptrs, dtype_code, ctypes.c_void_p(out.data_ptr()),
                     ctypes.c_void_p(work.data_ptr()), st) == 0, L.tt_last_error()
    return out


def full_noalloc(tu, cores, dtype_code):
    L = tu.lib()
    dims, ranks = _meta(cores)
    out = torch.empty(dims, dtype=cores[0].dtype, device="cuda")
    ptrs = (ctypes.c_void_p * len(cores))(*[c.data_ptr() for c in cores])
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = L.tt_full_noalloc(len(cores), tu._i64(dims), tu._i64(ranks), ptrs, dtype_code,
                               ctypes.c_void_p(out.data_ptr()), st)
    assert status == 0, L.tt_last_error()
    return out


CASES = [
    # (dims, ranks incl. r_0 = r_d = 1, torch dtype, C-ABI dtype code, relative tolerance)
    ((40, 33, 27, 21), (1, 7, 13, 5, 1), torch.float32, 0, 1e-6),
    # inner ranks of 300 and 280 over few output rows: the contraction splits
    # its inner dimension (FP64 partials in the scratch)
    ((6, 10, 5), (1, 300, 280, 1), torch.float32, 0, 1e-6),
    ((96, 80, 64), (1, 24, 16, 1), torch.float64, 1, 1e-14),
]


def _cores(i):
    dims, ranks, tdt, _, _ = CASES[i]
    return [torch.from_numpy(c).to(tdt).cuda().contiguous()
            for c in synth.gaussian_cores(dims, ranks, seed=100 + i)]


def test_split_case_uses_split_partials(tu):
    # the second case's work size includes FP64 partials beyond the two
    # intermediate buffers of an unsplit contraction
    dims, ranks, _, code, _ = CASES[1]
    L = tu.lib()
    need = int(L.tt_full_work_bytes(3, tu._i64(dims), tu._i64(ranks), code))
    inter = 2 * (6 * 10 * 280 * 4 + 256)
    assert need > inter + 6 * 10 * 280 * 8


def test_noalloc_matches_tt_full_twice_in_a_row(tu):
    for rep in range(2):
        for i, (dims, ranks, tdt, code, tol) in enumerate(CASES):
            cores = _cores(i)
            ref = full_with_work(tu, cores, code)
            got = full_noalloc(tu, cores, code)
            torch.cuda.synchronize()
            err = (got.double() - ref.double()).norm() / ref.double().norm()
            assert err.item() <= tol, (rep, dims, err.item())


def test_noalloc_allocates_nothing_after_first_call(tu):
    inputs = [(_cores(i), CASES[i][3]) for i in range(len(CASES))]
    outs = [torch.empty(CASES[i][0], dtype=CASES[i][2], device="cuda") for i in range(len(CASES))]
    L = tu.lib()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(i):
        cores, code = inputs[i]
        dims, ranks = _meta(cores)
        ptrs = (ctypes.c_void_p * len(cores))(*[c.data_ptr() for c in cores])
        assert L.tt_full_noalloc(len(cores), tu._i64(dims), tu._i64(ranks), ptrs, code,
                                 ctypes.c_void_p(outs[i].data_ptr()), st) == 0, L.tt_last_error()

    for i in range(len(CASES)):   # the first calls may load the module (and its array)
        call(i)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    for i in range(len(CASES)):
        call(i)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_reserved() == res0
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_contractions_above_its_scratch(tu):
    L = tu.lib()
    limit = int(L.tt_full_noalloc_max_work_bytes())
    assert limit == 32 << 20
    dims, ranks = [4096, 64, 64], [1, 64, 64, 1]      # intermediates of 4096*64*64 floats
    need = L.tt_full_work_bytes(3, tu._i64(dims), tu._i64(ranks), 0)
    assert need > limit
    ptrs = (ctypes.c_void_p * 3)(1, 1, 1)
    status = L.tt_full_noalloc(3, tu._i64(dims), tu._i64(ranks), ptrs, 0, ctypes.c_void_p(1), None)
    assert status == 1
    assert b"scratch" in L.tt_last_error()

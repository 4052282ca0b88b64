"""The partitioned sweep (tt_utv_sharded) against the whole-tensor sweep and
the FP64 oracle, on one GPU: P ranks are P host threads, each with its own
CUDA stream and its slab of the tensor, and the collectives are staged
through host memory (each rank synchronizes its stream, the partial sums are
added in rank order, every rank copies the same total back).  No kernel
waits for another rank: the ranks meet only on the host, at barriers with a
time limit, so a failing rank ends the test instead of stalling it.

Checked: ranks equal to the whole-tensor sweep's and the oracle's, the
represented tensor equal to the whole-tensor sweep's (up to the summation
order of the partial sums) and to the oracle's within the test tolerance,
every rank holding the same result, steps with identity sketches (the
whole unfolding gathered) and the partitioned last core gathered."""
import threading

import numpy as np
import pytest
import torch

import synth
from oracle import tt as otc
from test_gpu_parity import np_cores, rel_diff, tu  # noqa: F401

pytestmark = pytest.mark.gpu


class HostHub:
    def __init__(self, nranks, timeout=120.0):
        self.n = nranks
        self.slots = [None] * nranks
        self.bar = threading.Barrier(nranks, timeout=timeout)


class ThreadComm:
    """Host-staged collectives among the threads of one process."""

    def __new__(cls, rank, nranks, device, hub):
        import paper_2501_07904_gb300 as m

        class _C(m.ShardComm):
            def allreduce(self, t):
                torch.cuda.current_stream().synchronize()
                hub.slots[self.rank] = t.cpu()
                hub.bar.wait()
                total = hub.slots[0].clone()
                for r in range(1, hub.n):
                    total += hub.slots[r]
                hub.bar.wait()
                t.copy_(total)
                torch.cuda.current_stream().synchronize()

            def allgather(self, send, recv):
                torch.cuda.current_stream().synchronize()
                hub.slots[self.rank] = send.cpu()
                hub.bar.wait()
                whole = torch.cat([hub.slots[r] for r in range(hub.n)])
                hub.bar.wait()
                recv.copy_(whole)
                torch.cuda.current_stream().synchronize()

        return _C(rank, nranks, device)


def run_sharded(tu, A, P, **kw):
    direction = kw.get("direction") or ("RL" if kw.get("variant", "URV") == "URV" else "LR")
    hub = HostHub(P)
    dev = torch.device("cuda", 0)
    A_t = torch.from_numpy(np.ascontiguousarray(A))
    out, errs = [None] * P, [None] * P

    def work(r):
        try:
            torch.cuda.set_device(0)
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                local = tu.slab(A_t, P, r, direction).to(dev, non_blocking=False)
                comm = ThreadComm(r, P, dev, hub)
                res = tu.tt_utv_sharded(local, list(A.shape), comm, **kw)
                s.synchronize()
                out[r] = (res, comm.calls)
        except BaseException as e:  # noqa: BLE001
            errs[r] = e
            hub.bar.abort()

    th = [threading.Thread(target=work, args=(r,)) for r in range(P)]
    for t in th:
        t.start()
    for t in th:
        t.join(300)
    for e in errs:
        if e is not None:
            raise e
    return out


CASES = [
    # (tensor, sweep, tolerance against the oracle): URV partitions mode 1,
    # ULV mode 4; the small partitioned mode (16) makes the last step's
    # sketch the identity, so that unfolding is gathered
    (synth.gaussian_tt((16, 29, 41, 24), (1, 5, 7, 4, 1), 1e-6, seed=61, dtype=np.float32), "URV"),
    (synth.gaussian_tt((24, 41, 29, 16), (1, 4, 7, 5, 1), 1e-6, seed=62, dtype=np.float32), "ULV"),
]


@pytest.mark.parametrize("precision, tol", [("fp64", 1e-10), ("fp32", 1e-5), ("mixed", 5e-5)])
@pytest.mark.parametrize("case", [0, 1])
@pytest.mark.parametrize("l_full", [256, 24])
@pytest.mark.parametrize("P", [2, 4])
def test_sharded_equals_whole(tu, P, l_full, case, precision, tol):
    A, variant = CASES[case]
    if precision == "fp64":
        A = A.astype(np.float64)
    kw = dict(eps=1e-3, variant=variant, precision=precision, l_full=l_full)
    whole = tu.tt_utv(torch.from_numpy(np.ascontiguousarray(A)).cuda(), **kw)
    ref = otc.tt_utv(np.asarray(A, np.float64), eps=1e-3, variant=variant, l_full=l_full)
    outs = run_sharded(tu, A, P, **kw)
    normA2 = ref["normA2"]
    c_whole = np_cores(whole)
    for r, (res, calls) in enumerate(outs):
        assert calls > 0
        assert res.ranks == whole.ranks == ref["ranks"], (r, res.ranks, whole.ranks, ref["ranks"])
        assert res.sketch_l == whole.sketch_l
        assert abs(res.norm_sq - whole.norm_sq) <= 1e-12 * whole.norm_sq
        c = np_cores(res)
        d_whole = rel_diff(c, c_whole, normA2)
        d_ref = rel_diff(c, ref["cores"], normA2)
        print(f"SHARD P={P} {variant} {precision} l_full={l_full} rank={r} vs_whole={d_whole:.2e} "
              f"vs_oracle={d_ref:.2e} sketch={res.sketch_l}")
        # FP64 partials are summed in another order than the whole sweep's
        # products; in FP32 a sketched step carries that rounding into its
        # basis, so there the partitioned and whole results agree only to
        # the precision's own error band
        bound = max(1e-12, tol / 10) if precision == "fp64" or sum(res.sketch_l) == 0 else tol / 2
        assert d_whole <= bound, d_whole
        assert d_ref <= tol, d_ref
    # every rank returns the same cores
    c0 = [g.cpu() for g in outs[0][0].cores]
    for res, _ in outs[1:]:
        for a, b in zip(c0, res.cores):
            assert torch.equal(a, b.cpu())


def test_sharded_one_rank_is_tt_utv(tu):
    A, variant = CASES[0]
    kw = dict(eps=1e-3, variant=variant, l_full=24)
    whole = tu.tt_utv(torch.from_numpy(A).cuda(), **kw)
    (res, calls), = run_sharded(tu, A, 1, **kw)
    assert calls == 0
    assert res.ranks == whole.ranks
    for a, b in zip(res.cores, whole.cores):
        assert torch.equal(a, b)


@pytest.mark.parametrize("variant", ["URV", "ULV"])
def test_sharded_direct_tails(tu, variant):
    # noise 1e-3 at eps 1e-2: no step is tight, so every step but an identity
    # sketch sums its residual per slab and all-reduces it
    dims = (16, 29, 41, 24) if variant == "URV" else (24, 41, 29, 16)
    ranks = (1, 5, 7, 4, 1) if variant == "URV" else (1, 4, 7, 5, 1)
    A = synth.gaussian_tt(dims, ranks, 1e-3, seed=63, dtype=np.float32)
    kw = dict(eps=1e-2, variant=variant, precision="mixed", l_full=24, direct_tails=True)
    A_t = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    whole = tu.tt_utv(A_t, **kw)
    outs = run_sharded(tu, A, 2, **kw)
    t0 = outs[0][0].tail_sq
    for res, _ in outs:
        assert res.ranks == whole.ranks
        assert res.tail_sq == t0                   # the all-reduced sums are the same bits
        err2, normA2 = tu.tt_rse(A_t, res.cores)
        assert abs(sum(res.tail_sq) - err2) <= 0.03 * err2, (res.tail_sq, err2)
        for a, b in zip(res.tail_sq, whole.tail_sq):
            assert abs(a - b) <= 0.02 * b + 1e-9 * normA2, (res.tail_sq, whole.tail_sq)

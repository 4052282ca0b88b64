"""Python binding of the GB300 TT-UTV library (libttutv.so, include/ttutv.h).

Argument marshalling only: every step of the sweep runs in the library's CUDA
kernels.  PyTorch provides device memory (the library allocates through
callbacks into torch's caching allocator) and the stream.  If the library is
not built this module raises; there is no CPU fallback.

    import paper_2501_07904_gb300 as tu
    res = tu.tt_utv(A_cuda, eps=1e-2, variant="URV")      # TT-URV, right-to-left
    res.cores, res.ranks, res.tail_sq
    X = tu.tt_full(res.cores)                             # Eq. TT
    x = tu.TTEvalMasked.apply(idx, *cores)                # masked evaluation, autograd
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from dataclasses import dataclass, field

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
# TTUTV_CHECKED=1 loads the bounds-checked build (libttutv_bc.so) instead
LIB_PATH = os.path.join(_PKG, "libttutv_bc.so" if os.environ.get("TTUTV_CHECKED") == "1"
                        else "libttutv.so")
TT_MAXD = 16

STATUS = {0: "TT_OK", 1: "TT_EINVAL", 2: "TT_ENONFINITE", 3: "TT_ENOMEM", 4: "TT_ECUDA",
          5: "TT_ENOCONV", 6: "TT_ETIMEOUT", 7: "TT_EUNSUPPORTED"}
for _code, _name in STATUS.items():
    globals()[_name] = _code
PRECISION = {"fp64": 0, "fp32": 1, "mixed": 2}
SMALL = {"auto": 0, "fp32": 1, "fp64": 2, "df": 3}
INNER = {"qlp": 0, "usvp": 1, "lurv": 2}
TT_F32, TT_F64 = 0, 1
TT_URV, TT_ULV = 0, 1
TT_RL, TT_LR = 0, 1

# Every symbol include/ttutv.h declares.
EXPORTS = ["tt_opts_default", "tt_utv", "tt_utv_sharded", "tt_svd", "tt_result_free",
           "tt_full_work_bytes",
           "tt_full", "tt_full_noalloc", "tt_orthogonalize_work_bytes", "tt_orthogonalize", "tt_full_noalloc_max_work_bytes", "tt_rse_work_bytes",
           "tt_rse", "tt_eval_plan_create", "tt_eval_plan_destroy", "tt_eval_plan_device_bytes",
           "tt_eval_plan_at", "tt_eval_plan_backward", "tt_eval_plan_backward_mixed",
           "tt_tangent_project", "tt_tangent_eval", "tt_eval_at",
           "tt_eval_at_backward", "tt_sketch_matrix", "tt_wait_selftest", "tt_bounds_violations",
           "tt_kernel_launches",
           "tt_last_error",
           "tt_version"]
PHASES = ["gram", "small", "carry", "core", "sketch", "orth", "project"]
TT_NPHASES = 8


class TTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class tt_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("small_precision", ctypes.c_int32),
                ("oversample", ctypes.c_int32), ("l_full", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("weights", ctypes.POINTER(ctypes.c_double)),
                ("orth_precision", ctypes.c_int32), ("reverse", ctypes.c_int32),
                ("phase_ms", ctypes.POINTER(ctypes.c_double)),
                ("power_iters", ctypes.c_int32), ("inner", ctypes.c_int32),
                ("usvp_iters", ctypes.c_int32), ("lhat", ctypes.c_int32),
                ("direct_tails", ctypes.c_int32)]


class tt_result(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("dtype", ctypes.c_int32), ("orth", ctypes.c_int32),
                ("pad_", ctypes.c_int32),
                ("dims", ctypes.c_int64 * TT_MAXD), ("ranks", ctypes.c_int64 * (TT_MAXD + 1)),
                ("cores", ctypes.c_void_p * TT_MAXD), ("norm_sq", ctypes.c_double),
                ("tail_sq", ctypes.c_double * TT_MAXD), ("delta_sq", ctypes.c_double * TT_MAXD),
                ("sketch_l", ctypes.c_int32 * TT_MAXD), ("small_fp64", ctypes.c_int32 * TT_MAXD)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                ctypes.c_void_p)
ALLGATHER_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                ctypes.c_void_p, ctypes.c_void_p)


class tt_shard(ctypes.Structure):
    _fields_ = [("nranks", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("allreduce", ALLREDUCE_FN), ("allgather", ALLGATHER_FN),
                ("ctx", ctypes.c_void_p)]

_lib_handle = None


def lib():
    """Load libttutv.so (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2501_07904_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64, U64, D, SZ = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                               ctypes.c_double, ctypes.c_size_t)
    PI64 = ctypes.POINTER(ctypes.c_int64)
    L.tt_opts_default.argtypes = [ctypes.POINTER(tt_opts)]
    L.tt_opts_default.restype = None
    L.tt_utv.argtypes = [P, I32, I32, PI64, D, PI64, I32, I32, ctypes.POINTER(tt_opts), ALLOC_FN,
                         FREE_FN, P, P, ctypes.POINTER(tt_result)]
    L.tt_utv.restype = I32
    L.tt_utv_sharded.argtypes = [P, I32, I32, PI64, D, PI64, I32, I32, ctypes.POINTER(tt_opts),
                                 ALLOC_FN, FREE_FN, P, P, ctypes.POINTER(tt_shard),
                                 ctypes.POINTER(tt_result)]
    L.tt_utv_sharded.restype = I32
    L.tt_svd.argtypes = [P, I32, I32, PI64, D, PI64, I32, ctypes.POINTER(tt_opts), ALLOC_FN,
                         FREE_FN, P, P, ctypes.POINTER(tt_result)]
    L.tt_svd.restype = I32
    L.tt_result_free.argtypes = [ctypes.POINTER(tt_result), FREE_FN, P, P]
    L.tt_result_free.restype = None
    L.tt_full_work_bytes.argtypes = [I32, PI64, PI64, I32]
    L.tt_full_work_bytes.restype = SZ
    L.tt_full.argtypes = [I32, PI64, PI64, ctypes.POINTER(P), I32, P, P, P]
    L.tt_full.restype = I32
    L.tt_full_noalloc.argtypes = [I32, PI64, PI64, ctypes.POINTER(P), I32, P, P]
    L.tt_full_noalloc.restype = I32
    L.tt_full_noalloc_max_work_bytes.argtypes = []
    L.tt_full_noalloc_max_work_bytes.restype = SZ
    L.tt_rse_work_bytes.argtypes = [I32, PI64, PI64, I32]
    L.tt_rse_work_bytes.restype = SZ
    L.tt_orthogonalize_work_bytes.argtypes = [I32, PI64, PI64, I32]
    L.tt_orthogonalize_work_bytes.restype = SZ
    L.tt_orthogonalize.argtypes = [I32, PI64, PI64, ctypes.POINTER(P), I32, I32, ctypes.POINTER(P),
                                   P, P]
    L.tt_orthogonalize.restype = I32
    L.tt_rse.argtypes = [I32, PI64, PI64, ctypes.POINTER(P), I32, P, P, P, P]
    L.tt_rse.restype = I32
    L.tt_eval_plan_create.argtypes = [I32, PI64, PI64, P, I64, ALLOC_FN, FREE_FN, P, P,
                                      ctypes.POINTER(P)]
    L.tt_eval_plan_create.restype = I32
    L.tt_eval_plan_destroy.argtypes = [P, P]
    L.tt_eval_plan_destroy.restype = None
    L.tt_eval_plan_device_bytes.argtypes = [P]
    L.tt_eval_plan_device_bytes.restype = SZ
    L.tt_eval_plan_at.argtypes = [P, ctypes.POINTER(P), P, P]
    L.tt_eval_plan_at.restype = I32
    L.tt_eval_plan_backward.argtypes = [P, ctypes.POINTER(P), P, ctypes.POINTER(P), P]
    L.tt_eval_plan_backward.restype = I32
    L.tt_eval_plan_backward_mixed.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), P,
                                              ctypes.POINTER(P), P]
    L.tt_eval_plan_backward_mixed.restype = I32
    L.tt_tangent_project.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), P, ctypes.POINTER(P), P]
    L.tt_tangent_project.restype = I32
    L.tt_tangent_eval.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), P, P]
    L.tt_tangent_eval.restype = I32
    L.tt_eval_at.argtypes = [I32, PI64, PI64, ctypes.POINTER(P), P, I64, P, P]
    L.tt_eval_at.restype = I32
    L.tt_eval_at_backward.argtypes = [I32, PI64, PI64, ctypes.POINTER(P), P, I64, P,
                                      ctypes.POINTER(P), P]
    L.tt_eval_at_backward.restype = I32
    L.tt_sketch_matrix.argtypes = [I64, I64, U64, I32, I32, P, P]
    L.tt_sketch_matrix.restype = I32
    L.tt_wait_selftest.argtypes = [I32, I64, P]
    L.tt_wait_selftest.restype = I32
    L.tt_kernel_launches.argtypes = []
    L.tt_bounds_violations.argtypes = [ctypes.POINTER(I32), I32]
    L.tt_bounds_violations.restype = I64
    L.tt_kernel_launches.restype = ctypes.c_uint64
    L.tt_last_error.argtypes = []
    L.tt_last_error.restype = ctypes.c_char_p
    L.tt_version.argtypes = []
    L.tt_version.restype = ctypes.c_char_p
    _lib_handle = L
    return L


def _check(status):
    if status != 0:
        raise TTError(status, lib().tt_last_error().decode())


def _i64(seq):
    return (ctypes.c_int64 * max(1, len(seq)))(*[int(x) for x in seq])


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream, ctypes.c_void_p(stream.cuda_stream)


class _TorchAllocator:
    """Allocation callbacks into torch's caching allocator (stream-ordered)."""

    def __init__(self, device):
        self.device = device
        self.live = {}
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)

    def _do_alloc(self, nbytes, stream, ctx):
        try:
            t = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        except RuntimeError:
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _do_free(self, p, stream, ctx):
        self.live.pop(p, None)

    def take(self, ptr, shape, dtype):
        buf = self.live.pop(ptr)
        n = math.prod(shape)
        el = _ELSIZE[dtype]
        return buf[: n * el].view(dtype).view(shape)


_ELSIZE = {torch.float32: 4, torch.float64: 8}
_tls = threading.local()


def _allocator(device):
    """The calling thread's allocator for ``device`` (its ctypes callbacks are
    built once and reused by every call on that thread)."""
    cache = getattr(_tls, "alloc", None)
    if cache is None:
        cache = _tls.alloc = {}
    a = cache.get(device)
    if a is None:
        a = cache[device] = _TorchAllocator(device)
    a.live.clear()
    return a


@dataclass
class TTResult:
    """Cores G_k (device, shape (r_{k-1}, I_k, r_k)) and per-unfolding records."""
    cores: list
    ranks: list
    norm_sq: float
    tail_sq: list           # ||E_k||_F^2 per unfolding k = 1..d-1
    delta_sq: list          # eps_k^2 per unfolding (0 for fixed ranks)
    sketch_l: list          # 0 = exact Gram path, else sketch width
    small_fp64: list
    orth: str               # "right" (cores 2..d) or "left" (cores 1..d-1)
    info: dict = field(default_factory=dict)


def _sweep(fn, A, eps, ranks, extra, precision, seed, oversample, l_full, small, weights, stream,
           timing=False, orth="auto", reverse=False, power_iters=0, dims=None, shard=None,
           inner="qlp", usvp_iters=8, lhat="full", direct_tails=False):
    if not isinstance(A, torch.Tensor):
        raise TypeError("A must be a torch.Tensor")
    if A.dtype not in (torch.float32, torch.float64):
        raise TypeError("A must be float32 or float64")
    A = A.contiguous()
    d = A.dim()
    dims = list(A.shape) if dims is None else [int(x) for x in dims]
    if len(dims) != d:
        raise ValueError("dims must have one entry per mode of A")
    dev = A.device if A.is_cuda else torch.device("cuda", torch.cuda.current_device())
    st, st_ptr = _stream(stream)
    opts = tt_opts()
    lib().tt_opts_default(ctypes.byref(opts))
    opts.precision = PRECISION[precision]
    opts.small_precision = SMALL[small]
    opts.orth_precision = SMALL[orth]
    opts.oversample = int(oversample)
    opts.l_full = int(l_full)
    opts.seed = int(seed)
    opts.reverse = 1 if reverse else 0
    opts.power_iters = int(power_iters)
    opts.inner = INNER[inner]
    opts.usvp_iters = int(usvp_iters)
    opts.lhat = {"full": 0, "l11": 1}[lhat]
    opts.direct_tails = 1 if direct_tails else 0
    wbuf = None
    if weights is not None:
        wbuf = (ctypes.c_double * len(weights))(*[float(x) for x in weights])
        opts.weights = ctypes.cast(wbuf, ctypes.POINTER(ctypes.c_double))
    tbuf = None
    if timing:
        tbuf = (ctypes.c_double * (TT_MAXD * TT_NPHASES))()
        opts.phase_ms = ctypes.cast(tbuf, ctypes.POINTER(ctypes.c_double))
    dims = _i64(dims)
    fr = _i64(ranks) if ranks is not None else None
    alloc = _allocator(dev)
    res = tt_result()
    dtype = TT_F64 if A.dtype == torch.float64 else TT_F32
    with torch.cuda.device(dev), torch.cuda.stream(st):
        tail = (ctypes.byref(shard.cstruct),) if shard is not None else ()
        status = fn(ctypes.c_void_p(A.data_ptr()), dtype, d, dims,
                    float(eps) if eps is not None else 0.0, fr, *extra, ctypes.byref(opts),
                    alloc._alloc, alloc._free, None, st_ptr, *tail, ctypes.byref(res))
        if status != 0:
            msg = lib().tt_last_error().decode()
            alloc.live.clear()
            raise TTError(status, msg)
        out_dtype = torch.float64 if res.dtype == TT_F64 else torch.float32
        rk = [int(res.ranks[k]) for k in range(d + 1)]
        cores = [alloc.take(res.cores[k], (rk[k], int(res.dims[k]), rk[k + 1]), out_dtype)
                 for k in range(d)]
    alloc.live.clear()
    info = {}
    if timing:
        info["phase_ms"] = [{ph: tbuf[s * TT_NPHASES + i] for i, ph in enumerate(PHASES)}
                            for s in range(d - 1)]
    return TTResult(cores=cores, ranks=rk, norm_sq=float(res.norm_sq),
                    tail_sq=[float(res.tail_sq[k]) for k in range(d - 1)],
                    delta_sq=[float(res.delta_sq[k]) for k in range(d - 1)],
                    sketch_l=[int(res.sketch_l[k]) for k in range(d - 1)],
                    small_fp64=[int(res.small_fp64[k]) for k in range(d - 1)],
                    orth="right" if res.orth == 0 else "left", info=info)


def tt_utv(A, eps=None, ranks=None, variant="URV", precision="fp32", seed=0, oversample=16,
           l_full=256, small="auto", weights=None, stream=None, timing=False, orth="auto",
           reverse=False, direction=None, power_iters=0, inner="qlp", usvp_iters=8,
           lhat="full", direct_tails=False):
    """TT-URV right-to-left (Alg. 3) or TT-ULV left-to-right (Alg. 1/2).

    Give ``eps`` (prescribed relative accuracy, Alg. 2) or ``ranks``
    (r_1..r_{d-1}).  ``A`` may live on the GPU or on the host (copied in).
    ``direction`` defaults to the variant's recommended sweep ("RL" for URV,
    "LR" for ULV); ULV with "RL" is the appendix's Alg. 4 keeping
    [L_11; L_21], which computes the URV right-to-left sweep (and URV with
    "LR" the ULV left-to-right one).  ``reverse`` factors the index-reversed
    tensor and returns its cores read back as cores of ``A`` (Remark after
    Thm 3.2: URV then gives a left-orthogonal TT).  ``power_iters`` adds q
    subspace iterations to every sketched range.  ``inner`` picks the small
    rank-revealing factor: "qlp" (pivoted QLP), "usvp" (USV-plus-style
    deflation) or "lurv" (Givens-based low-rank URV warm-started from a
    pivoted QR), the last two with ``usvp_iters`` power iterations per basis
    vector.
    ``lhat="l11"`` with variant "ULV" and direction "RL" runs the appendix's
    Alg. 4 as printed: the carry keeps L_11 alone and the default weights are
    1/(d-1).  ``direct_tails`` makes every non-tight step report its error
    ||E_k||^2 summed directly from its residual (one more pass over the
    unfolding) instead of as ||C||^2 - ||carry||^2; ranks and cores are the
    same.
    """
    if (eps is None) == (ranks is None):
        raise ValueError("give exactly one of eps or ranks")
    if direction is None:
        direction = "RL" if variant == "URV" else "LR"
    v = ({"URV": TT_URV, "ULV": TT_ULV}[variant], {"RL": TT_RL, "LR": TT_LR}[direction])
    return _sweep(lib().tt_utv, A, eps, ranks, v, precision, seed, oversample, l_full, small,
                  weights, stream, timing, orth, reverse, power_iters, inner=inner,
                  usvp_iters=usvp_iters, lhat=lhat, direct_tails=direct_tails)


class _DevBuf:
    """A raw device pointer seen as a 1-D torch tensor (no copy)."""

    def __init__(self, ptr, n, typestr, device):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}
        self.device = device


def _device_view(ptr, n, dtype, device):
    typestr = {torch.float64: "<f8", torch.uint8: "|u1"}[dtype]
    return torch.as_tensor(_DevBuf(ptr, n, typestr, device), device=device)


class ShardComm:
    """Communication of one rank of a partitioned sweep (tt_utv_sharded).

    allreduce(t) sums a 1-D FP64 device tensor over the ranks in place;
    allgather(send, recv) concatenates 1-D uint8 device tensors in rank
    order.  Both are called on the sweep's host thread with the sweep's CUDA
    stream current and must order their work on it.  Subclasses provide the
    transport; the C callbacks built here only wrap the library's raw device
    pointers as tensors."""

    def __init__(self, rank, nranks, device):
        self.rank, self.nranks, self.device = int(rank), int(nranks), torch.device(device)
        self._ar = ALLREDUCE_FN(self._c_allreduce)
        self._ag = ALLGATHER_FN(self._c_allgather)
        self.cstruct = tt_shard(self.nranks, self.rank, self._ar, self._ag, None)
        self.calls = 0

    def _c_allreduce(self, ptr, count, stream, ctx):
        try:
            with torch.cuda.stream(torch.cuda.ExternalStream(stream or 0, device=self.device)):
                self.allreduce(_device_view(ptr, count, torch.float64, self.device))
            self.calls += 1
            return 0
        except Exception:  # reported to the library as a failed collective
            return 4

    def _c_allgather(self, send, recv, nbytes, stream, ctx):
        try:
            with torch.cuda.stream(torch.cuda.ExternalStream(stream or 0, device=self.device)):
                self.allgather(_device_view(send, nbytes, torch.uint8, self.device),
                               _device_view(recv, nbytes * self.nranks, torch.uint8, self.device))
            self.calls += 1
            return 0
        except Exception:
            return 4

    def allreduce(self, t):
        raise NotImplementedError

    def allgather(self, send, recv):
        raise NotImplementedError


class TorchDistComm(ShardComm):
    """torch.distributed transport (NCCL for one GPU per process, the usual
    multi-GPU launch).  The sweep's stream is current, so the collectives are
    ordered after the work that produced their input and before what reads
    their output."""

    def __init__(self, group=None, device=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        super().__init__(dist.get_rank(group), dist.get_world_size(group), dev)

    def allreduce(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)

    def allgather(self, send, recv):
        self.dist.all_gather_into_tensor(recv, send, group=self.group)


def slab(A, nranks, rank, direction="RL"):
    """This rank's slab of the whole tensor A for tt_utv_sharded: an equal part
    of mode 1 (right-to-left sweep) or of mode d (left-to-right sweep)."""
    axis = 0 if direction == "RL" else A.dim() - 1
    size = A.shape[axis]
    if size % nranks:
        raise ValueError(f"mode {axis + 1} ({size}) does not split into {nranks} equal slabs")
    b = size // nranks
    return A.narrow(axis, rank * b, b).contiguous()


def tt_utv_sharded(A_local, dims, comm, eps=None, ranks=None, variant="URV", direction=None,
                   precision="fp32", seed=0, oversample=16, l_full=256, small="auto", weights=None,
                   stream=None, timing=False, orth="auto", power_iters=0, direct_tails=False):
    """tt_utv of a tensor partitioned over ranks (one GPU each): A_local is this
    rank's slab (see slab()), dims the whole tensor's mode sizes, comm a
    ShardComm.  Every rank returns the whole result (with ``direct_tails`` a
    sketched step's residual is summed per slab and all-reduced)."""
    if (eps is None) == (ranks is None):
        raise ValueError("give exactly one of eps or ranks")
    if direction is None:
        direction = "RL" if variant == "URV" else "LR"
    v = ({"URV": TT_URV, "ULV": TT_ULV}[variant], {"RL": TT_RL, "LR": TT_LR}[direction])
    return _sweep(lib().tt_utv_sharded, A_local, eps, ranks, v, precision, seed, oversample, l_full,
                  small, weights, stream, timing, orth, False, power_iters, dims=dims, shard=comm,
                  direct_tails=direct_tails)


def tt_svd(A, eps=None, ranks=None, direction="LR", precision="fp32", l_full=256, small="auto",
           weights=None, stream=None, oversample=16):
    """TT-SVD (the paper's comparison method) through the same sweep.  A step
    whose basis side exceeds ``l_full`` factors the projection onto a
    Rademacher range of r + ``oversample`` columns (fixed ranks)."""
    if (eps is None) == (ranks is None):
        raise ValueError("give exactly one of eps or ranks")
    dr = {"LR": TT_LR, "RL": TT_RL}[direction]
    return _sweep(lib().tt_svd, A, eps, ranks, (dr,), precision, 0, oversample, l_full, small,
                  weights, stream)


def _core_meta(cores):
    d = len(cores)
    dims = [int(g.shape[1]) for g in cores]
    ranks = [int(cores[0].shape[0])] + [int(g.shape[2]) for g in cores]
    return d, dims, ranks


def tt_full(cores, stream=None):
    """Full tensor from TT cores (Eq. TT), computed by the library's GEMM."""
    d, dims, ranks = _core_meta(cores)
    dtype = cores[0].dtype
    cores = [g.contiguous() for g in cores]
    st, st_ptr = _stream(stream)
    code = TT_F64 if dtype == torch.float64 else TT_F32
    D, R = _i64(dims), _i64(ranks)
    nbytes = lib().tt_full_work_bytes(d, D, R, code)
    dev = cores[0].device
    with torch.cuda.device(dev), torch.cuda.stream(st):
        out = torch.empty(dims, dtype=dtype, device=dev)
        work = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=dev)
        ptrs = (ctypes.c_void_p * d)(*[g.data_ptr() for g in cores])
        _check(lib().tt_full(d, D, R, ptrs, code, ctypes.c_void_p(out.data_ptr()),
                             ctypes.c_void_p(work.data_ptr()), st_ptr))
    return out


def tt_orthogonalize(cores, side="left", stream=None):
    """The same TT tensor with left-orthogonal cores 1..d-1 (``side="left"``)
    or right-orthogonal cores 2..d (``"right"``), by Cholesky-QR2 of each
    core's unfolding (Def. 2.2; see tt_orthogonalize in ttutv.h)."""
    d, dims, ranks = _core_meta(cores)
    dtype = cores[0].dtype
    cores = [g.contiguous() for g in cores]
    st, st_ptr = _stream(stream)
    code = TT_F64 if dtype == torch.float64 else TT_F32
    D, R = _i64(dims), _i64(ranks)
    nbytes = lib().tt_orthogonalize_work_bytes(d, D, R, code)
    dev = cores[0].device
    with torch.cuda.device(dev), torch.cuda.stream(st):
        out = [torch.empty_like(g) for g in cores]
        work = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=dev)
        ptrs = (ctypes.c_void_p * d)(*[g.data_ptr() for g in cores])
        optrs = (ctypes.c_void_p * d)(*[g.data_ptr() for g in out])
        _check(lib().tt_orthogonalize(d, D, R, ptrs, code, {"left": 1, "right": 0}[side], optrs,
                                      ctypes.c_void_p(work.data_ptr()), st_ptr))
    return out


def tt_rse(A, cores, stream=None):
    """Streamed (||A - A_TT||_F^2, ||A||_F^2) in FP64, computed by the library
    (the TT is contracted slab by slab, never as a whole); the relative error
    of Sec. 4 is the square root of their ratio."""
    d, dims, ranks = _core_meta(cores)
    if list(A.shape) != dims:
        raise ValueError(f"A has shape {tuple(A.shape)}, the cores describe {tuple(dims)}")
    dtype = cores[0].dtype
    if A.dtype != dtype or not A.is_cuda:
        raise TypeError("A must be a device tensor of the cores' dtype")
    A = A.contiguous()
    cores = [g.contiguous() for g in cores]
    st, st_ptr = _stream(stream)
    code = TT_F64 if dtype == torch.float64 else TT_F32
    D, R = _i64(dims), _i64(ranks)
    nbytes = lib().tt_rse_work_bytes(d, D, R, code)
    dev = A.device
    with torch.cuda.device(dev), torch.cuda.stream(st):
        out = torch.empty(2, dtype=torch.float64, device=dev)
        work = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=dev)
        ptrs = (ctypes.c_void_p * d)(*[g.data_ptr() for g in cores])
        _check(lib().tt_rse(d, D, R, ptrs, code, ctypes.c_void_p(A.data_ptr()),
                            ctypes.c_void_p(work.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                            st_ptr))
        err2, norm2 = (float(x) for x in out.cpu())
    return err2, norm2


def _eval_operands(cores, idx, gout=None):
    """Validated contiguous operands of the masked evaluation: FP32 CUDA cores,
    int64 indices (and FP32 output gradients) on the cores' device.  The
    returned tensors must stay referenced until the library call has been
    enqueued (their device pointers are passed to it)."""
    if not cores:
        raise ValueError("no cores")
    dev = cores[0].device
    for g in cores:
        if not isinstance(g, torch.Tensor) or not g.is_cuda or g.dtype != torch.float32 \
                or g.dim() != 3 or g.device != dev:
            raise TypeError("cores must be float32 CUDA tensors of shape (r_{k-1}, I_k, r_k) "
                            "on one device")
    if not isinstance(idx, torch.Tensor) or idx.dtype != torch.int64 or not idx.is_cuda \
            or idx.device != dev:
        raise TypeError("idx must be an int64 CUDA tensor on the cores' device")
    cores_c = [g.contiguous() for g in cores]
    idx_c = idx.reshape(-1).contiguous()
    gout_c = None
    if gout is not None:
        if not isinstance(gout, torch.Tensor) or gout.dtype != torch.float32 or not gout.is_cuda \
                or gout.device != dev or gout.numel() != idx_c.numel():
            raise TypeError("gout must be a float32 CUDA tensor with one value per index, on the "
                            "cores' device")
        gout_c = gout.reshape(-1).contiguous()
    return dev, cores_c, idx_c, gout_c


def _check_cores(cores, dims, ranks):
    d = len(dims)
    if len(cores) != d:
        raise ValueError(f"expected {d} cores")
    for k, g in enumerate(cores):
        if tuple(g.shape) != (ranks[k], dims[k], ranks[k + 1]):
            raise ValueError(f"core {k} has shape {tuple(g.shape)}, the plan wants "
                             f"{(ranks[k], dims[k], ranks[k + 1])}")


class EvalPlan:
    """Plan of the masked evaluation for one index set (decoded indices, the
    entries ordered by each core's index, chunk flags), built once on the
    GPU and reused by every evaluation and gradient.  Its device block comes
    from torch's caching allocator and is released by close() or garbage
    collection.  An index outside [0, prod(dims)) raises TTError(TT_EINVAL)."""

    def __init__(self, dims, ranks, idx, stream=None):
        dims = [int(x) for x in dims]
        ranks = [int(x) for x in ranks]
        if not isinstance(idx, torch.Tensor) or idx.dtype != torch.int64 or not idx.is_cuda:
            raise TypeError("idx must be an int64 CUDA tensor")
        self.dims, self.ranks = dims, ranks
        self.device = idx.device
        self.shape = idx.shape
        idx_c = idx.reshape(-1).contiguous()
        self.n = idx_c.numel()
        self._alloc = _TorchAllocator(self.device)
        self._h = None
        st, st_ptr = _stream(stream)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device), torch.cuda.stream(st):
            _check(lib().tt_eval_plan_create(len(dims), _i64(dims), _i64(ranks),
                                             ctypes.c_void_p(idx_c.data_ptr()), self.n,
                                             self._alloc._alloc, self._alloc._free, None, st_ptr,
                                             ctypes.byref(h)))
        self._h = h

    @property
    def device_bytes(self):
        return int(lib().tt_eval_plan_device_bytes(self._h))

    def _cores(self, cores):
        _check_cores(cores, self.dims, self.ranks)
        for g in cores:
            if not g.is_cuda or g.dtype != torch.float32 or g.device != self.device:
                raise TypeError("cores must be float32 CUDA tensors on the plan's device")
        return [g.contiguous() for g in cores]

    def at(self, cores, stream=None):
        """x_e at the plan's indices (FP32, shaped like the plan's idx)."""
        cores_c = self._cores(cores)
        st, st_ptr = _stream(stream)
        with torch.cuda.device(self.device), torch.cuda.stream(st):
            out = torch.empty(self.n, dtype=torch.float32, device=self.device)
            ptrs = (ctypes.c_void_p * len(cores_c))(*[g.data_ptr() for g in cores_c])
            _check(lib().tt_eval_plan_at(self._h, ptrs, ctypes.c_void_p(out.data_ptr()), st_ptr))
        return out.view(self.shape)

    def _gout(self, gout):
        if not isinstance(gout, torch.Tensor) or gout.dtype != torch.float32 or not gout.is_cuda \
                or gout.device != self.device or gout.numel() != self.n:
            raise TypeError("gout must be a float32 CUDA tensor with one value per index")
        return gout.reshape(-1).contiguous()

    def _out(self, out, like):
        if out is None:
            return [torch.zeros_like(g) for g in like]
        _check_cores(out, self.dims, self.ranks)
        if any(not g.is_contiguous() or g.dtype != torch.float32 or g.device != self.device
               for g in out):
            raise TypeError("out must hold contiguous float32 tensors on the plan's device")
        return list(out)

    @staticmethod
    def _ptrs(ts):
        return (ctypes.c_void_p * len(ts))(*[g.data_ptr() for g in ts])

    def backward(self, cores, gout, stream=None, out=None, right=None):
        """Core gradients of sum_e gout_e x_e; accumulated into ``out`` (a list
        of tensors shaped like the cores) if given, else into fresh zeros.
        With ``right``, the interfaces right of each core come from those
        cores and the ones left of it from ``cores``.  Bitwise reproducible
        for this plan."""
        cores_c = self._cores(cores)
        right_c = cores_c if right is None else self._cores(right)
        gout_c = self._gout(gout)
        st, st_ptr = _stream(stream)
        with torch.cuda.device(self.device), torch.cuda.stream(st):
            grads = self._out(out, cores_c)
            if right is None:
                _check(lib().tt_eval_plan_backward(self._h, self._ptrs(cores_c),
                                                   ctypes.c_void_p(gout_c.data_ptr()),
                                                   self._ptrs(grads), st_ptr))
            else:
                _check(lib().tt_eval_plan_backward_mixed(self._h, self._ptrs(cores_c),
                                                         self._ptrs(right_c),
                                                         ctypes.c_void_p(gout_c.data_ptr()),
                                                         self._ptrs(grads), st_ptr))
        return grads

    def tangent_project(self, U, V, z, stream=None, out=None):
        """Increments dU_1..dU_d of the projection of P_Omega Z (z: its values
        on the plan's indices) onto the tangent space at the TT tensor whose
        left-orthogonal cores are U and right-orthogonal cores are V (see
        tt_tangent_project).  ``out`` (tensors shaped like the cores) is
        overwritten if given."""
        U_c, V_c = self._cores(U), self._cores(V)
        z_c = self._gout(z)
        st, st_ptr = _stream(stream)
        with torch.cuda.device(self.device), torch.cuda.stream(st):
            dU = [torch.empty_like(g) for g in U_c] if out is None else self._out(out, U_c)
            _check(lib().tt_tangent_project(self._h, self._ptrs(U_c), self._ptrs(V_c),
                                            ctypes.c_void_p(z_c.data_ptr()), self._ptrs(dU),
                                            st_ptr))
        return dU

    def tangent_eval(self, U, V, dU, stream=None):
        """P_Omega of the tangent vector sum_k U_<k dU_k V_>k at the plan's
        indices (see tt_tangent_eval), at the plan's own ranks."""
        U_c, V_c, dU_c = self._cores(U), self._cores(V), self._cores(dU)
        st, st_ptr = _stream(stream)
        with torch.cuda.device(self.device), torch.cuda.stream(st):
            out = torch.empty(self.n, dtype=torch.float32, device=self.device)
            _check(lib().tt_tangent_eval(self._h, self._ptrs(U_c), self._ptrs(V_c),
                                         self._ptrs(dU_c), ctypes.c_void_p(out.data_ptr()), st_ptr))
        return out.view(self.shape)

    def close(self, stream=None):
        if getattr(self, "_h", None) is not None:
            st, st_ptr = _stream(stream)
            with torch.cuda.device(self.device):
                lib().tt_eval_plan_destroy(self._h, st_ptr)
            self._h = None
            self._alloc.live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tt_eval_at(cores, idx, stream=None):
    """x_e = G_1[i_1] ... G_d[i_d] at int64 row-major linear indices (FP32).
    ``idx`` may be an EvalPlan.  An index outside [0, prod(dims)) raises
    TTError(TT_EINVAL) before any core memory is read for it."""
    if isinstance(idx, EvalPlan):
        return idx.at(cores, stream)
    d, dims, ranks = _core_meta(cores)
    dev, cores_c, idx_c, _ = _eval_operands(cores, idx)
    st, st_ptr = _stream(stream)
    with torch.cuda.device(dev), torch.cuda.stream(st):
        out = torch.empty(idx_c.numel(), dtype=torch.float32, device=dev)
        ptrs = (ctypes.c_void_p * d)(*[g.data_ptr() for g in cores_c])
        _check(lib().tt_eval_at(d, _i64(dims), _i64(ranks), ptrs, ctypes.c_void_p(idx_c.data_ptr()),
                                idx_c.numel(), ctypes.c_void_p(out.data_ptr()), st_ptr))
    return out.view(idx.shape)


def tt_eval_at_backward(cores, idx, gout, stream=None):
    """Core gradients of sum_e gout_e x_e (FP32), fresh zeroed buffers.
    ``idx`` may be an EvalPlan.  Deterministic: the same inputs give
    bitwise-equal gradients (no floating-point atomics)."""
    if isinstance(idx, EvalPlan):
        return idx.backward(cores, gout, stream)
    d, dims, ranks = _core_meta(cores)
    dev, cores_c, idx_c, gout_c = _eval_operands(cores, idx, gout)
    st, st_ptr = _stream(stream)
    with torch.cuda.device(dev), torch.cuda.stream(st):
        grads = [torch.zeros_like(g) for g in cores_c]
        ptrs = (ctypes.c_void_p * d)(*[g.data_ptr() for g in cores_c])
        gptrs = (ctypes.c_void_p * d)(*[g.data_ptr() for g in grads])
        _check(lib().tt_eval_at_backward(d, _i64(dims), _i64(ranks), ptrs,
                                         ctypes.c_void_p(idx_c.data_ptr()), idx_c.numel(),
                                         ctypes.c_void_p(gout_c.data_ptr()), gptrs, st_ptr))
    return grads


class TTEvalMasked(torch.autograd.Function):
    """Masked TT evaluation with the library's hand-written backward kernels.
    ``apply(idx, *cores)``: idx an int64 CUDA tensor or an EvalPlan (reused
    across calls, as in an optimisation loop)."""

    @staticmethod
    def forward(ctx, idx, *cores):
        if isinstance(idx, EvalPlan):
            ctx.plan = idx
            ctx.save_for_backward(*cores)
        else:
            ctx.plan = None
            ctx.save_for_backward(idx, *cores)
        return tt_eval_at(list(cores), idx)

    @staticmethod
    def backward(ctx, gout):
        saved = ctx.saved_tensors
        if ctx.plan is not None:
            idx, cores = ctx.plan, list(saved)
        else:
            idx, cores = saved[0], list(saved[1:])
        grads = tt_eval_at_backward(cores, idx, gout.to(torch.float32).contiguous())
        return (None, *grads)


def sketch_matrix(rows, cols, seed=0, step=0, dtype=torch.float32, device="cuda", stream=None):
    """The Rademacher sketch matrix Omega the sweep draws at step ``step``."""
    st, st_ptr = _stream(stream)
    out = torch.empty((rows, cols), dtype=dtype, device=device)
    code = TT_F64 if dtype == torch.float64 else TT_F32
    _check(lib().tt_sketch_matrix(rows, cols, seed, step, code, ctypes.c_void_p(out.data_ptr()),
                                  st_ptr))
    return out


def wait_selftest(arrive, limit_ns=50_000_000, stream=None):
    """Run the tensor-core kernels' bounded wait on a barrier that is (arrive)
    or is not completed; raises TTError(TT_ETIMEOUT) when the wait runs out."""
    st, st_ptr = _stream(stream)
    _check(lib().tt_wait_selftest(1 if arrive else 0, int(limit_ns), st_ptr))


def version():
    return lib().tt_version().decode()


def bounds_violations(reset=False):
    """(count, first source line) of the bounds-checked build's skipped
    out-of-range accesses since the last reset; count -1 from the normal build."""
    line = ctypes.c_int32(0)
    n = lib().tt_bounds_violations(ctypes.byref(line), 1 if reset else 0)
    return int(n), int(line.value)


def kernel_launches():
    """Kernels this library has launched in the process so far."""
    return int(lib().tt_kernel_launches())

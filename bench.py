#!/usr/bin/env python
"""Benchmark of the TT-UTV sweep on GB300.

Workload (default "c5"): a 128^4 FP32 tensor (1 GiB) built from Gaussian TT
cores of ranks (1,64,64,64,1) plus Gaussian noise at 1e-3 relative norm,
decomposed by TT-URV right-to-left (Alg. 3 with the prescribed-accuracy rule
of Sec. 3.1) at eps = 1e-2.  One step = one full sweep (all unfoldings, all
kernels, the per-step rank reads included).  Metric: tensor GB/s = bytes of
the input tensor / sweep time.  The default precision is mixed (tcgen05
tensor cores); a mixed run also times the same sweep in plain FP32 on the
same input and reports both, with each one's error against the FP64 oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp32|fp64]
    python bench.py --impl reference ...   # the FP64 CPU oracle on a bounded sample

Under torchrun (N > 1) every rank decomposes its own copy of the workload
(independent problems, no collective on the data path: weak scaling); rank 0
prints the JSON line with the whole-job throughput over the slowest rank.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "TT-UTV sweep tensor GB/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070 / 1e3  # 152 SMs x 128 FP32 lanes x FMA (2 flop) x 2.07 GHz

L2_BYTES = 129 * 10**6

WORKLOADS = {
    "c5": dict(dims=(128, 128, 128, 128), ranks=(1, 64, 64, 64, 1), rel_noise=1e-3, seed=0,
               eps=1e-2, variant="URV",
               desc="128^4 f32 tensor from Gaussian TT cores ranks (1,64,64,64,1) + 1e-3 relative "
                    "Gaussian noise, eps=1e-2, TT-URV right-to-left"),
    "c3": dict(dims=(32, 32, 32, 32, 32), ranks=(1, 20, 20, 20, 20, 1), rel_noise=1e-4, seed=0,
               eps=1e-3, variant="URV",
               desc="32^5 f32 tensor from Gaussian TT cores ranks (1,20,20,20,20,1) + 1e-4 relative "
                    "Gaussian noise, eps=1e-3, TT-URV right-to-left (precision study: every step "
                    "is tight)"),
    "c4": dict(kind="masked", ranks=(1, 32, 16, 1),
               desc="masked TT evaluation + core gradients of the completion workload: "
                    "256x256x64 f32 volume of 20 Gaussian blobs, Bernoulli(0.3) observation "
                    "set (1.26M entries), TT ranks (1,32,16,1) from the TT-URV initialisation"),
    "c4-rgrad": dict(kind="rgrad", ranks=(1, 32, 16, 1),
                     desc="Riemannian gradient completion (Sec. 4.2.2) of the 256x256x64 f32 "
                          "blob volume from its Bernoulli(0.3) observation set, TT ranks "
                          "(1,32,16,1): tangent projection, exact line-search step, fixed-rank "
                          "TT-URV retraction of the full 4.2M-entry iterate"),
    "mri-rgrad": dict(kind="rgrad", problem="mri", ranks=(1, 55, 41, 1),
                      desc="Riemannian gradient completion at the size and TT ranks of the "
                           "paper's MRI experiment (Sec. 4.2.2): a 181x217x181 f32 volume of "
                           "40 Gaussian blobs standing in for the MRI data, Bernoulli(0.3) "
                           "observation set, TT ranks (1,55,41,1), TT-URV retraction"),
    "c5-half": dict(dims=(64, 128, 128, 128), ranks=(1, 64, 64, 64, 1), rel_noise=1e-3, seed=0,
                    eps=1e-2, variant="URV",
                    desc="64x128^3 f32 (512 MiB) slab of the 128^4 workload's generator, for "
                         "profiler captures"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 200 sweeps of ~4 ms: a timed region long enough for the clock sampler
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp32", "mixed", "fp64"])
    ap.add_argument("--inner", default="qlp", choices=["qlp", "usvp", "lurv"],
                    help="small rank-revealing factor of each sweep step")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the plain-FP32 comparison timed beside a mixed-precision run")
    ap.add_argument("--workload", default="c5", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    return ap.parse_args()


def make_input(wl):
    return synth.gaussian_tt(wl["dims"], wl["ranks"], wl["rel_noise"], wl["seed"], np.float32)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, enabled=True):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        self.enabled = enabled

    def __enter__(self):
        if not self.enabled:
            return self
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------- roofline inputs

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path)), "measured"
        except ValueError:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def source_hash():
    """Hash of the sources of the kernel whose DRAM traffic profiles/ncu_traffic.json
    records (the tensor-core product); a change there invalidates the figure."""
    h = hashlib.sha256()
    for name in ("tc_gemm.cu", "tc_common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2501_07904_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key, workload):
    """DRAM bytes per launch from the committed ncu summary, if it still matches the source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except ValueError:
        return None
    if d.get("source_hash") != source_hash():
        return None
    ent = d.get("kernels", {}).get(f"{workload}:{kernel_key}")
    return None if ent is None else ent.get("traffic_bytes")


def phase_model(wl, res, precision="mixed"):
    """Algorithmic bytes and flops of the streaming products of every step of
    the right-to-left sweep, keyed (step, phase).  Step s factors unfolding
    C (m x n), m = I_1...I_{k-1}, n = I_k r_k, k = d - s: an exact step reads C
    for the Gram and again for the carry C Z (m x r); a sketched step (width
    l) reads C for Y = C^T Omega and again for B = C W (the project phase also
    forms B^T B)."""
    dims = wl["dims"]
    d = len(dims)
    out = {}
    for s in range(d - 1):
        k = d - s
        m = int(np.prod(dims[:k - 1]))
        n = dims[k - 1] * res.ranks[k]
        r = res.ranks[k - 1]
        l = res.sketch_l[k - 2]
        if l == 0:
            out[(s, "gram")] = dict(bytes=4.0 * m * n, flops=float(m) * n * (n + 1))
            if precision != "fp64" and res.small_fp64[k - 2]:
                # a tight step's Gram: compensated sums of exact products on
                # the FP32 pipes, 10 FP32 instructions per product (symmetric half)
                out[(s, "gram")]["fp32_instr"] = 10.0 * m * n * (n + 1) / 2
            out[(s, "carry")] = dict(bytes=4.0 * m * n + 4.0 * m * r, flops=2.0 * m * n * r)
        else:
            out[(s, "sketch")] = dict(bytes=4.0 * m * n + 4.0 * n * l, flops=2.0 * m * n * l)
            out[(s, "project")] = dict(bytes=4.0 * m * n + 8.0 * m * l, flops=2.0 * m * n * l + float(m) * l * (l + 1))
    return out


# --------------------------------------------------------------- our arm

def run_ours(args, wl, rank, world):
    import torch

    import paper_2501_07904_gb300 as tu

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    A_np = make_input(wl)
    nbytes = A_np.nbytes
    A_host = torch.from_numpy(A_np).pin_memory()
    A = A_host.to(dev)
    st = torch.cuda.current_stream()
    kw = dict(eps=wl["eps"], variant=wl["variant"], precision=args.precision, inner=args.inner)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        res = tu.tt_utv(A, **kw)
    torch.cuda.synchronize()
    ranks = res.ranks

    # timed region: K sweeps, device-resident input (larger than the 129 MB L2)
    phase_sum = None
    barrier()
    torch.cuda.synchronize()
    l0 = tu.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index, not args.no_clocks) as clk:
        t0 = time.perf_counter()
        ev0.record(st)
        for _ in range(args.steps):
            res = tu.tt_utv(A, timing=True, **kw)
            ph = res.info["phase_ms"]
            if phase_sum is None:
                phase_sum = [dict(p) for p in ph]
            else:
                for a, b in zip(phase_sum, ph):
                    for key in a:
                        a[key] += b[key]
        ev1.record(st)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    barrier()
    launches = tu.kernel_launches() - l0
    ms = slowest_ms(ev0.elapsed_time(ev1) / args.steps, world, dev)
    value = job_gbs(nbytes, world, ms)
    clocks = clk.summary()
    phases = [{k: v / args.steps for k, v in p.items()} for p in phase_sum]

    # roofline of the dominant streaming product (largest modeled phase time)
    model = phase_model(wl, res, args.precision)
    peaks, peak_src = measured_peaks()
    roof = None
    timed = [(sk, phases[sk[0]].get(sk[1], 0.0)) for sk in model]
    timed = [t for t in timed if t[1] > 0.0]
    if timed:
        (dom_step, dom_phase), dom_ms = max(timed, key=lambda t: t[1])
        mm = model[(dom_step, dom_phase)]
        gbs = mm["bytes"] / (dom_ms * 1e-3) / 1e9
        tfl = mm["flops"] / (dom_ms * 1e-3) / 1e12
        f_hbm = gbs / peaks["hbm_gbs"]
        if args.precision == "mixed":
            # TF32 tensor peak: the measured dense bf16 rate x the nominal TF32/BF16 ratio (1.1/2.25)
            c_peak = peaks["bf16_tflops"] * 0.5
            c_name = f"TF32 tensor: measured bf16 {peaks['bf16_tflops']} TFLOP/s x 0.5 (nominal ratio)"
            c_bound = "tensor"
        else:
            c_peak = FP32_PEAK_TFLOPS
            c_name = "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"
            c_bound = "alu"
        f_c = tfl / c_peak
        if "fp32_instr" in mm:
            # compensated Gram: bound by FP32 instruction issue, 152 SMs x 128
            # lanes x 2.07 GHz = 40.3 T lane-instructions/s
            c_peak = FP32_PEAK_TFLOPS / 2
            tfl = mm["fp32_instr"] / (dom_ms * 1e-3) / 1e12
            c_name = "FP32 issue: 152 SMs x 128 lanes x 2.07 GHz (lane-instructions)"
            c_bound = "alu"
            f_c = tfl / c_peak
        if f_c > f_hbm:
            roof = {"bound": c_bound, "achieved": round(tfl, 2), "peak": round(c_peak, 1),
                    "unit": "Tinstr/s" if "fp32_instr" in mm else "TFLOP/s",
                    "frac": round(f_c, 4), "peak_source": c_name,
                    "hbm_frac": round(f_hbm, 4), "hbm_gbs": round(gbs, 1)}
        else:
            roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": round(f_hbm, 4), "peak_source": peak_src,
                    "compute_frac": round(f_c, 4)}
        roof.update({"kernel": f"step{dom_step}:{dom_phase}", "ms": round(dom_ms, 4),
                     "algorithmic_bytes": mm["bytes"], "algorithmic_flops": mm["flops"],
                     "traffic": ncu_traffic(f"step{dom_step}:{dom_phase}:{args.precision}", args.workload)})

    # the whole sweep against HBM: algorithmic bytes of every streaming
    # product of the sweep (the schedule this build runs) over the sweep time
    sweep_bytes = sum(mm["bytes"] for mm in model.values())
    sweep_roof = {"scope": "whole sweep", "algorithmic_bytes": sweep_bytes,
                  "ms": round(ms, 4), "achieved": round(sweep_bytes / (ms * 1e-3) / 1e9, 1),
                  "peak": peaks["hbm_gbs"], "unit": "GB/s",
                  "frac": round(sweep_bytes / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                  "peak_source": peak_src,
                  "schedule": "every exact unfolding read twice (Gram, carry), every sketched "
                              "one twice (sketch, projection), each carry written once"}
    if roof is not None:
        roof["scope"] = f"dominant kernel ({roof['kernel']}); the whole sweep is sweep_roofline"

    # accuracy of this run (untimed): error equality, RSE, sampled diff vs the oracle
    acc = accuracy(tu, torch, A, res, args.workload)
    # the same sweep once more (untimed) with every non-tight step's error
    # summed directly from its residual: same ranks and cores, exact tails
    rd = tu.tt_utv(A, direct_tails=True, **kw)
    err2, normA2 = tu.tt_rse(A.to(rd.cores[0].dtype), rd.cores)
    acc["direct_tails"] = {
        "same_cores": bool(all(torch.equal(a, b) for a, b in zip(rd.cores, res.cores))),
        "tails_over_err2": sum(rd.tail_sq) / err2 if err2 > 0 else None,
        "tails_rel": [float(t) / normA2 for t in rd.tail_sq]}
    del rd

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        core_bytes = sum(c.numel() * c.element_size() for c in res.cores)
        outs = [torch.empty(c.shape, dtype=c.dtype, pin_memory=True) for c in res.cores]
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            r2 = tu.tt_utv(A_host, **kw)
            outs = [torch.empty(c.shape, dtype=c.dtype, pin_memory=True) for c in r2.cores] \
                if [tuple(c.shape) for c in r2.cores] != [tuple(o.shape) for o in outs] else outs
            for o, c in zip(outs, r2.cores):
                o.copy_(c, non_blocking=True)
        e1.record(st)
        torch.cuda.synchronize()
        ms_e2e = slowest_ms(e0.elapsed_time(e1) / args.steps, world, dev)
        # the host-to-device copy alone (pinned source, the same bytes)
        scratch = torch.empty_like(A)
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(st)
        for _ in range(args.steps):
            scratch.copy_(A_host, non_blocking=True)
        h1.record(st)
        torch.cuda.synchronize()
        ms_h2d = h0.elapsed_time(h1) / args.steps
        del scratch
        e2e = {"value": round(job_gbs(nbytes, world, ms_e2e), 2), "unit": "GB/s",
               "ms_per_step": round(ms_e2e, 4), "h2d_bytes_per_step": int(nbytes),
               "d2h_bytes_per_step": int(core_bytes),
               "h2d_ms": round(ms_h2d, 4), "h2d_gbs": round(nbytes / (ms_h2d * 1e-3) / 1e9, 1),
               "sweep_ms": round(ms, 4),
               "rest_ms": round(ms_e2e - ms_h2d - ms, 4),
               "breakdown": "e2e = H2D copy (pinned, one cudaMemcpyAsync) + the sweep on the "
                            "device copy + rest (core copies back, allocation of the device "
                            "input, host work)"}

    # the same sweep in plain FP32 on the same input, for the mixed vs FP32 comparison
    compare = None
    if args.precision == "mixed" and not args.no_compare:
        kw32 = dict(kw, precision="fp32")
        for _ in range(2):
            r32 = tu.tt_utv(A, **kw32)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(st)
        for _ in range(args.steps):
            r32 = tu.tt_utv(A, **kw32)
        c1.record(st)
        torch.cuda.synchronize()
        ms32 = slowest_ms(c0.elapsed_time(c1) / args.steps, world, dev)
        acc32 = accuracy(tu, torch, A, r32, args.workload)
        compare = {"precision": "fp32", "ms_per_step": round(ms32, 4),
                   "value": round(job_gbs(nbytes, world, ms32), 2), "unit": "GB/s",
                   "speedup_of_mixed": round(ms32 / ms, 3), "accuracy": acc32}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, inner=args.inner)

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "tf32x2/f32", "fp32": "f32", "fp64": "f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {wl['desc']}", "precision": args.precision,
                   "inner": args.inner, "l2": l2_note(wl),
                   "parallelism": f"replicas x{world} (independent problems)", "ranks": ranks,
                   "bytes_per_step": nbytes},
        "roofline": roof, "sweep_roofline": sweep_roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clocks, "accuracy": acc, "plain_fp32": compare,
        "phase_ms": [{k: round(v, 4) for k, v in p.items() if v > 0} for p in phases],
        "wall_s": round(wall, 3),
    }
    return out


def slowest_ms(ms, world, device):
    """Max over ranks of a per-rank time (ms): the job is as slow as its
    slowest replica."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_gbs(nbytes, world, ms):
    """Whole-job tensor GB/s: each of `world` replicas decomposes its own
    `nbytes` tensor, the slowest in `ms` milliseconds."""
    return world * nbytes / (ms * 1e-3) / 1e9


def l2_note(wl):
    """How the timed region relates to the 129 MB L2: input and first carry sizes."""
    n = 1
    for i in wl["dims"]:
        n *= i
    t = 4 * n
    carry = t // wl["dims"][-1 if wl["variant"] == "URV" else 0] * wl["ranks"][-2 if wl["variant"] == "URV" else 1]
    side = "larger" if t > L2_BYTES else "SMALLER"
    return (f"inputs {side} than L2: {t / 2**20:.0f} MiB tensor, first carry "
            f"{carry / 2**20:.0f} MiB, L2 {L2_BYTES / 1e6:.0f} MB")


def accuracy(tu, torch, A, res, workload):
    out = {"ranks": res.ranks}
    # ||A - A_TT||^2 and ||A||^2 streamed by the library (FP64 sums)
    err2, normA2 = tu.tt_rse(A.to(res.cores[0].dtype), res.cores)
    out["rse"] = (err2 / normA2) ** 0.5
    out["tails_over_err2"] = sum(res.tail_sq) / err2 if err2 > 0 else None
    gold = os.path.join(ROOT, "tests", "golden", f"{workload.split('-')[0]}_URV.npz")
    if workload in ("c5", "c3") and os.path.exists(gold):
        g = np.load(gold)
        vals = tu.tt_eval_at([c.float() for c in res.cores],
                             torch.from_numpy(g["sample_idx"]).to(A.device)).double().cpu().numpy()
        out["oracle_inner"] = "qlp"  # the stored expected values come from the pivoted-QLP oracle
        out["oracle_ranks"] = [int(x) for x in g["ranks"]]
        out["oracle_rse"] = float(g["rse"])
        # tails ||E_k||^2 / ||A||^2 per unfolding k = 1..d-1 beside the oracle's
        out["tails_rel"] = [float(t) / normA2 for t in res.tail_sq]
        out["oracle_tails_rel"] = [float(t) / float(g["normA2"]) for t in g["tails"]]
        out["rel_err_vs_oracle_sampled"] = float(
            np.sqrt(np.sum((vals - g["sample_val"]) ** 2) / np.sum(g["sample_ref"] ** 2)))
    return out


# -------------------------------------------------------- CPU oracle arms

def cpu_sample(wl, steps=1):
    """Bounded sample of the workload for the oracle: the first s slices of
    mode 1, about 0.9 s of oracle work per slice on a GB300 node's host cores.
    One sweep of the sample is about 10 s; for a timed loop of `steps` sweeps
    (the reference arm) the sample shrinks so the loop stays near 2.5 min."""
    dims = list(wl["dims"])
    s = max(1, min(12, int(150.0 / (0.9 * max(1, steps)))))
    return s, dims


def cpu_baseline(wl, repeats=1, inner="qlp"):
    from oracle import tt as otc  # the FP64 oracle: only this leg of bench.py runs it

    s, dims = cpu_sample(wl)
    A = make_input(wl)[:s].astype(np.float64)
    t0 = time.perf_counter()
    for _ in range(repeats):
        otc.tt_utv(A, eps=wl["eps"], variant=wl["variant"], inner=inner)
    dt = (time.perf_counter() - t0) / repeats
    nbytes = A.size * 4
    return {"value": round(nbytes / dt / 1e9, 4), "unit": "GB/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"first {s} of {dims[0]} mode-1 slices ({s}x{'x'.join(map(str, dims[1:]))} f32, "
                      f"{nbytes / 1e6:.0f} MB), same eps and sweep; {dt:.2f} s per sweep",
            "seconds": round(dt, 3)}


def run_reference(args, wl, rank, world):
    if rank != 0:
        return None
    s, dims = cpu_sample(wl, args.steps + min(args.warmup, 1))
    from oracle import tt as otc

    A = make_input(wl)[:s].astype(np.float64)
    nbytes = A.size * 4
    for _ in range(min(args.warmup, 1)):
        otc.tt_utv(A, eps=wl["eps"], variant=wl["variant"], inner=args.inner)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        otc.tt_utv(A, eps=wl["eps"], variant=wl["variant"], inner=args.inner)
    dt = (time.perf_counter() - t0) / args.steps
    value = nbytes / dt / 1e9
    sample = (f"first {s} of {dims[0]} mode-1 slices ({s}x{'x'.join(map(str, dims[1:]))} f32, "
              f"{nbytes / 1e6:.0f} MB), same eps and sweep")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}", "precision": "fp64 oracle",
                       "l2": "n/a (CPU)", "parallelism": "1 process, host cores"},
            "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ---------------------------------------------------- masked evaluation (c4)

MASKED_METRIC = "masked TT eval + gradient TFLOP/s"


def masked_flops_per_entry(ranks):
    """Algorithmic FLOPs of one entry of x = G_1[i_1]..G_d[i_d] and of its core
    gradients with the interfaces recomputed: forward sum_{k>=2} 2 r_{k-1} r_k
    (the first core is a copy); per core k, the left interface
    sum_{2<=j<k} 2 r_{j-1} r_j, the right one sum_{k<j<d} 2 r_{j-1} r_j (the
    last core is a copy), the gout scaling r_k and the outer product
    2 r_{k-1} r_k.  ranks = (r_0 = 1, ..., r_d = 1)."""
    d = len(ranks) - 1
    step = [2 * ranks[j] * ranks[j + 1] for j in range(d)]  # core j+1 (1-based) product
    fwd = sum(step[1:])
    bwd = 0
    for k in range(d):                       # core k+1 (1-based)
        left = sum(step[1:k])                # cores 2..k
        right = sum(step[k + 1:d - 1])       # cores k+2..d-1
        bwd += left + right + ranks[k + 1] + step[k]
    return fwd, bwd


def c4_problem(tu, torch, dev):
    cfg = synth.CONFIGS["c4"]
    shape, ranks = cfg["shape"], list(cfg["ranks"])
    M = synth.make_config("c4")
    idx = synth.observation_mask(shape, cfg["p_obs"], cfg["mask_seed"])
    vals = np.ascontiguousarray(M.reshape(-1)[idx])
    z = np.zeros(M.size, np.float32)
    z[idx] = vals / (len(idx) / M.size)
    cores = tu.tt_utv(torch.from_numpy(z.reshape(shape)).to(dev), ranks=ranks[1:-1]).cores
    return shape, ranks, idx, vals, cores


def run_c4(args, wl, rank, world):
    import torch

    import paper_2501_07904_gb300 as tu

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    shape, ranks, idx, vals, cores = c4_problem(tu, torch, dev)
    n = len(idx)
    i_t = torch.from_numpy(idx).to(dev)
    v_t = torch.from_numpy(vals).to(dev)
    plan = tu.EvalPlan(shape, ranks, i_t)
    st = torch.cuda.current_stream()
    gout = plan.at(cores) - v_t              # the residual of the initial cores
    grads = [torch.zeros_like(c) for c in cores]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > the 129 MB L2

    def step():
        x = plan.at(cores)
        for g in grads:
            g.zero_()
        plan.backward(cores, gout, out=grads)
        return x

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    l0 = tu.kernel_launches()
    with ClockSampler(dev.index, not args.no_clocks) as clk:
        for e0, e1 in ev:
            flush.fill_(1)                    # L2 flushed between timed steps
            e0.record(st)
            step()
            e1.record(st)
        torch.cuda.synchronize()
    barrier()
    launches = tu.kernel_launches() - l0
    ms = slowest_ms(sum(a.elapsed_time(b) for a, b in ev) / args.steps, world, dev)
    fwd_f, bwd_f = masked_flops_per_entry(ranks)
    flops = (fwd_f + bwd_f) * n
    value = world * flops / (ms * 1e-3) / 1e12

    # forward and backward apart (same flush discipline), for the roofline line
    def timed(fn, reps=20):
        tot = 0.0
        for _ in range(reps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            b.record(st)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / reps
    ms_f = timed(lambda: plan.at(cores))
    ms_b = timed(lambda: plan.backward(cores, gout, out=grads))
    roof = {"bound": "alu", "achieved": round(flops / (ms * 1e-3) / 1e12, 2),
            "peak": round(FP32_PEAK_TFLOPS, 1), "unit": "TFLOP/s",
            "frac": round(flops / (ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS, 4),
            "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz",
            "scope": "forward (1 launch) + backward (2d launches) of one step",
            "flops_per_entry": {"forward": fwd_f, "backward": bwd_f}, "entries": n,
            "forward": {"ms": round(ms_f, 4), "tflops": round(fwd_f * n / (ms_f * 1e-3) / 1e12, 2)},
            "backward": {"ms": round(ms_b, 4), "tflops": round(bwd_f * n / (ms_b * 1e-3) / 1e12, 2)},
            "traffic": None}

    # determinism and accuracy of this run (untimed)
    g1 = plan.backward(cores, gout)
    g2 = plan.backward(cores, gout)
    bitwise = all(torch.equal(a, b) for a, b in zip(g1, g2))
    from oracle import tt as otc  # accuracy check against the FP64 oracle (sampled, untimed)
    sub = np.random.default_rng(7).choice(n, 20000, replace=False)
    c64 = [c.double().cpu().numpy() for c in cores]
    xs = plan.at(cores).double().cpu().numpy()[sub]
    ref = otc.tt_eval_at(c64, idx[sub])
    acc = {"sampled_entries": len(sub),
           "max_rel_err_vs_oracle": float(np.max(np.abs(xs - ref)) / np.max(np.abs(ref))),
           "gradients_bitwise_reproducible": bool(bitwise)}

    # end to end through the public API with host buffers: cores in, gradients and loss out
    e2e = None
    if not args.no_e2e:
        h_cores = [c.cpu().pin_memory() for c in cores]
        h_grads = [torch.empty(c.shape, dtype=c.dtype, pin_memory=True) for c in cores]
        h_loss = torch.empty(1, dtype=torch.float32, pin_memory=True)
        d_cores = [torch.empty_like(c) for c in cores]
        in_bytes = sum(c.numel() * 4 for c in h_cores)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier()
        e0.record(st)
        for _ in range(args.steps):
            for dc, hc in zip(d_cores, h_cores):
                dc.copy_(hc, non_blocking=True)
            r = plan.at(d_cores) - v_t
            loss = 0.5 * torch.dot(r, r)
            gg = plan.backward(d_cores, r)
            for hg, g in zip(h_grads, gg):
                hg.copy_(g, non_blocking=True)
            h_loss.copy_(loss.view(1), non_blocking=True)
        e1.record(st)
        torch.cuda.synchronize()
        ms_e = slowest_ms(e0.elapsed_time(e1) / args.steps, world, dev)
        e2e = {"value": round(world * flops / (ms_e * 1e-3) / 1e12, 3), "unit": "TFLOP/s",
               "ms_per_step": round(ms_e, 4), "h2d_bytes_per_step": int(in_bytes),
               "d2h_bytes_per_step": int(in_bytes + 4),
               "step": "cores H2D, x = P_Omega(TT), residual and loss, gradients, gradients and loss D2H"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = c4_cpu_baseline(cores, idx, ranks)

    return {
        "metric": MASKED_METRIC, "value": round(value, 3), "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"c4: {wl['desc']}", "entries": n, "ranks": ranks,
                   "l2": "flushed between timed steps (256 MiB write): the plan and operands "
                         "(~80 MB) fit in the 129 MB L2",
                   "parallelism": f"replicas x{world} (independent problems)",
                   "entries_per_s": round(world * n / (ms * 1e-3), 1),
                   "plan_device_bytes": plan.device_bytes},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clk.summary(), "accuracy": acc,
    }


def c4_cpu_baseline(cores, idx, ranks, target_s=10.0, chunk=1 << 16):
    """The oracle's masked evaluation and gradient (FP64, numpy on the host
    cores) on successive blocks of the observation set for about target_s."""
    from oracle import tt as otc  # the FP64 oracle: only this leg of bench.py runs it

    c64 = [c.double().cpu().numpy() for c in cores]
    rng = np.random.default_rng(3)
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < target_s and done < len(idx):
        blk = idx[done:done + chunk]
        otc.tt_eval_at(c64, blk)
        otc.tt_eval_grad(c64, blk, rng.standard_normal(len(blk)))
        done += len(blk)
    dt = time.perf_counter() - t0
    f, b = masked_flops_per_entry(ranks)
    return {"value": round((f + b) * done / dt / 1e12, 6), "unit": "TFLOP/s",
            "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"first {done} of {len(idx)} observed entries in blocks of {chunk}, "
                      f"forward + gradient; {dt:.1f} s",
            "seconds": round(dt, 3)}


def run_reference_c4(args, wl, rank, world):
    if rank != 0:
        return None
    from oracle import tt as otc  # the FP64 oracle is this arm

    cfg = synth.CONFIGS["c4"]
    ranks = list(cfg["ranks"])
    shape = cfg["shape"]
    idx = synth.observation_mask(shape, cfg["p_obs"], cfg["mask_seed"])
    cores = synth.gaussian_cores(shape, ranks, seed=0)     # the oracle's cost does not depend on values
    budget = 150.0 / max(1, args.steps)                     # seconds per step: the loop stays near 2.5 min
    chunk = 1 << 14
    n = max(chunk, min(len(idx), int(budget * 3.5e4)) // chunk * chunk)  # ~3.5e4 entries/s
    rng = np.random.default_rng(3)
    gout = rng.standard_normal(n)

    def one():
        for s in range(0, n, chunk):
            otc.tt_eval_at(cores, idx[s:s + chunk])
            otc.tt_eval_grad(cores, idx[s:s + chunk], gout[s:s + chunk])
    for _ in range(min(args.warmup, 1)):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = (time.perf_counter() - t0) / args.steps
    f, b = masked_flops_per_entry(ranks)
    value = (f + b) * n / dt / 1e12
    sample = (f"first {n} of {len(idx)} observed entries in blocks of {chunk}, forward + gradient "
              f"(Gaussian cores of the workload's ranks)")
    return {"impl": "reference", "metric": MASKED_METRIC, "value": round(value, 6),
            "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"c4: {wl['desc']}", "precision": "fp64 oracle",
                       "l2": "n/a (CPU)", "parallelism": "1 process, host cores"},
            "cpu_baseline": {"value": round(value, 6), "unit": "TFLOP/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


RGRAD_METRIC = "RGrad completion iterations/s"


def rgrad_problem(name="c4"):
    cfg = synth.CONFIGS[name]
    shape = cfg["shape"]
    M = synth.make_config(name)
    idx = synth.observation_mask(shape, cfg["p_obs"], cfg["mask_seed"])
    return cfg, shape, M, idx, np.ascontiguousarray(M.reshape(-1)[idx])


def run_rgrad(args, wl, rank, world):
    """RGrad iterations of the completion workload.  Timed: args.steps
    iterations with the TT-URV retraction after args.warmup untimed ones, in
    one call (the iterate, its frames and the plans stay resident).  Also
    reported: the RSE / PSNR curves of the three retractions (the paper's
    comparison, Sec. 4.2.2) and their time per iteration."""
    import torch

    import paper_2501_07904_gb300 as tu
    from paper_2501_07904_gb300.completion import rgrad

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cfg, shape, M, idx, vals = rgrad_problem(wl.get("problem", "c4"))
    ranks = list(cfg["ranks"][1:-1])
    i_t = torch.from_numpy(idx).to(dev)
    v_t = torch.from_numpy(vals).to(dev)
    truth = torch.from_numpy(M).to(dev).double()
    held = torch.ones(M.size, dtype=torch.bool, device=dev)
    held[i_t] = False
    st = torch.cuda.current_stream()
    W, K = args.warmup, args.steps

    def run(method, keep):
        marks, iters = {}, []

        def cb(t, cores):
            if t in (W, W + K):
                e = torch.cuda.Event(enable_timing=True)
                e.record(st)
                marks[t] = (e, tu.kernel_launches())
            if keep:
                iters.append([c.clone() for c in cores])
        torch.cuda.synchronize()
        cores, losses, alphas = rgrad(v_t, i_t, shape, ranks, steps=W + K, retraction=method,
                                      callback=cb)
        torch.cuda.synchronize()
        ms = marks[W][0].elapsed_time(marks[W + K][0]) / K
        return cores, losses, alphas, ms, marks[W + K][1] - marks[W][1], iters

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    barrier()
    with ClockSampler(dev.index, not args.no_clocks) as clk:
        cores, losses, alphas, ms, launches, _ = run("URV", False)
    ms = slowest_ms(ms, world, dev)
    value = world * 1e3 / ms

    def metrics(cs):
        x = tu.tt_full(cs).double().reshape(-1)
        t = truth.reshape(-1)
        rse = float(torch.linalg.vector_norm(x - t) / torch.linalg.vector_norm(t))
        rse_u = float(torch.linalg.vector_norm((x - t)[held]) / torch.linalg.vector_norm(t[held]))
        psnr = 10.0 * np.log10(float(t.abs().max()) ** 2 / float(((x - t) ** 2).mean()))
        return round(rse, 5), round(rse_u, 5), round(psnr, 2)

    curves = {}
    show = sorted({0, 1, 2, 5, 10, 20, 40, W + K} & set(range(W + K + 1)))
    for method in ("URV", "ULV", "SVD"):
        _, ls, al, ms_m, _, iters = run(method, True)
        m = [metrics(c) for c in iters]
        curves[method] = {"ms_per_iter": round(ms_m, 3),
                          "iters": show,
                          "rse": [m[t][0] for t in show],
                          "rse_unobserved": [m[t][1] for t in show],
                          "psnr_db": [m[t][2] for t in show],
                          "loss": [float(f"{ls[t]:.5g}") for t in show]}

    e2e = None
    if not args.no_e2e:
        h_vals = torch.from_numpy(vals).pin_memory()
        h_idx = torch.from_numpy(idx).pin_memory()
        h_out = None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        dv, di = h_vals.to(dev, non_blocking=True), h_idx.to(dev, non_blocking=True)
        out, _, _ = rgrad(dv, di, shape, ranks, steps=K, retraction="URV")
        h_out = [c.to("cpu", non_blocking=True) for c in out]
        e1.record(st)
        torch.cuda.synchronize()
        ms_e = slowest_ms(e0.elapsed_time(e1) / K, world, dev)
        e2e = {"value": round(world * 1e3 / ms_e, 3), "unit": "iterations/s",
               "ms_per_step": round(ms_e, 3),
               "h2d_bytes_per_step": int((h_vals.numel() * 4 + h_idx.numel() * 8) / K),
               "d2h_bytes_per_step": int(sum(c.numel() * 4 for c in h_out) / K),
               "step": f"one rgrad() call of {K} iterations from host values and indices "
                       f"(plan builds and the spectral initialisation included), cores back to "
                       f"the host; per iteration"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = rgrad_cpu_baseline(shape, idx, vals, ranks)

    return {
        "metric": RGRAD_METRIC, "value": round(value, 3), "unit": "iterations/s", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": round(ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {wl['desc']}", "entries": len(idx), "ranks": ranks,
                   "l2": "inputs larger than L2 (the 4.2M-entry full iterate and its sweeps, "
                         "the 1.26M-entry plans)",
                   "parallelism": f"replicas x{world} (independent problems)"},
        "roofline": None, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "accuracy": {"loss_first_last": [losses[0], losses[-1]], "alphas_positive": all(a > 0 for a in alphas)},
        "curves": curves,
    }


def rgrad_iteration_oracle(shape, idx, vals, cores, ranks):
    """One oracle RGrad iteration from the given cores (FP64, host)."""
    from oracle import rgrad as org  # the FP64 oracle: only the baseline legs run it
    from oracle import tt as otc

    ntot = int(np.prod(shape))
    full = otc.tt_full(cores).reshape(-1)
    z = full[idx] - vals
    U, V = org.left_orthogonal(cores), org.right_orthogonal(cores)
    G = np.zeros(ntot)
    G[idx] = z
    dU = org.tangent_project(U, V, G.reshape(shape))
    xi = otc.tt_full(org.tangent_cores(U, V, dU)).reshape(-1)
    alpha = org.step_size(xi[idx], z)
    return org.retract((full - alpha * xi).reshape(shape), [1, *ranks, 1], "URV")


def rgrad_cpu_baseline(shape, idx, vals, ranks):
    cores = synth.gaussian_cores(shape, [1, *ranks, 1], seed=0)
    v64 = vals.astype(np.float64)
    t0 = time.perf_counter()
    rgrad_iteration_oracle(shape, idx, v64, cores, ranks)
    dt = time.perf_counter() - t0
    return {"value": round(1.0 / dt, 5), "unit": "iterations/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"one full RGrad iteration of the oracle (FP64, dense tangent projection, "
                      f"oracle TT-URV retraction) on the workload; {dt:.1f} s"}


def run_reference_rgrad(args, wl, rank, world):
    if rank != 0:
        return None
    cfg, shape, M, idx, vals = rgrad_problem(wl.get("problem", "c4"))
    ranks = list(cfg["ranks"][1:-1])
    cores = synth.gaussian_cores(shape, [1, *ranks, 1], seed=0)
    v64 = vals.astype(np.float64)
    steps = max(1, min(args.steps, 3))           # a bounded sample: a few iterations
    t0 = time.perf_counter()
    for _ in range(steps):
        cores = rgrad_iteration_oracle(shape, idx, v64, cores, ranks)
    dt = (time.perf_counter() - t0) / steps
    value = 1.0 / dt
    sample = f"{steps} oracle RGrad iterations (FP64, host) of the workload"
    return {"impl": "reference", "metric": RGRAD_METRIC, "value": round(value, 5),
            "unit": "iterations/s", "n_gpus": world, "steps": steps, "warmup": 0,
            "ms_per_step": round(dt * 1e3, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}", "precision": "fp64 oracle",
                       "l2": "n/a (CPU)", "parallelism": "1 process, host cores"},
            "cpu_baseline": {"value": round(value, 5), "unit": "iterations/s",
                             "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 5), "unit": "iterations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    kind = wl.get("kind", "sweep")
    if args.impl == "reference":
        fn = {"masked": run_reference_c4, "rgrad": run_reference_rgrad}.get(kind, run_reference)
    else:
        fn = {"masked": run_c4, "rgrad": run_rgrad}.get(kind, run_ours)
    out = fn(args, wl, rank, world)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

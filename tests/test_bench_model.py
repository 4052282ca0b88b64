"""Host-side figures of bench.py's roofline: the algorithmic bytes and flops
of each streaming product of the right-to-left sweep, and the peaks."""
import types

import pytest

import bench


def test_c5_phase_model():
    wl = bench.WORKLOADS["c5"]
    res = types.SimpleNamespace(ranks=[1, 64, 64, 64, 1], sketch_l=[128, 128, 0],
                                small_fp64=[0, 0, 0])
    m = bench.phase_model(wl, res, "mixed")
    # step 0 (k = 4, exact): C is 2^21 x 128, Gram = symmetric half, carry to rank 64
    assert m[(0, "gram")] == dict(bytes=4.0 * 2 ** 21 * 128, flops=2.0 ** 21 * 128 * 129)
    assert m[(0, "carry")]["bytes"] == 4.0 * 2 ** 21 * (128 + 64)
    assert m[(0, "carry")]["flops"] == 2.0 * 2 ** 21 * 128 * 64
    # step 1 (k = 3, sketched, l = 128): C is 2^14 x (128 * 64)
    assert m[(1, "sketch")]["bytes"] == 4.0 * 2 ** 14 * 8192 + 4.0 * 8192 * 128
    assert (2, "gram") not in m and (2, "sketch") in m
    assert not any("fp32_instr" in v for v in m.values())


def test_tight_gram_is_counted_in_fp32_instructions():
    wl = bench.WORKLOADS["c3"]
    res = types.SimpleNamespace(ranks=[1, 20, 20, 20, 20, 1], sketch_l=[32, 48, 48, 0],
                                small_fp64=[1, 1, 1, 1])
    g = bench.phase_model(wl, res, "fp32")[(0, "gram")]
    assert g["fp32_instr"] == 10.0 * 2 ** 20 * 32 * 33 / 2
    assert "fp32_instr" not in bench.phase_model(wl, res, "fp64")[(0, "gram")]


def test_peaks_and_l2_note():
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(80.55, rel=1e-3)
    assert bench.l2_note(bench.WORKLOADS["c5"]).startswith("inputs larger than L2: 1024 MiB")
    assert "first carry 512 MiB" in bench.l2_note(bench.WORKLOADS["c5"])

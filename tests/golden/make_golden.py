"""Write the oracle's expected values for the workloads too large to run the
oracle inside the GPU test session (c2, c3, c5).  Calls only ``oracle`` and
the seeded generators in ``synth``; run from the repository root:

    python tests/golden/make_golden.py [c2 c3 c5]

Outputs tests/golden/<cfg>_<method>.npz with ranks, per-unfolding tails,
||A||^2, RSE, the oracle's values at 4096 seeded sample indices and its cores
(c2, c3: FP64; c5: rounded once to FP32 to halve the file, 4.2 MB, which
moves the represented tensor by about 1e-7 of its norm).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import tt  # noqa: E402

OUT = os.path.dirname(os.path.abspath(__file__))
N_SAMPLES = 4096
SAMPLE_SEED = 12345


def save(name, A, res, keep_cores, core_dtype=np.float64):
    cfg = name.split("_")[0]
    dims = A.shape
    out = dict(ranks=np.array(res["ranks"]), tails=np.array(res["tails"]),
               normA2=res["normA2"], delta2=np.array(res["delta2"] or []),
               dims=np.array(dims), config=cfg)
    idx = synth.random_indices(dims, N_SAMPLES, SAMPLE_SEED)
    out["sample_idx"] = idx
    out["sample_val"] = tt.tt_eval_at(res["cores"], idx)
    out["sample_ref"] = np.asarray(A, dtype=np.float64).ravel()[idx]
    if keep_cores:
        out["rse"] = tt.rse(A, res["cores"])
        for k, g in enumerate(res["cores"]):
            out[f"core{k}"] = g
    else:
        # RSE from the error equality of Thm 3.1 / 3.2 (pinned in test_oracle_tt.py)
        out["rse"] = float(np.sqrt(sum(res["tails"]) / res["normA2"]))
        for k, g in enumerate(res["cores"]):
            out[f"core{k}"] = g.astype(core_dtype)
    np.savez_compressed(os.path.join(OUT, name + ".npz"), **out)
    print(name, res["ranks"], "rse", out["rse"], flush=True)


def main(which):
    if "c2" in which:
        A = synth.make_config("c2")
        for v in ("URV", "ULV"):
            t = time.time()
            save(f"c2_{v}", A, tt.tt_utv(A, eps=1e-6, variant=v), True)
            print("  ", round(time.time() - t, 1), "s")
        save("c2_SVD", A, tt.tt_svd(A, eps=1e-6, direction="LR"), True)
    if "c3" in which:
        A = synth.make_config("c3")
        for v in ("URV", "ULV"):
            t = time.time()
            save(f"c3_{v}", A, tt.tt_utv(A, eps=1e-3, variant=v), True)
            print("  ", round(time.time() - t, 1), "s")
    if "c5" in which:
        A = synth.make_config("c5")
        t = time.time()
        save("c5_URV", A, tt.tt_utv(A, eps=1e-2, variant="URV"), False, np.float32)
        print("  ", round(time.time() - t, 1), "s")


if __name__ == "__main__":
    main(sys.argv[1:] or ["c2", "c3", "c5"])

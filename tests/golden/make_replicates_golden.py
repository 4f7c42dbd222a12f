"""Writes tests/golden/replicates_240h.json from the FP64 oracle alone.

64 replicate runs of the paper's benchmark protocol BMII (5 x 2 Gy, one
fraction a day from t = 0; "Defining the search problem") over the paper's
whole horizon of ten days (240 h: five days of treatment, five of regrowth;
"The Main GA Loop"), each replicate growing its own seeded spheroid (radius 5
on a 32^3 lattice, large enough that the tumour never fills it; Philox key 0xB0B,
protocol word = replicate index).  The file keeps the 64 final live counts,
which the GPU test compares as a distribution with 64 GPU replicates drawn
under a different key, and the replicates' live counts at every whole day.

Nothing here calls the CUDA library; run it with
    python tests/golden/make_replicates_golden.py
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from synth import workloads  # noqa: E402
from synth.params import P0  # noqa: E402

N, L, R, HOURS, KEY = 64, 32, 5, 240, 0xB0B
OUT = os.path.join(HERE, "replicates_240h.json")


def main():
    doses, waits = workloads.benchmark_bmii()
    off = np.arange(N + 1, dtype=np.int32) * len(doses)
    d = np.tile(np.array(doses, dtype=np.float64), N)
    w = np.tile(np.array(waits, dtype=np.float64), N)
    t0 = time.time()
    ref = oracle.run_batch(P0, [L] * N, [R] * N, KEY, off, d, w, t_end_steps=HOURS * 600, init_word=0xFFFFFFFE,
                           hours=HOURS)
    dt = time.time() - t0
    out = {"what": "FP64 oracle, 64 replicates of BMII (5 x 2 Gy daily from t = 0) over 240 h, 32^3 lattice, "
                   "seeded spheroid R = 5 per replicate (init word = replicate index), parameter set P0, key 0xB0B",
           "written_by": "tests/golden/make_replicates_golden.py (calls oracle/ only)",
           "oracle_seconds": round(dt, 1), "n": N, "L": L, "R": R, "hours": HOURS, "key": KEY,
           "doses": doses, "waits": waits, "n_final": [int(x) for x in ref["n_final"]],
           "daily_counts": ref["counts"][:, ::24].tolist()}
    with open(OUT, "w") as f:
        json.dump(out, f)
        f.write("\n")
    print(f"wrote {OUT}: mean {np.mean(ref['n_final']):.1f}, sd {np.std(ref['n_final']):.1f}, {dt:.0f} s")


if __name__ == "__main__":
    main()

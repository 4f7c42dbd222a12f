"""Writes tests/golden/single_protocol_288h.json from the FP64 oracle alone.

The single-protocol workload: a 40^3 lattice, the seeded spheroid of radius 5
(515 cells), 10 x 2 Gy at 24 h intervals from t = 0, a fixed 288 h horizon
(172,800 steps at 600 steps per hour, "GA Resolution, constraints"), the
build's parameter set P0.  The oracle runs the whole horizon once (about seven
minutes on one host core) and the file keeps what a GPU run is compared with:
all 289 hourly live counts, the decision statistics (how many threshold
decisions were taken and how many of them fell inside the near-threshold
band), a SHA-256 of the final cell words, and the final fields on the central
plane z = 20 together with their whole-lattice sums.

Nothing here calls the CUDA library; run it with
    python tests/golden/make_single_protocol_golden.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synth import workloads  # noqa: E402
from synth.params import P0  # noqa: E402

SEED = 0x00C0_FFEE_0000_0042  # the seed of the GPU parity tests
L, R, HOURS = 40, 5, 288
OUT = os.path.join(HERE, "single_protocol_288h.json")


def main():
    doses, waits = workloads.daily_fractions(10, 2.0, 24.0)
    t0 = time.time()
    ref = oracle.run(P0, L, R, SEED, 0, doses, waits, t_end_steps=HOURS * 600, hours=HOURS)
    dt = time.time() - t0
    st = ref["state"]
    zc = L // 2
    plane = slice(zc * L * L, (zc + 1) * L * L)
    out = {
        "what": "FP64 oracle, single protocol: 40^3, R = 5, 10 x 2 Gy daily from t = 0, 288 h fixed horizon, "
                "parameter set P0, seed 0x00C0FFEE00000042, protocol word 0",
        "written_by": "tests/golden/make_single_protocol_golden.py (calls oracle/ only)",
        "oracle_seconds": round(dt, 1),
        "L": L, "R": R, "hours": HOURS, "seed": SEED, "doses": doses, "waits": waits,
        "counts": [int(c) for c in ref["counts"]],
        "stats": ref["stats"],
        "cum_dose": ref["cum_dose"],
        "final_cells_sha256": hashlib.sha256(st.cell.astype("<u4").tobytes()).hexdigest(),
        "final_kind_histogram": np.bincount(st.cell & 7, minlength=6).tolist(),
        "field_sums": [float(np.sum(st.O)), float(np.sum(st.G)), float(np.sum(st.H))],
        "central_plane_z": zc,
        "central_plane": {"O": st.O[plane].tolist(), "G": st.G[plane].tolist(), "H": st.H[plane].tolist()},
    }
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")
    print(f"wrote {OUT}: n_live {ref['stats']['n_live']}, decisions {ref['stats']['n_decisions']}, "
          f"near {ref['stats']['n_near']}, {dt:.0f} s")


if __name__ == "__main__":
    main()

"""Error of BF16 / FP16 field storage (FP32 arithmetic) against the FP64 oracle.

64 seeded protocols of the GA-batch generator on 64^3 lattices (spheroid R = 8),
first wait shortened to 30 min so a fraction falls inside the window; every
protocol runs 3,600 steps (6 simulated hours) on the GPU in FP32, BF16 and
FP16 storage and on the oracle (host threads).  Prints one JSON line per
precision: maximum and median field error relative to the medium value, final
live-count errors, and the device mass sums (FP64 and Kahan FP32).

    python tests/precision_report.py [n_protocols] [steps]
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2303_08123_b300 import Simulator, csr  # noqa: E402
from synth import workloads  # noqa: E402
from synth.params import P0  # noqa: E402


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 64
    T = int(sys.argv[2]) if len(sys.argv) > 2 else 3600
    L, R, seed = 64, 8, 0x5EED_0004
    prot = workloads.ga_batch(n, seed=4)
    prot = [(d, [0.5] + w[1:]) for d, w in prot]
    off, d, w = csr(prot)
    ref = oracle.run_batch(P0, [L] * n, [R] * n, seed, off, d, w, t_end_steps=T)
    # fields of a few protocols for the field error (the oracle's batch runner keeps counts only)
    sample = list(range(0, n, max(1, n // 8)))
    ref_state = {p: oracle.run(P0, L, R, seed, p, prot[p][0], prot[p][1], t_end_steps=T)["state"] for p in sample}
    med = np.array([P0.medium_O, P0.medium_G, 10 ** (3 - P0.medium_pH)])
    for precision in ("fp32", "bf16", "fp16"):
        sim = Simulator([L] * n, [R] * n, seed=seed, precision=precision, t_end_steps=T, dose_cap_gy=20.0)
        sim.load_protocols(off, d, w)
        sim.run(0)
        cnt, _ = sim.fitness()
        t64, t32 = sim.field_totals()
        ferr = []
        for p in sample:
            O, G, H, _ = sim.get_state(p)
            st = ref_state[p]
            ferr.append([float(np.max(np.abs(a.astype(np.float64) - b))) / m
                         for a, b, m in zip((O, G, H), (st.O, st.G, st.H), med)])
        ferr = np.array(ferr)
        cerr = np.abs(cnt.astype(np.float64) - ref["n_final"]) / ref["n_final"]
        kahan = float(np.max(np.abs(t32.astype(np.float64) - t64) / np.abs(t64)))
        print(json.dumps({
            "precision": precision, "protocols": n, "steps": T, "lattice": L,
            "field_err_max_rel_medium": {k: float(ferr[:, i].max()) for i, k in enumerate("OGH")},
            "field_err_median_rel_medium": {k: float(np.median(ferr[:, i])) for i, k in enumerate("OGH")},
            "count_err_max": float(cerr.max()), "count_err_mean": float(cerr.mean()),
            "count_exact_fraction": float(np.mean(cnt == ref["n_final"])),
            "kahan_fp32_vs_fp64_total_max_rel": kahan}), flush=True)
        sim.close()


if __name__ == "__main__":
    main()

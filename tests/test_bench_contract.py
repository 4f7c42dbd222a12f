"""The benchmark's reference arm (the FP64 oracle on the host cores) runs
without a GPU and prints one JSON line with the keys the benchmark contract
names."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600, check=True)
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["ms_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_fused_pass_plan_matches_the_tile_shapes():
    """The bench's count of fused passes per CA step (its gpu_launches and
    roofline labels): passes of two substeps, of four on the deep TMA shapes 7
    and 8, the last pass shorter by the remainder."""
    import importlib
    import sys as _sys
    _sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    from synth.params import P0, P_PHYS
    saved = bench.PARAMS
    try:
        bench.PARAMS = P0  # n_sub = 4
        assert [bench.fused_passes(s) for s in (3, 5, 6)] == [(2, 2)] * 3
        assert [bench.fused_passes(s) for s in (7, 8)] == [(1, 4)] * 2
        bench.PARAMS = P_PHYS  # 128 substeps per step
        assert bench.fused_passes(6) == (64, 2) and bench.fused_passes(7) == (32, 4)
        bench.PARAMS = P0.replace(n_sub=6)
        assert bench.fused_passes(6) == (3, 2) and bench.fused_passes(8) == (2, 4)
    finally:
        bench.PARAMS = saved

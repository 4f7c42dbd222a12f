"""The host GA loop over the batched simulator (GPU): generations run, every
protocol stays valid, and the per-generation JSONL log holds what it says."""
import io
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_run_ga_logs_every_generation():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_08123_b300 import _build, ga, screen
    _build.build()
    setup = screen.SimSetup(L=16, R=3, regrowth_h=2)
    cfg = ga.GAConfig(n_slots=24, d_max=2.5, total_cap=8.0, min_gap=4, population=16,
                      mutations=("swap", "split", "dose_time", "dose_value"), p_mut=0.5)
    log = io.StringIO()
    hist = screen.run_ga(setup, cfg, 2, np.random.default_rng(3), log=log)
    lines = [json.loads(l) for l in log.getvalue().splitlines()]
    assert [l["generation"] for l in lines] == [0, 1, 2] and len(hist) == 3
    for l, (best, used) in zip(lines, hist):
        assert l["best_count"] == best and l["simulations"] == used and l["mean_count"] >= best
        d, w = l["best_protocol"]["dose_gy"], l["best_protocol"]["wait_h"]
        assert ga.is_valid(ga.from_pairs(d, w, cfg.n_slots), cfg)

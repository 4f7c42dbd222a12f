"""Throughput benchmark: GA protocols evaluated per second on one B300.

Default workload (per GPU): the ragged hypofractionated batch, 1,024 protocols
whose spheroid radius is uniform in 4-20 sites on lattices of side
16 ceil(5R/16) (32^3 to 112^3); 5-15 fractions per protocol with doses from
{1, ..., 5} Gy and waits from {6, ..., 60} h, total dose capped at 30 Gy; FP32
fields; horizon = last fraction + 120 h.  A bench step is one simulated hour
(600 CA steps) of the whole batch, all hot-path kernels included (irradiation,
reaction-diffusion, cell update, division, hourly counts).  The batch is first
advanced, untimed, to --start-hour (the last W of those hours are the warm-up),
so the timed window does not sit on the cheap hours right after seeding.
protocols/s = protocol-steps per second of the window divided by the batch's
mean horizon in steps (an extrapolation, labelled so in the line).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload ragged|ga_batch|single] [--start-hour H]

N > 1 runs under torchrun, one batch per rank (weak scaling, no collective on
the data path).  `--impl reference` times the FP64 CPU oracle on this host's
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
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

from synth import workloads  # noqa: E402
from synth.params import P0, P_PHYS  # noqa: E402

N_PROT, L, R = 256, 64, 8
SEED = 0x5EED_2023
METRIC = "GA protocols evaluated/sec"
UNIT = "protocols/s"
STEPS_PER_HOUR = 600


WORKLOAD = "ragged"
PARAMS, PARAMS_NOTE = P0, ""
START_HOUR = 24
CPU_SAMPLE_STEPS = {"ragged": 100, "single": 6000}  # oracle steps per protocol of one CPU sample


def t_end_steps():
    """Fixed horizon of the workload in steps (0: last fraction + 120 h per protocol)."""
    return 288 * STEPS_PER_HOUR if WORKLOAD == "single" else 0


def workload():
    """(protocols, mean horizon in h, lattice sides, radii) of the benchmarked batch."""
    if WORKLOAD == "single":
        prot = [workloads.daily_fractions(10, 2.0, 24.0)]
        return prot, 288.0, np.array([40], dtype=np.int32), np.array([5], dtype=np.int32)
    rank = int(os.environ.get("RANK", "0"))  # under torchrun every rank evaluates its own protocols
    if WORKLOAD == "ragged":
        Ls, Rs, prot = workloads.ragged_batch(N_PROT, seed=3 + 1000 * rank)
    else:
        prot = workloads.ga_batch(N_PROT, seed=2 + 1000 * rank)
        Ls, Rs = np.full(N_PROT, L, dtype=np.int32), np.full(N_PROT, R, dtype=np.int32)
    t_end_h = [sum(w) + 120.0 for _, w in prot]
    return prot, float(np.mean(t_end_h)), Ls, Rs


def workload_config(mean_t_end_h, precision="fp32"):
    if WORKLOAD == "single":
        return {
            "workload": "single protocol, 40^3 lattice, seeded spheroid R=5 (515 cells), 10 x 2 Gy at 24 h "
                        f"intervals, fixed 288 h horizon (12 days), {precision} fields, n_sub={PARAMS.n_sub}"
                        + PARAMS_NOTE,
            "step": "one simulated hour (600 CA steps)",
            "protocols_per_s": "1 / (seconds per simulated hour x 288 h)",
            "mean_horizon_h": 288.0,
            "l2": "L2-resident (fields 1.5 MB): latency-bound; the HBM fraction is a reference, not a DRAM figure",
            "parallelism": "one protocol",
        }
    if WORKLOAD == "ragged":
        _, _, Ls, _ = workload()
        return {
            "workload": f"ragged batch {N_PROT} protocols, spheroid radius uniform 4-20, lattice 16*ceil(5R/16) "
                        f"(32^3-112^3, mean {float(np.mean(Ls.astype(np.float64) ** 3)):.0f} sites), "
                        "5-15 fractions of {1..5} Gy, waits {6..60} h, cap 30 Gy, "
                        f"{precision} fields, n_sub={PARAMS.n_sub}" + PARAMS_NOTE,
            "step": "one simulated hour (600 CA steps) of the whole batch",
            "timed_window": f"hours {START_HOUR}..{START_HOUR}+K after the seeded start (advanced untimed first)",
            "protocols_per_s": "protocol-steps/s of the timed window divided by the mean horizon (last fraction "
                               "+ 120 h): extrapolated from that window",
            "mean_horizon_h": round(mean_t_end_h, 2),
            "l2": "working set > 126 MB L2: no flush needed",
            "parallelism": "independent protocol batch per GPU, persistent tile scheduling",
        }
    return {
        "workload": f"ga_batch {N_PROT} protocols x {L}^3 lattice, seeded spheroid R={R} (2109 cells), "
                    "10 fractions/protocol, doses {0.5..2.5} Gy, waits {6..60} h, cap 20 Gy, "
                    f"{precision} fields, n_sub={PARAMS.n_sub}" + PARAMS_NOTE,
        "step": "one simulated hour (600 CA steps) of the whole batch",
        "timed_window": f"hours {START_HOUR}..{START_HOUR}+K after the seeded start (advanced untimed first)",
        "protocols_per_s": "protocol-steps/s of the timed window divided by the mean horizon (last fraction + "
                           "120 h): extrapolated from that window; --full-run times the whole batch",
        "mean_horizon_h": round(mean_t_end_h, 2),
        "l2": "working set > 126 MB L2 (fields alone 805 MB at 256 protocols): no flush needed",
        "parallelism": "independent protocol batch per GPU",
    }


# --------------------------------------------------------------------------- helpers
def _csr(protocols):
    off, d, w = [0], [], []
    for dd, ww in protocols:
        d.extend(dd)
        w.extend(ww)
        off.append(len(d))
    return np.array(off, dtype=np.int32), np.array(d, dtype=np.float64), np.array(w, dtype=np.float64)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=10)

    def summary(self):
        self.file.flush()
        self.file.seek(0)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.file.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def fused_passes(shape):
    """Fused passes per CA step on a tile shape: passes of four substeps on the
    deep TMA shapes (7, 8), of two elsewhere (the last one shorter)."""
    depth = 4 if shape in (7, 8) else 2
    return (PARAMS.n_sub + depth - 1) // depth, depth


def traffic_for(kernel, n_sites):
    """DRAM bytes per launch from the committed ncu capture (64 protocols of
    64^3; bytes per site scaled to the batch's sites), or None when a kernel
    source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)[kernel]
        d["sources"]
    except Exception:
        return None
    return d["dram_bytes_per_site"] * n_sites if sources_sha(d["sources"]) == d["source_sha"] else None


def sources_sha(names):
    """Hash of the kernel sources a committed counter capture was taken with."""
    h = hashlib.sha256()
    for n in names:
        h.update(open(os.path.join(ROOT, "paper_2303_08123_b300", "csrc", n), "rb").read())
    return h.hexdigest()[:16]


def cpu_baseline(mean_t_end_h, max_steps=None):
    """The FP64 oracle on this host's cores: one protocol per core, a bounded
    number of steps each; extrapolated to whole protocols by the mean horizon."""
    import oracle
    cores = os.cpu_count() or 1
    prot, _, Ls, Rs = workload()
    n = min(cores, N_PROT)
    steps = max_steps or CPU_SAMPLE_STEPS.get(WORKLOAD, 1200)
    off, d, w = _csr(prot[:n])
    t0 = time.perf_counter()
    res = oracle.run_batch(PARAMS, Ls[:n], Rs[:n], SEED, off, d, w, max_steps=steps, n_threads=n)
    dt = time.perf_counter() - t0
    site_steps = float(np.sum(res["steps"] * Ls[:n].astype(np.float64) ** 3))
    per_protocol = mean_t_end_h * STEPS_PER_HOUR * float(np.mean(Ls.astype(np.float64) ** 3))
    return {"value": site_steps / dt / per_protocol, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{n} protocols x {steps} steps of the benchmarked workload on {n} threads "
                      f"({dt:.1f} s); extrapolated by the {mean_t_end_h:.1f} h mean horizon",
            "site_steps_per_s": site_steps / dt}


def precision_error(precision, n, steps):
    """Oracle leg of a 2-byte-storage run, outside every timed region: n seeded
    protocols of the GA-batch generator on 64^3 (R = 8, first wait 30 min so a
    fraction falls inside the window) run `steps` steps on the GPU with this
    storage and on the FP64 oracle (host threads).  Maximum field error
    relative to the medium value, and live-count errors."""
    import oracle
    from paper_2303_08123_b300 import Simulator, csr
    Lq, Rq, seed = 64, 8, 0x5EED_0004
    prot = [(dd, [0.5] + ww[1:]) for dd, ww in workloads.ga_batch(n, seed=4)]
    off, d, w = csr(prot)
    from concurrent.futures import ThreadPoolExecutor
    ref = oracle.run_batch(PARAMS, [Lq] * n, [Rq] * n, seed, off, d, w, t_end_steps=steps)
    sample = list(range(0, n, max(1, n // 4)))
    with ThreadPoolExecutor(len(sample)) as ex:  # the oracle's ctypes calls release the GIL
        futs = {p: ex.submit(oracle.run, PARAMS, Lq, Rq, seed, p, prot[p][0], prot[p][1], t_end_steps=steps)
                for p in sample}
        ref_state = {p: f.result()["state"] for p, f in futs.items()}
    med = np.array([PARAMS.medium_O, PARAMS.medium_G, 10 ** (3 - PARAMS.medium_pH)])
    sim = Simulator([Lq] * n, [Rq] * n, seed=seed, precision=precision, t_end_steps=steps, dose_cap_gy=20.0,
                    params=PARAMS)
    sim.load_protocols(off, d, w)
    sim.run(0)
    cnt, _ = sim.fitness()
    ferr = np.zeros(3)
    for p in sample:
        st = ref_state[p]
        got = sim.get_state(p)[:3]
        ferr = np.maximum(ferr, [float(np.max(np.abs(a.astype(np.float64) - b))) / m
                                 for a, b, m in zip(got, (st.O, st.G, st.H), med)])
    sim.close()
    cerr = np.abs(cnt.astype(np.float64) - ref["n_final"]) / np.maximum(1, ref["n_final"])
    return {"sample": f"{n} GA-batch protocols on 64^3 (R=8), {steps} steps from the seeded start, oracle FP64; "
                      f"fields compared on {len(sample)} of them",
            "field_err_max_rel_medium": {k: float(v) for k, v in zip("OGH", ferr)},
            "count_err_max_rel": float(cerr.max()), "count_exact_fraction": float(np.mean(cnt == ref["n_final"]))}


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    prot, mean_h, _, _ = workload()
    vals = []
    # each step: the same bounded oracle sample as the cpu_baseline of our arm's line
    for _ in range(args.warmup):
        cpu_baseline(mean_h, max_steps=20)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(mean_h))
    ms_per_step = (time.perf_counter() - t0) * 1e3 / max(1, args.steps)
    v = statistics.mean(x["value"] for x in vals)
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(mean_h), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2303_08123_b300 import Simulator, csr

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prot, mean_h, Ls, Rs = workload()
    off, d, w = csr(prot)
    K, W = args.steps, args.warmup
    start_h = max(START_HOUR, W)  # the timed window opens at this hour; the last W hours before it are warm-up
    hours = start_h + K + 2

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sim = Simulator(Ls, Rs, seed=SEED, precision=args.precision, hours=hours, params=PARAMS,
                    dose_cap_gy=30.0, device=dev, path=args.path, tile_shape=args.tile_shape, z_chunk=args.z_chunk,
                    t_end_steps=t_end_steps())
    sim.load_protocols(off, d, w)
    if args.path == "fused" and args.tile_shape == 0:
        shape, shape_ms = sim.autotune(10)  # re-seeds the batch at step 0
    else:
        shape, shape_ms = args.tile_shape, None
    stream = torch.cuda.current_stream(dev)
    if args.full_run:
        return full_run(args, sim, prot, mean_h, Ls, shape, shape_ms, world, rank, dev, barrier)
    if start_h > W:  # untimed advance to the warm-up hours (sim.run(0) would run to every horizon)
        sim.run(STEPS_PER_HOUR * (start_h - W))
    for _ in range(W):
        sim.run(STEPS_PER_HOUR)
    barrier()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        start.record(stream)
        for _ in range(K):
            sim.run(STEPS_PER_HOUR)
        stop.record(stream)
        barrier()
    ms = start.elapsed_time(stop)
    t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    ms_per_step = ms / K
    sites = float(np.sum(Ls.astype(np.float64) ** 3))
    protocol_steps_per_s = world * N_PROT * STEPS_PER_HOUR * K / (ms / 1e3)
    value = protocol_steps_per_s / (mean_h * STEPS_PER_HOUR)
    site_steps_per_s = world * sites * STEPS_PER_HOUR * K / (ms / 1e3)
    per_ca_step = (fused_passes(shape)[0] + 2) if args.path == "fused" else (PARAMS.n_sub + 3)
    launches_per_step = STEPS_PER_HOUR * per_ca_step + 2  # passes (or substeps + cell), claim, resolve; tick, count

    # per-kernel device time over plain steps of the same batch (CUDA events on the launching stream)
    kms, kl = sim.profile_steps(60)
    interior = float(np.sum((Ls.astype(np.float64) - 2) ** 3))
    es = 4 if args.precision == "fp32" else 2
    if args.path == "fused":
        kn = ("k_tma" if shape in (5, 6, 7, 8) else
              ("k_fused1" if args.precision == "fp32" else "k_fused1h") if shape in (3, 4) else "k_fused")
        n_pass, depth = fused_passes(shape)
        k_last = PARAMS.n_sub - depth * (n_pass - 1)
        if n_pass == 1:
            last = f"{kn} (one pass per step: irradiation + {k_last} substeps + cell update)"
            classes = {last: (kms[1], kl[1], interior * (6 * es + 8))}
            traffic_key = {last: f"{kn}_last_shape{shape}"}
        else:
            first = f"{kn} (first pass: irradiation + {depth} substeps)" if n_pass == 2 else \
                f"{kn} (passes before the last: {depth} substeps each, irradiation in the first)"
            last = f"{kn} (last pass: {k_last} substeps + cell update)"
            classes = {first: (kms[0], kl[0], interior * (6 * es + 4)),
                       last: (kms[1], kl[1], interior * (6 * es + 8))}
            traffic_key = {first: f"{kn}_first_shape{shape}", last: f"{kn}_last_shape{shape}"}
    else:
        classes = {"k_substep": (kms[0], kl[0], interior * (6 * es + 4)),
                   "k_cell": (kms[1], kl[1], interior * (3 * es + 8))}
        traffic_key = {"k_substep": "k_substep", "k_cell": "k_cell"}
    name = max(classes, key=lambda k: classes[k][0])
    k_ms, k_n, alg_bytes = classes[name]
    avg_ms = k_ms / k_n
    hbm, peak_kind = peaks()
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "peak_kind": f"{peak_kind} copy bandwidth",
            "traffic": traffic_for(traffic_key[name], sites),
            "traffic_source": "ncu capture on 64 x 64^3 (profiles/traffic.json), scaled by sites",
            "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_ms,
            "kernel_share": {k: float(v / kms.sum()) for k, v in
                             zip(("reaction-diffusion", "cell-update pass", "claim", "resolve"), kms)}}
    step_bytes = 32 if args.precision == "fp32" else 20
    roof_step = {"fused_alg_bytes_per_site_step": step_bytes,
                 "achieved_GBps": site_steps_per_s / world * step_bytes / 1e9,
                 "frac": site_steps_per_s / world * step_bytes / 1e9 / hbm}

    # end to end through the public API with host buffers: the protocol table
    # H2D (and spheroid reseed) inside the timed region, then E simulated hours
    # from the seeded start, the fitness read back after every hour
    E = min(K, 5)
    barrier()
    t0 = time.perf_counter()
    sim.load_protocols(off, d, w)
    for _ in range(E):
        sim.run(STEPS_PER_HOUR)
        cnt, fit = sim.fitness()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = world * N_PROT * STEPS_PER_HOUR * E / e2e_s / (mean_h * STEPS_PER_HOUR)
    h2d = (off.nbytes + d.nbytes + w.nbytes) / E
    d2h = cnt.nbytes + fit.nbytes

    # plain form: one protocol at a time, per-step launches, no graph
    plain = Simulator(Ls[:1], Rs[:1], seed=SEED, precision=args.precision, use_graphs=False, dose_cap_gy=30.0,
                      device=dev, path=args.path, params=PARAMS, t_end_steps=t_end_steps())
    po, pd, pw = csr(prot[:1])
    plain.load_protocols(po, pd, pw)
    plain.run(50)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    plain.run(STEPS_PER_HOUR)
    b.record(stream)
    torch.cuda.synchronize()
    # the plain form evaluates protocols one after another: scale the first protocol's time by lattice volume
    plain_val = STEPS_PER_HOUR / (a.elapsed_time(b) / 1e3) / (mean_h * STEPS_PER_HOUR) * \
        float(Ls[0]) ** 3 / float(np.mean(Ls.astype(np.float64) ** 3))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == "fp32" else args.precision, "data": "synthetic",
                "config": dict(workload_config(mean_h, args.precision), path=args.path, tile_shape=shape,
                               autotune_ms_per_step=None if shape_ms is None else [round(x, 4) for x in shape_ms]),
                "site_updates_per_s": site_steps_per_s,
                "roofline": roof, "step_roofline": roof_step,
                "plain": {"value": plain_val, "unit": UNIT,
                          "how": "one protocol per launch sequence, per-step launches, no graph"},
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "steps": E, "window": f"hours 0..{E} after sim_load_protocols (the load, its H2D copy "
                                              "and the re-seeding inside the timed region)"},
                "gpu_launches": launches_per_step * K,
                "clocks": clk.summary()}
        if args.precision != "fp32" or args.error_vs_oracle:
            line["error_vs_oracle"] = precision_error(args.precision, args.error_sample, args.error_steps)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(mean_h)
        print(json.dumps(line))
    sim.close()
    plain.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def full_run(args, sim, prot, mean_h, Ls, shape, shape_ms, world, rank, dev, barrier):
    """The whole job: every protocol of the batch run to its own horizon and
    scored, timed as one step (no extrapolation from early hours)."""
    import torch
    from paper_2303_08123_b300 import csr
    stream = torch.cuda.current_stream(dev)
    horizons = np.array([t_end_steps() / STEPS_PER_HOUR if t_end_steps() else sum(w) + 120.0 for _, w in prot])
    barrier()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        start.record(stream)
        sim.run(0)
        cnt, _ = sim.fitness()
        stop.record(stream)
        barrier()
    ms = start.elapsed_time(stop)
    t = torch.tensor([ms], device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms = float(t.item())
    if rank == 0:
        sites = Ls.astype(np.float64) ** 3
        site_steps = float(np.sum(sites * horizons)) * STEPS_PER_HOUR
        line = {"metric": METRIC, "value": world * N_PROT / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": 1,
                "warmup": 0, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == "fp32" else args.precision, "data": "synthetic",
                "config": dict(workload_config(mean_h, args.precision), path=args.path, tile_shape=shape,
                               step="the whole batch, every protocol to its own horizon, then scored",
                               protocols_per_s="protocols / wall time of the whole batch (measured, not extrapolated)",
                               max_horizon_h=float(horizons.max())),
                "site_updates_per_s": world * site_steps / (ms / 1e3),
                "final_count_mean": float(np.mean(cnt)),
                # every CA step: the fused passes, claim, resolve; every hour: clock tick and count; then fitness
                "gpu_launches": int(STEPS_PER_HOUR * horizons.max() * ((fused_passes(shape)[0] + 2)
                                                                       if args.path == "fused" else PARAMS.n_sub + 3)
                                    + 2 * int(np.ceil(horizons.max())) + 1),
                "clocks": clk.summary()}
        print(json.dumps(line))
    sim.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--path", default="fused", choices=["fused", "substep"])
    ap.add_argument("--tile-shape", type=int, default=0, help="fused tile shape 1-8 (0: autotune)")
    ap.add_argument("--z-chunk", type=int, default=0, help="planes per fused CTA (0: split to fill the GPU)")
    ap.add_argument("--workload", default="ragged", choices=["ga_batch", "ragged", "single"],
                    help="ragged: 1,024 protocols on 32^3-112^3 (default); ga_batch: 256 x 64^3; "
                         "single: one protocol on 40^3 for 288 h")
    ap.add_argument("--start-hour", type=int, default=None,
                    help="simulated hour at which the timed window opens (default 24; 0 for --workload single)")
    ap.add_argument("--error-vs-oracle", action="store_true",
                    help="report error_vs_oracle for FP32 storage too (always reported for BF16 / FP16)")
    ap.add_argument("--error-sample", type=int, default=8,
                    help="2-byte storage: protocols checked against the oracle for error_vs_oracle")
    ap.add_argument("--error-steps", type=int, default=1200,
                    help="2-byte storage: steps of the error_vs_oracle check")
    ap.add_argument("--protocols", type=int, default=None,
                    help="batch size per GPU (default 1,024 ragged, 256 ga_batch; smaller: profiling cases)")
    ap.add_argument("--params", default="p0", choices=["p0", "phys"],
                    help="p0: coarse-grained diffusion (4 substeps per step); phys: physical-rate variant "
                         "(128 substeps per step)")
    ap.add_argument("--full-run", action="store_true",
                    help="time the whole batch to every horizon (about ten minutes for the default workload)")
    args = ap.parse_args()
    global N_PROT, WORKLOAD, PARAMS, PARAMS_NOTE, START_HOUR
    WORKLOAD = args.workload
    START_HOUR = args.start_hour if args.start_hour is not None else (0 if args.workload == "single" else 24)
    if args.params == "phys":
        PARAMS, PARAMS_NOTE = P_PHYS, " (physical-rate diffusion variant, uptake per substep scaled by 4/128)"
    N_PROT = args.protocols if args.protocols else (1024 if args.workload == "ragged" else 256)
    if args.workload == "single":
        N_PROT = 1
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""Surrogate-screened GA: the network ranks a large pool of candidate protocols,
the full batched simulator evaluates the ones it promotes.

The paper's GA scores every candidate with the simulator ("The Main GA Loop");
here the simulator still scores every protocol that enters the
population, and the surrogate (trained on the simulator's own output) only
decides which candidates are worth simulating.

    features(protocols)         15 slots x (dose / 5 Gy, wait / 60 h, mask) = 45 inputs
    simulate(protocols, ...)    final live counts from one batched libsim run
    fit_surrogate(net, X, y)    minibatch Adam on standardised targets
    run_ga(...)                 GA generations, optionally screened by a surrogate
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import ga
from .sim import Simulator, csr
from .surrogate import Surrogate

MAX_FRAC = 15


def features(protocols, dose_scale: float = 5.0, wait_scale: float = 60.0) -> np.ndarray:
    X = np.zeros((len(protocols), 3 * MAX_FRAC), dtype=np.float32)
    for i, (d, w) in enumerate(protocols):
        k = min(len(d), MAX_FRAC)
        X[i, 0:3 * k:3] = np.asarray(d[:k]) / dose_scale
        X[i, 1:3 * k:3] = np.asarray(w[:k]) / wait_scale
        X[i, 2:3 * k:3] = 1.0
    return X


@dataclasses.dataclass
class SimSetup:
    L: int = 24
    R: int = 5
    regrowth_h: int = 6
    seed: int = 0x6A
    dose_cap_gy: float = 30.0
    params: object = None


def simulate(protocols, setup: SimSetup, seed_offset: int = 0) -> np.ndarray:
    """Final live-cell count of every protocol (one batched run to each horizon)."""
    kw = {} if setup.params is None else {"params": setup.params}
    sim = Simulator([setup.L] * len(protocols), [setup.R] * len(protocols), seed=setup.seed + seed_offset,
                    regrowth_h=setup.regrowth_h, dose_cap_gy=setup.dose_cap_gy, max_fractions=MAX_FRAC, **kw)
    sim.load_protocols(*csr(protocols))
    sim.run(0)
    n, _ = sim.fitness()
    sim.close()
    return n.astype(np.float64)


def fit_surrogate(net: Surrogate, X, y, epochs: int = 200, batch: int = 256, lr: float = 1e-3, seed: int = 0):
    """Train on standardised targets; returns (mean, std) to undo the scaling."""
    rng = np.random.default_rng(seed)
    mu, sd = float(np.mean(y)), float(np.std(y) + 1e-9)
    t = ((np.asarray(y) - mu) / sd).astype(np.float32)
    n = (len(X) // batch) * batch
    for _ in range(epochs):
        perm = rng.permutation(len(X))[:n]
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            net.train_step(X[idx], t[idx], lr)
    return mu, sd


def run_ga(setup: SimSetup, cfg: ga.GAConfig, generations: int, rng, net: Surrogate | None = None,
           pool: int = 0, scaling=None, log=None):
    """GA with elitism.  Without a surrogate every child is simulated; with one,
    `pool` children are generated per generation, the surrogate keeps the
    cfg.population - elites most promising (lowest predicted count) and only
    those are simulated.  Returns per-generation best count and simulations used.
    `log` (a writable text file, optional) receives one JSON line per generation:
    best and mean final count, simulations so far, the best protocol."""
    import json

    def record(g, counts, pop, used):
        if log is not None:
            b = int(np.argmin(counts))
            doses, waits = ga.to_pairs(pop[b])
            log.write(json.dumps({"generation": g, "best_count": float(counts[b]), "mean_count": float(counts.mean()),
                                  "simulations": used, "best_protocol": {"dose_gy": doses, "wait_h": waits}}) + "\n")
            log.flush()

    pop = [ga.random_protocol(cfg, rng) for _ in range(cfg.population)]
    counts = simulate([ga.to_pairs(p) for p in pop], setup, seed_offset=0)
    used = len(pop)
    history = [(float(counts.min()), used)]
    record(0, counts, pop, used)
    for g in range(1, generations + 1):
        elites, children = ga.next_generation(pop, -counts, cfg, rng,
                                              n_children=pool if net is not None else None)
        if net is not None:
            pred = net.predict(features([ga.to_pairs(c) for c in children]))
            keep = np.argsort(pred, kind="stable")[:cfg.population - len(elites)]
            children = [children[i] for i in keep]
        pop = elites + children
        counts = simulate([ga.to_pairs(p) for p in pop], setup, seed_offset=g)
        used += len(pop)
        history.append((float(counts.min()), used))
        record(g, counts, pop, used)
    return history


def simulations_to_equal_best(plain_hist, screened_hist, training: int):
    """Full simulations each arm spent until its best-so-far count first reached
    the best count the plain GA reaches by its last generation; the screened
    arm's training simulations are counted.  Returns (target count, plain
    simulations, screened simulations or None if it never got there)."""
    def first(hist, target, extra):
        best = float("inf")
        for count, used in hist:
            best = min(best, count)
            if best <= target:
                return used + extra
        return None
    target = min(c for c, _ in plain_hist)
    return target, first(plain_hist, target, 0), first(screened_hist, target, training)


def compare_arms(setup: SimSetup, cfg: ga.GAConfig, generations: int, plain_population: int,
                 simulated: int, pool: int, train: int, seed: int, epochs: int = 60, log_dir: str = ""):
    """The plain GA (plain_population children simulated per generation) against
    the screened GA (pool candidates per generation, the surrogate's best
    `simulated` of them simulated), the surrogate trained first on `train`
    simulated random protocols.  Returns a dict with both histories (best count,
    cumulative simulations per generation) and simulations_to_equal_best."""
    rng = np.random.default_rng(seed)
    train_set = [ga.to_pairs(ga.random_protocol(cfg, rng)) for _ in range(train)]
    y = simulate(train_set, setup, seed_offset=10_000)
    net = Surrogate(batch_max=max(4096, pool), seed=seed)
    fit_surrogate(net, features(train_set), y, epochs=epochs)
    out = {}
    for arm, population, kw in (("plain", plain_population, {}),
                                ("screened", simulated, {"net": net, "pool": pool})):
        log = open(f"{log_dir}/ga_{arm}.jsonl", "w") if log_dir else None
        hist = run_ga(setup, dataclasses.replace(cfg, population=population), generations,
                      np.random.default_rng(seed + 1), log=log, **kw)
        if log:
            log.close()
        out[arm] = hist
    net.close()
    out["training_simulations"] = train
    out["target"], out["plain_sims_to_best"], out["screened_sims_to_best"] = \
        simulations_to_equal_best(out["plain"], out["screened"], train)
    return out


def main():
    """Screened vs unscreened GA on small lattices: best final count reached
    against the number of full simulations spent (one JSON line per arm)."""
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2048)
    ap.add_argument("--generations", type=int, default=12)
    ap.add_argument("--population", type=int, default=128)
    ap.add_argument("--pool", type=int, default=2048)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--log", default="", help="directory for one JSONL file per arm (generation by generation)")
    ap.add_argument("--compare", action="store_true",
                    help="simulations-to-equal-best: plain GA of --plain-population against the screened GA "
                         "simulating --simulated of --pool candidates per generation")
    ap.add_argument("--plain-population", type=int, default=4096)
    ap.add_argument("--simulated", type=int, default=512)
    ap.add_argument("--L", type=int, default=24)
    ap.add_argument("--R", type=int, default=5)
    a = ap.parse_args()
    if a.compare:
        setup = SimSetup(L=a.L, R=a.R, regrowth_h=6)
        cfg = ga.GAConfig(n_slots=48, d_max=2.5, total_cap=8.0, min_gap=4,
                          mutations=("swap", "split", "dose_time", "dose_value"), p_mut=0.5)
        r = compare_arms(setup, cfg, a.generations, a.plain_population, a.simulated, a.pool, a.train, a.seed,
                         log_dir=a.log)
        print(json.dumps({"lattice": a.L, "radius": a.R, "generations": a.generations,
                          "plain_population": a.plain_population, "pool": a.pool, "simulated": a.simulated,
                          "training_simulations": a.train, "target_count": r["target"],
                          "plain_sims_to_best": r["plain_sims_to_best"],
                          "screened_sims_to_best": r["screened_sims_to_best"],
                          "plain_best": [h[0] for h in r["plain"]], "screened_best": [h[0] for h in r["screened"]],
                          "plain_sims": [h[1] for h in r["plain"]],
                          "screened_sims": [h[1] + a.train for h in r["screened"]]}))
        return
    setup = SimSetup(L=24, R=5, regrowth_h=6)
    cfg = ga.GAConfig(n_slots=48, d_max=2.5, total_cap=8.0, min_gap=4, population=a.population,
                      mutations=("swap", "split", "dose_time", "dose_value"), p_mut=0.5)
    rng = np.random.default_rng(a.seed)
    train = [ga.to_pairs(ga.random_protocol(cfg, rng)) for _ in range(a.train)]
    y = simulate(train, setup, seed_offset=10_000)
    net = Surrogate(batch_max=4096, seed=a.seed)
    fit_surrogate(net, features(train), y, epochs=60)
    for arm, kw in (("full simulation only", {}), ("surrogate-screened", {"net": net, "pool": a.pool})):
        log = open(f"{a.log}/ga_{arm.split()[0].replace('-', '_')}.jsonl", "w") if a.log else None
        hist = run_ga(setup, cfg, a.generations, np.random.default_rng(a.seed + 1), log=log, **kw)
        if log:
            log.close()
        extra = a.train if kw else 0
        print(json.dumps({"arm": arm, "best_count": [h[0] for h in hist],
                          "simulations": [h[1] + extra for h in hist], "training_simulations": extra}))


if __name__ == "__main__":
    main()

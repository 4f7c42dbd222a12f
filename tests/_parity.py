"""Helpers shared by the GPU parity tests: synthetic lattice states and the
comparison rule for one step (fields within tolerance, discrete state
bit-exact except near-threshold decisions and their 2-hop neighbourhood)."""
import numpy as np

from synth.params import P0, M

FIELD_TOL = 1e-5  # per-step field tolerance, relative to the medium value of each field
# Near-threshold decisions (oracle margin inside the field tolerance) must stay
# below this share of all threshold decisions of a run.
NEAR_RATIO_MAX = 1e-6
# One flipped near-threshold decision changes at most three cell words within
# one step: its own site, the site its division would have filled, and the
# competing parent that wins (or loses) that site instead.
MISMATCH_PER_NEAR = 3


def medium(p=P0):
    return np.array([p.medium_O, p.medium_G, 10 ** (3 - p.medium_pH)])


def coords(L):
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def interior_mask(L):
    x, y, z = coords(L)
    return (x > 0) & (y > 0) & (z > 0) & (x < L - 1) & (y < L - 1) & (z < L - 1)


def random_state(L, seed, p=P0):
    """A crowded lattice whose fields straddle every threshold, in FP32."""
    rng = np.random.default_rng(seed)
    n = L ** 3
    inner = interior_mask(L)
    durs = [int(round(h * 600)) for h in p.dur_h]
    kind = rng.choice([0, 0, 1, 2, 3, 4, 4, 5], size=n)
    kind[~inner] = 0
    age = np.zeros(n, dtype=np.int64)
    for k in range(1, 5):
        sel = kind == k
        age[sel] = rng.integers(0, durs[k - 1], size=int(sel.sum()))
    near_end = (kind >= 1) & (kind <= 4) & (rng.random(n) < 0.3)
    age[near_end] = np.array(durs)[kind[near_end] - 1] - 1
    capped = (kind == M) & (rng.random(n) < 0.3)
    age[capped] = durs[3]
    doomed = (kind > 0) & (rng.random(n) < 0.1)
    cell = (kind | (age << 4) | (doomed * 8)).astype(np.uint32)
    med = medium(p)
    O = np.where(inner, rng.uniform(0.0, 0.3, n), med[0])
    G = np.where(inner, rng.uniform(0.0, 5.6, n), med[1])
    H = np.where(inner, rng.uniform(med[2], 6e-4, n), med[2])
    return [a.astype(np.float32) for a in (O, G, H)], cell


def near_ratio(stats):
    """Share of the oracle's threshold decisions that fell inside the near band."""
    return stats["n_near"] / max(1, stats["n_decisions"])


def dilate(mask, L, hops):
    m = mask.reshape(L, L, L).copy()
    for _ in range(hops):
        out = m.copy()
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    out |= np.roll(np.roll(np.roll(m, dz, 0), dy, 1), dx, 2)
        m = out
    return m.ravel()


def oracle_state(orc, L, fields, cell):
    st = orc.State(L)
    st.O[:], st.G[:], st.H[:] = (f.astype(np.float64) for f in fields)
    st.cell[:] = cell
    return st


def compare(L, gpu_fields, gpu_cell, ora_state, near, field_tol=FIELD_TOL, hops=2):
    """Field error (max over fields, relative to medium) and cell mismatches,
    split into those a near-threshold decision explains and the rest."""
    med = medium()
    errs = [float(np.max(np.abs(g.astype(np.float64) - o))) / m
            for g, o, m in zip(gpu_fields, (ora_state.O, ora_state.G, ora_state.H), med)]
    diff = gpu_cell != ora_state.cell
    ok = dilate(near != 0, L, hops)
    return dict(field_err=max(errs), field_errs=errs, mismatch=int(diff.sum()),
                unexplained=int((diff & ~ok).sum()), near=int(np.count_nonzero(near)))


def assert_one_step(r):
    """The one-step rule: fields within tolerance, every cell mismatch inside a
    flagged neighbourhood, and no more mismatches than the flagged decisions can
    cause."""
    assert r["field_err"] <= FIELD_TOL, r
    assert r["unexplained"] == 0, r
    assert r["mismatch"] <= MISMATCH_PER_NEAR * r["near"], r

"""Seeded random enumeration cases for the fuzz tests (a test helper: lattices and planning options
drawn from the seeded generator of the workloads module; no method arithmetic)."""
from __future__ import annotations

import numpy as np

from paper_1110_2561_gb300 import workloads as w

ALPHABETS = [(1,), (-1, 1), (-2, -1, 1, 2), (-3, 1, 2), (5, -7)]


def draw_lattice(rng: w.SplitMix64, n_lo: int, n_hi: int) -> w.Lattice:
    n = n_lo + rng.below(n_hi - n_lo + 1)
    kind = rng.below(4)
    J = ALPHABETS[rng.below(len(ALPHABETS))]
    if kind == 3:
        return w.random_graph(n, rng.below(3 * n + 1), rng, couplings=J)
    lat = w.induced_lattice(("square", "triangular", "cubic")[kind], n, rng.below(2) == 1, rng, couplings=J)
    return lat


def draw_options(rng: w.SplitMix64, n: int) -> dict:
    """Planning options that every graph of n >= 11 spins accepts (or that the planner rejects with
    a status, which the tests then expect)."""
    o = {}
    o["lane_model"] = rng.below(5)
    if rng.below(3) == 0:
        o["symmetry"] = 1
    elif rng.below(3) == 0:
        k = 1 + rng.below(3)
        lo = rng.below(1 << k)
        o.update(shard_bits=k, shard_lo=lo, shard_hi=lo + 1 + rng.below((1 << k) - lo))
    fixed = 1 if "symmetry" in o else o.get("shard_bits", 0)
    if rng.below(2) == 0 and n - fixed - 5 >= 7:
        o["inner_bits"] = 7 + rng.below(n - fixed - 5 - 7 + 1)     # low block (<= 7) <= q <= free - 5
    if rng.below(3) == 0:
        o["low_bits"] = 1 + rng.below(7)
    if rng.below(3) == 0:
        o["block_threads"] = 32 * (1 + rng.below(32))
    if rng.below(4) == 0:
        o["copies"] = 1 + rng.below(3)
    if rng.below(4) == 0:
        o["flush_tasks"] = 1 + rng.below(3)
    return o


def reference_range(o: dict, n: int):
    """The configuration words an option set enumerates: [lo, hi) for a shard range, else all."""
    if "shard_bits" in o:
        k = o["shard_bits"]
        return o["shard_lo"] << (n - k), o["shard_hi"] << (n - k)
    return 0, 1 << n


def cases(seed: int, count: int, n_lo: int, n_hi: int):
    rng = w.SplitMix64(seed)
    out = []
    for _ in range(count):
        lat = draw_lattice(rng, n_lo, n_hi)
        out.append((lat, draw_options(rng, lat.n)))
    return out


def as_edges(lat: w.Lattice) -> np.ndarray:
    return lat.edges

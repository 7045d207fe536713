"""Seeded synthetic inputs: lattices, disorder draws and request streams.

This module builds graphs (edge lists with integer couplings) and random draws only; it holds
none of the enumeration or thermodynamics arithmetic, so both the CUDA path and the CPU oracle
may be fed from it. Randomness comes from a hand-written splitmix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), so the same seed gives the same
inputs on every machine and numpy version.

Lattice conventions (the paper fixes none; Sec. 3 only uses periodic square lattices):
* site index i = (x * Ly + y) for 2-D and (x * Ly + y) * Lz + z for 3-D;
* square: bonds to +x and +y; triangular: also the (+1, +1) diagonal; simple cubic: +x, +y, +z;
* periodic lattices wrap every bond (Sec. 2: periodic boundary conditions); free lattices omit
  the wrapped bonds. A side of length 1 contributes no periodic bond (it would be a self loop);
  a periodic side of length 2 yields the same pair twice, which the graph builders sum.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED = 11102561
MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64: state += golden gamma; output = mix(state). Deterministic across platforms."""

    def __init__(self, seed: int = SEED):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) by rejection (no modulo bias)."""
        if n <= 0:
            raise ValueError("n must be positive")
        limit = (1 << 64) - ((1 << 64) % n)
        while True:
            x = self.next_u64()
            if x < limit:
                return x % n

    def uniform(self) -> float:
        """Uniform float in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def choice(self, seq):
        return seq[self.below(len(seq))]

    def shuffle(self, items: list) -> list:
        for i in range(len(items) - 1, 0, -1):
            j = self.below(i + 1)
            items[i], items[j] = items[j], items[i]
        return items


@dataclass
class Lattice:
    """A graph: n spins and an edge list of (i, j, J) rows (int64 array of shape (n_edges, 3))."""
    n: int
    edges: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.edges.shape[0])


def _offsets(kind: str):
    if kind == "square":
        return [(1, 0), (0, 1)]
    if kind == "triangular":
        return [(1, 0), (0, 1), (1, 1)]
    if kind == "cubic":
        return [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    raise ValueError(f"unknown lattice kind {kind!r}")


def lattice_bonds(kind: str, dims, periodic: bool):
    """List of (i, j) bonds of a full lattice box, site index as in the module docstring."""
    dims = tuple(int(d) for d in dims)
    offs = _offsets(kind)
    if len(dims) != len(offs[0]):
        raise ValueError(f"{kind} lattice needs {len(offs[0])} dimensions, got {dims}")

    def index(c):
        i = 0
        for ci, d in zip(c, dims):
            i = i * d + ci
        return i

    bonds = []
    for c in np.ndindex(*dims):
        for o in offs:
            t = []
            ok = True
            for ci, oi, d in zip(c, o, dims):
                v = ci + oi
                if v >= d:
                    if not periodic or d == 1:
                        ok = False
                        break
                    v -= d
                t.append(v)
            if not ok:
                continue
            i, j = index(c), index(t)
            if i == j:
                continue
            bonds.append((i, j))
    return bonds


def lattice(kind: str, dims, periodic: bool, J: int = 1, name: str | None = None) -> Lattice:
    """Uniform-coupling lattice (J on every bond)."""
    bonds = lattice_bonds(kind, dims, periodic)
    n = int(np.prod(dims))
    e = np.array([(i, j, J) for i, j in bonds], dtype=np.int64).reshape(-1, 3)
    nm = name or f"{kind}{'x'.join(map(str, dims))}{'-pbc' if periodic else '-free'}"
    return Lattice(n, e, nm, {"kind": kind, "dims": tuple(dims), "periodic": periodic})


def square(Lx: int, Ly: int, periodic: bool, J: int = 1) -> Lattice:
    return lattice("square", (Lx, Ly), periodic, J)


def triangular(Lx: int, Ly: int, periodic: bool, J: int = 1) -> Lattice:
    return lattice("triangular", (Lx, Ly), periodic, J)


def cubic(Lx: int, Ly: int, Lz: int, periodic: bool, J: int = 1) -> Lattice:
    return lattice("cubic", (Lx, Ly, Lz), periodic, J)


def ring(n: int, J: int = 1) -> Lattice:
    """1-D periodic chain of n >= 3 spins."""
    e = np.array([(i, (i + 1) % n, J) for i in range(n)], dtype=np.int64)
    return Lattice(n, e, f"ring{n}", {"kind": "ring"})


def random_graph(n: int, n_edges: int, rng: SplitMix64, couplings=(-2, -1, 1, 2)) -> Lattice:
    """Random multigraph without self loops; couplings drawn uniformly from `couplings`."""
    rows = []
    for _ in range(n_edges):
        i = rng.below(n)
        j = rng.below(n - 1)
        if j >= i:
            j += 1
        rows.append((i, j, rng.choice(couplings)))
    e = np.array(rows, dtype=np.int64).reshape(-1, 3)
    return Lattice(n, e, f"random{n}x{n_edges}", {"kind": "random"})


def with_random_couplings(lat: Lattice, rng: SplitMix64, couplings) -> Lattice:
    e = lat.edges.copy()
    for r in range(e.shape[0]):
        e[r, 2] = rng.choice(couplings)
    return Lattice(lat.n, e, lat.name + "-rand", dict(lat.meta))


def ea_instances(count: int = 4096, shapes=((4, 4), (4, 5), (5, 5), (5, 6)), seed: int = SEED):
    """Edwards-Anderson +-J instances on periodic square lattices of the given shapes in equal
    shares (count must be a multiple of len(shapes)), couplings uniform in {-1, +1}, the
    instance order shuffled. One splitmix64 stream drives the couplings, then the shuffle."""
    if count % len(shapes):
        raise ValueError("count must be a multiple of the number of shapes")
    rng = SplitMix64(seed)
    out = []
    for s, (lx, ly) in enumerate(shapes):
        base = square(lx, ly, True)
        for k in range(count // len(shapes)):
            lat = with_random_couplings(base, rng, (-1, 1))
            lat.name = f"ea{lx}x{ly}#{k}"
            out.append(lat)
    return rng.shuffle(out)


def _near_box(kind: str, n: int):
    """Smallest near-square (2-D) or near-cube (3-D) box with at least n sites."""
    if kind == "cubic":
        a = max(1, round(n ** (1.0 / 3.0)))
        best = None
        for x in range(max(1, a - 2), a + 3):
            for y in range(x, a + 4):
                for z in range(y, a + 5):
                    v = x * y * z
                    if v >= n and (best is None or (v, z - x) < (best[0], best[1])):
                        best = (v, z - x, (x, y, z))
        return best[2]
    a = max(1, math.isqrt(n))
    best = None
    for x in range(max(1, a - 2), a + 3):
        y = -(-n // x)
        v = x * y
        if best is None or (v, abs(y - x)) < (best[0], best[1]):
            best = (v, abs(y - x), (x, y))
    return best[2]


def induced_lattice(kind: str, n: int, periodic: bool, rng: SplitMix64, couplings=(-2, -1, 1, 2)) -> Lattice:
    """Lattice of exactly n spins: the near-square/near-cube box with >= n sites, restricted to
    its first n sites in index order (bonds, wrapped ones included, whose ends both survive),
    with couplings drawn per bond."""
    dims = _near_box(kind, n)
    bonds = [(i, j) for i, j in lattice_bonds(kind, dims, periodic) if i < n and j < n]
    rows = [(i, j, rng.choice(couplings)) for i, j in bonds]
    e = np.array(rows, dtype=np.int64).reshape(-1, 3)
    return Lattice(n, e, f"{kind}{n}{'-pbc' if periodic else '-free'}",
                   {"kind": kind, "dims": dims, "periodic": periodic})


@dataclass
class Request:
    arrival_s: float
    lattice: Lattice


def serving_stream(n_requests: int, rate_per_s: float = 50.0, n_range=(16, 38), seed: int = SEED,
                   couplings=(-2, -1, 1, 2)):
    """Poisson arrivals (exponential gaps of mean 1/rate) of lattice requests: N uniform in
    n_range (inclusive), geometry uniform over square / triangular / cubic, periodic or free
    with equal odds, couplings uniform over `couplings` per bond."""
    rng = SplitMix64(seed ^ 0x5E7E)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += -math.log(1.0 - rng.uniform()) / rate_per_s
        n = n_range[0] + rng.below(n_range[1] - n_range[0] + 1)
        kind = rng.choice(("square", "triangular", "cubic"))
        periodic = rng.below(2) == 1
        out.append(Request(t, induced_lattice(kind, n, periodic, rng, couplings)))
    return out


def temperature_grid(lo: float, hi: float, n: int) -> np.ndarray:
    return np.linspace(lo, hi, n, dtype=np.float64)

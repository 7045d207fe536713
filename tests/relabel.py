"""Spin relabelling for the oracle's frontier programme (test helper; no method arithmetic).

The frontier programme of the oracle adds sites in index order and keeps a table over the sites
that still have a bond to a site not yet added, so its cost grows as 2^(width of that frontier).
The table g(E, M) does not depend on how the spins are numbered (E and M are sums over bonds and
spins), so a test may renumber a lattice before handing it to the oracle. Numbering the sites
with the shortest side of the box varying fastest keeps the frontier to about one (free) or two
(periodic) cross-sections of the box; conditioning the programme on the spins of the first
cross-section along the longest side (``layer_cut``) turns a periodic box's wrap-around bonds into
fields, so the rest's frontier holds about one cross-section.
"""
from __future__ import annotations

import numpy as np

from paper_1110_2561_gb300 import workloads as w


def short_side_fastest(lat: w.Lattice) -> w.Lattice:
    """The same graph with its sites renumbered so that the box's coordinates vary fastest along
    the shortest side and slowest along the longest (sites of an induced lattice keep their
    relative order within that numbering). Lattices without box dimensions are returned as they
    are."""
    dims = lat.meta.get("dims")
    if not dims:
        return lat
    dims = tuple(int(d) for d in dims)
    coords = np.array(np.unravel_index(np.arange(lat.n), dims)).T          # site i = row-major index
    slow_to_fast = sorted(range(len(dims)), key=lambda a: -dims[a])         # longest side slowest
    key = np.zeros(lat.n, dtype=np.int64)
    for a in slow_to_fast:
        key = key * dims[a] + coords[:, a]
    order = np.argsort(key, kind="stable")
    new = np.empty(lat.n, dtype=np.int64)
    new[order] = np.arange(lat.n)
    e = lat.edges.copy()
    e[:, 0] = new[e[:, 0]]
    e[:, 1] = new[e[:, 1]]
    return w.Lattice(lat.n, e, lat.name + "-relabelled", dict(lat.meta))


def layer_cut(lat: w.Lattice):
    """(the lattice numbered by short_side_fastest, cut mask): the cut holds the sites whose
    coordinate along the box's longest side is 0 (the first cross-section in that numbering), for
    the oracle's programme conditioned on a cut. A lattice without box dimensions gets an empty cut."""
    dims = lat.meta.get("dims")
    r = short_side_fastest(lat)
    if not dims:
        return r, 0
    dims = tuple(int(d) for d in dims)
    coords = np.array(np.unravel_index(np.arange(lat.n), dims)).T
    slowest = max(range(len(dims)), key=lambda a: (dims[a], -a))
    # short_side_fastest keeps the site order along the slowest side, so the sites with coordinate 0
    # there are renumbered 0 .. k-1
    k = int((coords[:, slowest] == 0).sum())
    return r, (1 << k) - 1


def frontier_table(lat: w.Lattice, threads: int = 1):
    """The oracle's exact table of a box lattice by its frontier programme: sites renumbered along
    the short side, and for periodic cubic lattices (whose frontier spans two cross-sections and
    their wrap-around) conditioned on the first cross-section."""
    import oracle
    if lat.meta.get("kind") == "cubic" and lat.meta.get("periodic"):
        r, cut = layer_cut(lat)
        return oracle.g_frontier_cut(r.n, r.edges, cut, max_active=20, threads=threads)
    r = short_side_fastest(lat)
    return oracle.g_frontier(r.n, r.edges, max_active=20)

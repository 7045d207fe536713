"""The test helper that renumbers sites for the oracle's frontier programme keeps the table: on
small lattices of every kind the renumbered graph's oracle table equals the original's, and the
first-layer cut is that cross-section and gives the same table."""
import numpy as np
import pytest

import oracle
from paper_1110_2561_gb300 import workloads as w
from relabel import layer_cut, short_side_fastest


@pytest.mark.parametrize("lat", [w.square(3, 5, True), w.square(4, 3, False), w.triangular(3, 4, True),
                                 w.cubic(2, 3, 2, True), w.cubic(3, 2, 2, False),
                                 w.induced_lattice("square", 14, True, w.SplitMix64(3)),
                                 w.induced_lattice("triangular", 13, False, w.SplitMix64(4)),
                                 w.induced_lattice("cubic", 15, False, w.SplitMix64(5))],
                         ids=lambda l: l.name)
def test_relabelled_lattice_has_the_same_table(lat):
    r = short_side_fastest(lat)
    assert r.n == lat.n and sorted(np.bincount(r.edges[:, :2].ravel(), minlength=r.n)) == \
        sorted(np.bincount(lat.edges[:, :2].ravel(), minlength=lat.n))
    assert np.array_equal(oracle.g_edges(r.n, r.edges), oracle.g_edges(lat.n, lat.edges))
    assert np.array_equal(oracle.g_frontier(r.n, r.edges, max_active=20), oracle.g_edges(lat.n, lat.edges))


@pytest.mark.parametrize("lat", [w.square(3, 5, True), w.cubic(2, 3, 3, True), w.cubic(3, 2, 2, False),
                                 w.induced_lattice("cubic", 15, True, w.SplitMix64(6)),
                                 w.induced_lattice("square", 14, True, w.SplitMix64(7)),
                                 w.induced_lattice("triangular", 13, True, w.SplitMix64(8))],
                         ids=lambda l: l.name)
def test_layer_cut(lat):
    r, cut = layer_cut(lat)
    dims = lat.meta["dims"]
    coords = np.array(np.unravel_index(np.arange(lat.n), dims)).T
    slowest = max(range(len(dims)), key=lambda a: (dims[a], -a))
    k = int((coords[:, slowest] == 0).sum())
    assert cut == (1 << k) - 1 and 0 < k < lat.n
    assert np.array_equal(oracle.g_frontier_cut(r.n, r.edges, cut), oracle.g_edges(lat.n, lat.edges))

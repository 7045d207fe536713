"""Seeded random enumerations on the host: the kernels' walk (isg_debug_emulate, every counter
address checked against its lane's histogram bins) with random lattices, couplings and planning
options, against the oracle's popcount table over the same configuration range. An option set
the planner cannot take must be refused with a status."""
import numpy as np
import pytest

import oracle
import fuzz_cases as fc


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_emulated_walk_fuzz(isg, seed):
    done = 0
    for lat, o in fc.cases(seed, 60, 11, 18):
        g = isg.isg_graph_create(lat.n, lat.edges)
        lo, hi = fc.reference_range(o, lat.n)
        try:
            got = isg.isg_debug_emulate(g, **o)
        except isg.IsgError as e:
            assert e.status in (1, 2), (lat.name, o, str(e))       # INVALID or TOO_LARGE, nothing else
            continue
        assert np.array_equal(got, oracle.g_masks(lat.n, lat.edges, lo, hi)), (lat.name, o)
        done += 1
    assert done >= 45

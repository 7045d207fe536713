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


@pytest.mark.parametrize("seed", [21, 22])
def test_emulated_walk_fuzz_large_graphs_on_shards(isg, seed):
    """Graphs of 27 to 40 spins with random planning options, each walked on the host over one
    random shard of 2^16 configurations (shard_bits = N - 16): the oracle's table of that range, or
    a refusal with INVALID or TOO_LARGE (for example lane tables whose rows do not fit)."""
    from paper_1110_2561_gb300 import workloads as w
    rng = w.SplitMix64(seed)
    done = 0
    for _ in range(24):
        lat = fc.draw_lattice(rng, 27, 40)
        n = lat.n
        k = n - 16
        lo = rng.below(1 << k)
        o = dict(shard_bits=k, shard_lo=lo, shard_hi=lo + 1, lane_model=rng.below(5))
        if rng.below(2) == 0:
            o["inner_bits"] = 7 + rng.below(5)           # q in [7, 11] = free - 5
        if rng.below(3) == 0:
            o["low_bits"] = 1 + rng.below(7)
        if rng.below(3) == 0:
            o["block_threads"] = 32 * (1 + rng.below(32))
        if rng.below(4) == 0:
            o["copies"] = 1 + rng.below(3)
        if rng.below(4) == 0:
            o["flush_tasks"] = 1 + rng.below(3)
        g = isg.isg_graph_create(n, lat.edges)
        try:
            got = isg.isg_debug_emulate(g, **o)
        except isg.IsgError as e:
            assert e.status in (1, 2), (lat.name, o, str(e))
            continue
        assert np.array_equal(got, oracle.g_masks(n, lat.edges, lo << 16, (lo + 1) << 16)), (lat.name, o)
        done += 1
    assert done >= 16

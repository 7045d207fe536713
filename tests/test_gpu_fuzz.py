"""Seeded random enumerations on the GPU: random lattices (square, triangular, cubic, random
graphs; periodic or free; five coupling alphabets) and random planning options (lane model 0-4,
symmetry, shard ranges, inner bits, low block, block size, copies, flush interval), device and
host output, against the oracle's popcount table over the same configuration range. An option
set the device refuses, the host walk (which plans the same way) refuses with the same status."""
import os

import numpy as np
import pytest

import oracle
import fuzz_cases as fc

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


@pytest.mark.parametrize("seed", [21, 22])
def test_enumeration_fuzz(isg, cuda, seed):
    import torch
    done = 0
    for k, (lat, o) in enumerate(fc.cases(seed, 50, 11, 26)):
        g = isg.isg_graph_create(lat.n, lat.edges)
        lo, hi = fc.reference_range(o, lat.n)
        try:
            if k % 2:
                out = torch.zeros(isg.table_shape(g), dtype=torch.int64, device=cuda)
                isg.isg_enumerate(g, out, **o)
                torch.cuda.synchronize()
                got = out.cpu().numpy()
            else:
                got = isg.isg_enumerate(g, **o)
        except isg.IsgError as e:
            assert e.status in (1, 2), (lat.name, o, str(e))
            with pytest.raises(isg.IsgError) as ei:     # the host walk plans the same way: same refusal
                isg.isg_debug_emulate(g, **o)
            assert ei.value.status == e.status
            continue
        ref = oracle.g_masks(lat.n, lat.edges, lo, hi, threads=THREADS)
        assert np.array_equal(got, ref), (lat.name, o)
        done += 1
    assert done >= 35
    isg.isg_device_status()


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_batch_fuzz(isg, cuda, seed):
    """Random batches: 3 to 40 graphs of 3 to 24 spins (tiny ones for the thread-per-configuration
    kernel among them), options drawn from symmetry, split-and-convolve service, the lane model and
    the inner bits; every table equals the oracle's."""
    from paper_1110_2561_gb300 import workloads as w
    rng = w.SplitMix64(seed)
    for _ in range(4):
        lats = [fc.draw_lattice(rng, 3, 24) for _ in range(3 + rng.below(38))]
        o = {}
        if rng.below(2):
            o["symmetry"] = 1
        if rng.below(2):
            o["split"] = 1
        o["lane_model"] = (0, 1, 2, 3)[rng.below(4)]
        if rng.below(3) == 0:
            o["inner_bits"] = 7 + rng.below(6)
        graphs = [isg.isg_graph_create(l.n, l.edges) for l in lats]
        got = isg.isg_enumerate_batch(graphs, **o)
        for l, t in zip(lats, got):
            assert np.array_equal(t, oracle.g_masks(l.n, l.edges, threads=THREADS)), (l.name, o)
    isg.isg_device_status()

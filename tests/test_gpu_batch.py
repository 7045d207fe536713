"""Batched enumeration (isg_enumerate_batch, prepared batches with CUDA-graph replay) against the
oracle and against per-instance isg_enumerate."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1110_2561_gb300 import workloads as w

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


def mixed_graphs():
    rng = w.SplitMix64(31)
    gs = [w.square(4, 4, True), w.ring(5), w.Lattice(3, np.zeros((0, 3), np.int64), "free3"),
          w.with_random_couplings(w.square(4, 5, True), rng, (-1, 1)),
          w.with_random_couplings(w.triangular(4, 4, False), rng, (-2, -1, 1, 2)),
          w.cubic(2, 2, 3, True), w.random_graph(14, 40, rng), w.square(1, 2, False),
          w.induced_lattice("triangular", 19, True, rng)]
    return gs


def test_mixed_batch_against_oracle(isg, cuda):
    lats = mixed_graphs()
    hs = [isg.isg_graph_create(l.n, l.edges) for l in lats]
    outs = isg.isg_enumerate_batch(hs)                       # host tables
    for l, g in zip(lats, outs):
        assert np.array_equal(g, oracle.g_masks(l.n, l.edges, threads=THREADS)), l.name


def test_batch_device_tables_and_options(isg, cuda):
    import torch
    lats = mixed_graphs()
    hs = [isg.isg_graph_create(l.n, l.edges) for l in lats]
    ref = [oracle.g_masks(l.n, l.edges, threads=THREADS) for l in lats]
    for kw in [{}, dict(inner_bits=6), dict(low_bits=2, block_threads=64), dict(ctas_per_sm=1, block_threads=256),
               dict(lane_model=1), dict(lane_model=1, inner_bits=7, symmetry=1)]:
        outs = [torch.zeros(isg.table_shape(h), dtype=torch.int64, device=cuda) for h in hs]
        isg.isg_enumerate_batch(hs, outs, **kw)
        for o, r, l in zip(outs, ref, lats):
            assert np.array_equal(o.cpu().numpy(), r), (l.name, kw)


def test_batch_symmetry(isg, cuda):
    """Symmetry halving in a batch (mixed sizes, small graphs included) equals the oracle."""
    lats = mixed_graphs()
    hs = [isg.isg_graph_create(l.n, l.edges) for l in lats]
    outs = isg.isg_enumerate_batch(hs, symmetry=1)
    for l, g in zip(lats, outs):
        assert np.array_equal(g, oracle.g_masks(l.n, l.edges, threads=THREADS)), l.name
    b = isg.Batch(hs, symmetry=1)
    b.run()
    b.status()
    for k, l in enumerate(lats):
        assert np.array_equal(b.table(k).cpu().numpy(), oracle.g_masks(l.n, l.edges)), l.name
    b.close()


def test_batch_split_and_symmetry(isg, cuda):
    """split = 1 and symmetry = 1 at once on a mixed batch (EA 5x6 instances that go to split
    launches, smaller tile-served and small-kernel graphs): every table equals the oracle's (the
    frontier programme for the EA instances), and replaying the prepared batch gives the same
    tables."""
    from relabel import frontier_table
    lats = [l for l in w.ea_instances(64) if l.n == 30][:6] + mixed_graphs()
    hs = [isg.isg_graph_create(l.n, l.edges) for l in lats]
    ref = [frontier_table(l, THREADS) if l.n > 22 else oracle.g_masks(l.n, l.edges, threads=THREADS) for l in lats]
    outs = isg.isg_enumerate_batch(hs, split=1, symmetry=1)
    for l, g, r in zip(lats, outs, ref):
        assert np.array_equal(g, r), l.name
    b = isg.Batch(hs, split=1, symmetry=1)
    for _ in range(2):
        b.run()
        b.status()
        for k, l in enumerate(lats):
            assert np.array_equal(b.table(k).cpu().numpy(), ref[k]), l.name
    b.close()


def test_batch_rejects_shards(isg, cuda):
    h = isg.isg_graph_create(16, w.square(4, 4, True).edges)
    with pytest.raises(isg.IsgError) as ei:
        isg.isg_enumerate_batch([h], shard_bits=1, shard_hi=1)
    assert ei.value.status == 1
    with pytest.raises(isg.IsgError) as ei:                    # lane tables: single-graph calls only
        isg.isg_enumerate_batch([h], lane_model=4)
    assert ei.value.status == 1


def test_prepared_batch_replay(isg, cuda):
    """Two graph replays of a prepared batch give identical, correct tables."""
    import torch
    lats = mixed_graphs()
    hs = [isg.isg_graph_create(l.n, l.edges) for l in lats]
    b = isg.Batch(hs)
    for _ in range(2):
        b.run()
        b.status()
        for k, l in enumerate(lats):
            assert np.array_equal(b.table(k).cpu().numpy(), oracle.g_masks(l.n, l.edges)), l.name
    b.close()


def test_autotuned_batch(isg, cuda):
    """A batch planned by the autotuner (lane spins of the index order or of the bank-conflict
    model, shared by instances that differ only in coupling signs) gives the same tables as the
    default plan, and every one equals the oracle's frontier programme."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from relabel import frontier_table
    lats = w.ea_instances(count=256, seed=99)
    hs = [isg.isg_graph_create(l.n, l.edges) for l in lats]
    b0, b1 = isg.Batch(hs), isg.Batch(hs, autotune=1)
    b0.run()
    b1.run()
    b1.status()
    with ThreadPoolExecutor(max_workers=THREADS) as ex:
        refs = list(ex.map(frontier_table, lats))
    for k in range(len(lats)):
        assert torch.equal(b0.table(k), b1.table(k)), lats[k].name
        assert np.array_equal(b1.table(k).cpu().numpy(), refs[k]), lats[k].name
    b0.close()
    b1.close()


@pytest.mark.slow
def test_ea_4096_batch(isg, cuda):
    """The 4096 Edwards-Anderson +-J instances (4x4, 4x5, 5x5, 5x6 periodic, equal shares) in one
    prepared batch, autotuned as in the benchmark, and in a prepared batch with split = 1 (the 5x6
    instances by split launches): every one of the 4096 tables of both, bin for bin, equals the
    oracle's frontier programme (sites renumbered along the short side, which leaves g unchanged;
    instances spread over the host cores)."""
    from concurrent.futures import ThreadPoolExecutor
    from relabel import short_side_fastest
    lats = w.ea_instances()
    hs = [isg.isg_graph_create(l.n, l.edges) for l in lats]
    got = []
    for opts in (dict(autotune=1), dict(split=1)):
        b = isg.Batch(hs, **opts)
        b.run()
        b.status()
        got.append([b.table(k).cpu().numpy() for k in range(len(lats))])
        b.close()

    def ref(l):
        r = short_side_fastest(l)
        return oracle.g_frontier(r.n, r.edges, max_active=20)
    with ThreadPoolExecutor(max_workers=THREADS) as ex:
        refs = list(ex.map(ref, lats))
    shapes = set()
    for k, (l, r) in enumerate(zip(lats, refs)):
        assert int(r.sum()) == 1 << l.n
        assert np.array_equal(got[0][k], r), l.name
        assert np.array_equal(got[1][k], r), l.name
        shapes.add(l.n)
    assert shapes == {16, 20, 25, 30}

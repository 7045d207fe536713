"""Split-and-convolve enumeration on the GPU (isg_enumerate_split): exact tables against the
oracle's full enumeration, its frontier programme, and the direct GPU enumeration."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1110_2561_gb300 import workloads as w
from closed_forms import kaufman_energy_counts, kaufman_logz
from test_split_host import CASES, mask

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


@pytest.mark.parametrize("lat,boundary", CASES, ids=[c[0].name or "free-spins" for c in CASES])
def test_split_small_graphs(isg, cuda, lat, boundary):
    gh = isg.isg_graph_create(lat.n, lat.edges)
    # small graphs: the automatic choice is refused (no gain), so pass the planner's set explicitly
    # (an empty set, chosen for a graph without bonds, is written as spin 0 alone)
    boundary = boundary or isg.isg_split_plan(gh)["boundary"] or 1
    assert np.array_equal(isg.isg_enumerate_split(gh, boundary=boundary), oracle.g_masks(lat.n, lat.edges))


def test_split_table1(isg, cuda, table1_triples):
    lat = w.square(4, 4, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = isg.isg_enumerate_split(gh, boundary=mask(range(0, 4)) | mask(range(8, 12)))
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    assert {(int(g[e, m]), -lat.n + 2 * m, e_min + 2 * e) for e, m in zip(*np.nonzero(g))} == set(table1_triples)


def test_split_torus_6x6(isg, cuda):
    """The 6x6 torus with the library's boundary (two rows): every bin against the frontier oracle,
    into a device tensor and into host memory."""
    import torch
    lat = w.square(6, 6, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    ref = oracle.g_frontier(lat.n, lat.edges, 16)
    assert np.array_equal(isg.isg_enumerate_split(gh), ref)
    g = torch.full(isg.table_shape(gh), 7, dtype=torch.int64, device=cuda)      # overwritten
    isg.isg_enumerate_split(gh, g)
    torch.cuda.synchronize()
    assert np.array_equal(g.cpu().numpy(), ref)


def test_split_cubic_against_direct(isg, cuda):
    """3x3x4 cubic torus: the split table equals the direct enumeration's (itself parity-tested)."""
    lat = w.cubic(3, 3, 4, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    assert np.array_equal(isg.isg_enumerate_split(gh), isg.isg_enumerate(gh))


def test_split_ea_instances(isg, cuda):
    """Edwards-Anderson +-J instances of every shape, against the frontier oracle."""
    lats = w.ea_instances()
    for lat in [next(l for l in lats if l.n == n) for n in (16, 20, 25, 30)]:
        gh = isg.isg_graph_create(lat.n, lat.edges)
        b = isg.isg_split_plan(gh)["boundary"]          # explicit: small instances gain nothing automatically
        assert np.array_equal(isg.isg_enumerate_split(gh, boundary=b), oracle.g_frontier(lat.n, lat.edges, 16)), lat.name


def test_split_serving_mix(isg, cuda):
    """Request-stream graphs (square / triangular / cubic, periodic or free, J in {+-1, +-2})."""
    reqs = w.serving_stream(40)
    done = 0
    for r in reqs:
        lat = r.lattice
        if lat.n > 26:
            continue
        gh = isg.isg_graph_create(lat.n, lat.edges)
        try:
            got = isg.isg_enumerate_split(gh)
        except isg.IsgError as e:
            assert "TOO_LARGE" in str(e)        # no boundary cheaper than the full enumeration
            continue
        assert np.array_equal(got, oracle.g_frontier(lat.n, lat.edges, 20)), lat.name
        done += 1
    assert done >= 3


def test_split_torus_7x7(isg, cuda):
    """The 7x7 torus, N = 49 (2^49 configurations): every bin against the oracle's frontier
    programme, and ln Z against Kaufman's closed form."""
    lat = w.square(7, 7, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = isg.isg_enumerate_split(gh)
    assert int(g.sum()) == 2 ** 49
    assert all(int(g[:, m].sum()) == math.comb(49, m) for m in range(50))
    assert np.array_equal(g, oracle.g_frontier(lat.n, lat.edges, 16))
    T = np.array([1.0, 2.269, 3.5])
    lz = isg.isg_thermo(g, gh, T, [0.0], isg.ISG_FP64)[0][:, 0]
    for t, l in zip(T, lz):
        assert abs(l - kaufman_logz(7, 7, t)) <= 1e-12 * abs(l)


def test_split_rejects(isg, cuda):
    lat = w.square(4, 4, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    with pytest.raises(isg.IsgError, match="TOO_LARGE"):
        isg.isg_enumerate_split(gh)              # a 16-spin lattice: no boundary beats the full walk
    with pytest.raises(isg.IsgError, match="INVALID"):
        isg.isg_enumerate_split(gh, boundary=1 << 20)


def test_split_random_graphs(isg, cuda):
    """The seeded random graphs of the host tests (several coupling alphabets, isolated spins,
    empty and full boundary sets) through the kernel: every table equals the oracle's."""
    from test_split_host import _random_cases
    done = 0
    for lat, boundary in _random_cases():
        gh = isg.isg_graph_create(lat.n, lat.edges)
        try:
            b = boundary or isg.isg_split_plan(gh)["boundary"] or 1
            got = isg.isg_enumerate_split(gh, boundary=b)
        except isg.IsgError as e:
            assert "TOO_LARGE" in str(e)
            continue
        assert np.array_equal(got, oracle.g_edges(lat.n, lat.edges)), lat.name
        done += 1
    assert done >= 30


@pytest.mark.parametrize("shape,seed", [((6, 7), 21), ((7, 7), 21)], ids=["6x7-32bit", "7x7-64bit"])
def test_split_large_four_classes(isg, cuda, shape, seed):
    """Tori with couplings in {-2, -1, 1, 2} (four classes: the general field evaluation): on the
    6x7 torus the counts fit 32 bits, on the 7x7 torus (N = 49) they need the 64-bit accumulators.
    Every bin against the oracle's frontier programme."""
    lat = w.with_random_couplings(w.square(*shape, True), w.SplitMix64(seed), (-2, -1, 1, 2))
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = isg.isg_enumerate_split(gh)
    assert int(g.sum()) == 2 ** lat.n
    assert np.array_equal(g, oracle.g_frontier(lat.n, lat.edges, 16))


def test_split_torus_8x8(isg, cuda):
    """The 8x8 torus, N = 64: all 2^64 configurations (the largest graph the library takes). Every
    one of the 129 x 65 bins equals the oracle's frontier programme conditioned on one row (2^8 rest
    programmes of 56 spins, all host cores); every energy count equals Kaufman's exact count; and
    the facts that hold at any size: sum 2^64 (in Python integers), every column C(64, m), the
    M -> -M and bipartite E -> -E symmetries, two ground states, ln Z against Kaufman's closed form."""
    lat = w.square(8, 8, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = isg.isg_enumerate_split(gh)
    assert sum(int(v) for v in g.ravel()) == 2 ** 64
    assert all(sum(int(v) for v in g[:, m]) == math.comb(64, m) for m in range(65))
    assert np.array_equal(g, g[:, ::-1])
    assert np.array_equal(g.sum(axis=1), g.sum(axis=1)[::-1])
    assert int(g[0, 0]) == 1 and int(g[0, 64]) == 1 and not g[0, 1:64].any()
    assert [int(x) for x in g.sum(axis=1)] == kaufman_energy_counts(8, 8)
    T = np.array([1.5, 2.269, 3.0, 5.0])
    lz = isg.isg_thermo(g, gh, T, [0.0], isg.ISG_FP64)[0][:, 0]
    for t, l in zip(T, lz):
        assert abs(l - kaufman_logz(8, 8, t)) <= 1e-12 * abs(l)
    ref = oracle.g_frontier_cut(lat.n, lat.edges, mask(range(8)), max_active=18, threads=THREADS)
    assert np.array_equal(g, ref)


def test_specific_heat_peak_8x8_kaufman(isg, cuda):
    """The specific-heat maximum of the 8x8 torus (N = 64) from its exact table (split-and-
    convolve, then isg_specific_heat_peak in FP64) against the maximum of Kaufman's closed-form
    C(T), and the value of C there."""
    from closed_forms import kaufman_C, kaufman_C_peak
    lat = w.square(8, 8, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = isg.isg_enumerate_split(gh)
    t_gpu, c_gpu = isg.isg_specific_heat_peak(g, gh, 0.0, 1.5, 3.5, isg.ISG_FP64)
    t_k = kaufman_C_peak(8, 8, kaufman_C_peak(8, 8, t_gpu))
    assert abs(t_gpu - t_k) <= 1e-5 * t_k
    assert abs(c_gpu - kaufman_C(8, 8, t_gpu)) <= 1e-5 * c_gpu


def test_split_batch_ea_ensemble(isg, cuda):
    """isg_enumerate_split_batch over EA +-J instances of all four shapes (shared planning per
    shape), into device tensors and into host tables: every table equals the batched full
    enumeration's and the oracle's frontier programme."""
    import torch
    from relabel import frontier_table
    lats = w.ea_instances()[:96]
    hs = [isg.isg_graph_create(l.n, l.edges) for l in lats]
    dev = [torch.zeros(isg.table_shape(h), dtype=torch.int64, device=cuda) for h in hs]
    isg.isg_enumerate_split_batch(hs, dev)
    host = isg.isg_enumerate_split_batch(hs)
    torch.cuda.synchronize()
    ref = isg.isg_enumerate_batch(hs)
    for k, (l, d, h, r) in enumerate(zip(lats, dev, host, ref)):
        assert np.array_equal(d.cpu().numpy(), r) and np.array_equal(h, r), l.name
        assert np.array_equal(h, frontier_table(l)), l.name


def test_prepared_batch_with_split(isg, cuda):
    """A prepared batch with options.split over EA instances of all shapes (the larger ones served
    by split launches inside the captured graph, the others by the tile queue), replayed twice:
    every table equals the plain batch's, and the self-check status is clean."""
    import torch
    lats = w.ea_instances()[:64]
    hs = [isg.isg_graph_create(l.n, l.edges) for l in lats]
    ref = isg.Batch(hs)
    ref.run()
    got = isg.Batch(hs, split=1)
    for _ in range(2):
        got.run()
    torch.cuda.synchronize()
    got.status()
    for k, l in enumerate(lats):
        assert torch.equal(got.table(k), ref.table(k)), l.name
    assert sum(l.n == 30 for l in lats) >= 8            # some instances really take the split path

"""GPU parity of isg_enumerate against the CPU oracle: bit-exact int64 tables.

Small graphs are compared in full; the full-size workloads (6x6 torus, 3x3x4 cubic torus,
N = 36) run in the same launch configuration as the benchmark and are checked bin for bin against
the oracle's frontier programme (on the cubic torus conditioned on one layer of spins), against
the oracle on sampled shards, and against invariants that hold at any size (sum 2^N, binomial
columns, the M mirror, ground states)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1110_2561_gb300 import workloads as w

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


def gpu_table(isg, cuda, lat, **opt):
    import torch
    g = isg.isg_graph_create(lat.n, lat.edges)
    out = torch.zeros(isg.table_shape(g), dtype=torch.int64, device=cuda)
    isg.isg_enumerate(g, out, **opt)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check_invariants(g: np.ndarray, n: int):
    assert int(g.sum()) == 2 ** n
    for m in range(n + 1):
        assert int(g[:, m].sum()) == math.comb(n, m)
    assert np.array_equal(g, g[:, ::-1])
    assert (g >= 0).all()


SMALL = [w.square(4, 4, False), w.square(4, 4, True), w.square(3, 5, True), w.triangular(4, 4, True),
         w.cubic(2, 2, 4, True), w.ring(13), w.ring(5), w.square(1, 2, False),
         w.with_random_couplings(w.square(4, 5, True), w.SplitMix64(1), (-1, 1)),
         w.with_random_couplings(w.triangular(4, 5, False), w.SplitMix64(2), (-2, -1, 1, 2)),
         w.random_graph(18, 40, w.SplitMix64(3)), w.random_graph(16, 90, w.SplitMix64(4)),
         w.random_graph(15, 15, w.SplitMix64(5), couplings=(-7, 3, 5, 11, 13, 100)),
         w.induced_lattice("cubic", 19, True, w.SplitMix64(6)), w.lattice("square", (1, 14), True)]


@pytest.mark.parametrize("lat", SMALL, ids=lambda l: l.name)
def test_small_graphs_device_and_host(isg, cuda, lat):
    ref = oracle.g_masks(lat.n, lat.edges)
    assert np.array_equal(gpu_table(isg, cuda, lat), ref)
    g = isg.isg_graph_create(lat.n, lat.edges)
    assert np.array_equal(isg.isg_enumerate(g), ref)          # host buffer: synchronous, self-checked


def test_single_and_isolated_spins(isg, cuda):
    for n in (1, 2, 3, 7):
        g = isg.isg_graph_create(n, np.zeros((0, 3), np.int64))
        ref = oracle.g_edges(n, np.zeros((0, 3), np.int64))
        assert np.array_equal(isg.isg_enumerate(g), ref)
    lat = w.Lattice(20, np.array([(0, 1, 1), (5, 9, -2), (17, 3, 1)], dtype=np.int64))
    assert np.array_equal(gpu_table(isg, cuda, lat), oracle.g_masks(lat.n, lat.edges))


def test_degenerate_graphs_in_lane_tables(isg, cuda):
    """Warp-task plans (lane tables by default) on graphs with a single energy row (no bonds at
    all), with bonds whose duplicate couplings cancel to nothing, and a ring with a cancelled chord:
    the oracle's tables."""
    cases = [w.Lattice(20, np.zeros((0, 3), np.int64), "free20"),
             w.Lattice(16, np.array([(0, 1, 2), (1, 0, -2), (2, 3, 1), (4, 5, -1), (5, 4, 1)], np.int64), "cancel16"),
             w.Lattice(24, np.array([(i, (i + 1) % 24, 1) for i in range(24)] + [(0, 12, 3), (12, 0, -3)], np.int64),
                       "ring24-cancel")]
    for lat in cases:
        g = isg.isg_graph_create(lat.n, lat.edges)
        assert isg.isg_debug_plan(g)["lane_tables"] == 10
        assert np.array_equal(gpu_table(isg, cuda, lat), oracle.g_edges(lat.n, lat.edges)), lat.name
    isg.isg_device_status()


def test_table1_on_gpu(isg, cuda, table1_triples):
    """Table 1 of the paper from the GPU: the 4x4 periodic ferromagnet, all 80 cells."""
    lat = w.square(4, 4, True)
    g = gpu_table(isg, cuda, lat)
    e_min = -32
    got = {(e_min + 2 * int(e), -16 + 2 * int(m)): int(g[e, m]) for e, m in zip(*np.nonzero(g))}
    assert got == {(E, M): nc for nc, M, E in table1_triples}


PLANS = [dict(inner_bits=6), dict(low_bits=1, inner_bits=4), dict(low_bits=4, inner_bits=9), dict(low_bits=5, inner_bits=12),
         dict(block_threads=64, copies=1), dict(block_threads=1024, copies=16), dict(block_threads=256, copies=3),
         dict(flush_tasks=1), dict(ctas_per_sm=1, flush_tasks=1, block_threads=96, copies=2), dict(low_bits=2, inner_bits=2),
         dict(warp_aggregate=1), dict(bin_stride=64), dict(bin_stride=33, warp_aggregate=1, copies=1),
         dict(symmetry=1), dict(symmetry=1, low_bits=3, inner_bits=6, block_threads=128),
         dict(lane_model=1), dict(lane_model=1, symmetry=1), dict(lane_model=1, inner_bits=9, stride_residue=19),
         dict(lane_model=2), dict(lane_model=2, block_threads=1024, copies=16), dict(lane_model=3),
         dict(lane_model=4, inner_bits=6, low_bits=3), dict(lane_model=4, symmetry=1, flush_tasks=1),
         dict(lane_model=4, block_threads=64)]


@pytest.mark.parametrize("kw", PLANS, ids=lambda k: ",".join(f"{a}={b}" for a, b in k.items()))
def test_plan_invariance(isg, cuda, kw):
    """Every planner choice gives the same table (forced tiny flush intervals included)."""
    lat = w.with_random_couplings(w.triangular(4, 5, True), w.SplitMix64(8), (-2, -1, 1, 2))
    ref = oracle.g_masks(lat.n, lat.edges, threads=THREADS)
    assert np.array_equal(gpu_table(isg, cuda, lat, **kw), ref)


@pytest.mark.parametrize("kw", [dict(copies=2), dict(copies=3, block_threads=96, flush_tasks=1), dict(bin_stride=96),
                                dict(symmetry=1, copies=2), dict(shard_bits=3, shard_lo=2, shard_hi=7, inner_bits=8)],
                         ids=lambda k: ",".join(f"{a}={b}" for a, b in k.items()))
def test_lane_tables_forced_shapes(isg, cuda, kw):
    """Lane tables (ten sub-tables per copy) with several copies per CTA (warps sharing them), a
    wider row stride, a flush after every task, symmetry halving and a shard range, on a +-1 torus
    of 20 spins: the oracle's table (or shard range) bin for bin."""
    lat = w.with_random_couplings(w.square(4, 5, True), w.SplitMix64(21), (-1, 1))
    g = isg.isg_graph_create(lat.n, lat.edges)
    assert isg.isg_debug_plan(g, lane_model=4, **kw)["lane_tables"] == 10
    if "shard_bits" in kw:
        k = kw["shard_bits"]
        ref = oracle.g_masks(lat.n, lat.edges, kw["shard_lo"] << (lat.n - k), kw["shard_hi"] << (lat.n - k))
    else:
        ref = oracle.g_masks(lat.n, lat.edges)
    assert np.array_equal(gpu_table(isg, cuda, lat, lane_model=4, **kw), ref)
    isg.isg_device_status()


def test_symmetry_host_device_accumulate(isg, cuda):
    """Symmetry halving (spin N-1 up, then the M mirror) gives the oracle's table on the host, on
    the device, added into a table, on +-J couplings, and on the 6x6 torus at full size."""
    import torch
    lat = w.with_random_couplings(w.cubic(2, 3, 3, True), w.SplitMix64(13), (-1, 1))
    ref = oracle.g_masks(lat.n, lat.edges, threads=THREADS)
    g = isg.isg_graph_create(lat.n, lat.edges)
    assert np.array_equal(isg.isg_enumerate(g, symmetry=1), ref)
    out = torch.zeros(isg.table_shape(g), dtype=torch.int64, device=cuda)
    isg.isg_enumerate(g, out, symmetry=1)
    isg.isg_enumerate(g, out, symmetry=1, accumulate=1)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), 2 * ref)
    t6 = w.square(6, 6, True)
    gt = isg.isg_graph_create(t6.n, t6.edges)
    assert np.array_equal(isg.isg_enumerate(gt, symmetry=1), oracle.g_frontier(t6.n, t6.edges, max_active=16))


def test_shards_and_accumulate(isg, cuda):
    import torch
    lat = w.with_random_couplings(w.square(4, 5, True), w.SplitMix64(9), (-1, 1))
    g = isg.isg_graph_create(lat.n, lat.edges)
    out = torch.zeros(isg.table_shape(g), dtype=torch.int64, device=cuda)
    for lo, hi in [(0, 3), (3, 4), (4, 16)]:
        isg.isg_enumerate(g, out, shard_bits=4, shard_lo=lo, shard_hi=hi, accumulate=1)
        torch.cuda.synchronize()
        part = isg.isg_enumerate(g, shard_bits=4, shard_lo=lo, shard_hi=hi)
        assert np.array_equal(part, oracle.g_masks(lat.n, lat.edges, lo << 16, hi << 16))
    assert np.array_equal(out.cpu().numpy(), oracle.g_masks(lat.n, lat.edges))


def test_rejections(isg, cuda):
    g = isg.isg_graph_create(41, w.random_graph(41, 60, w.SplitMix64(1)).edges)
    with pytest.raises(isg.IsgError) as ei:
        isg.isg_enumerate(g)
    assert ei.value.status == 2
    big = w.ring(30, J=1 << 20)           # 2^20-sized couplings: far too many energy bins for shared memory
    with pytest.raises(isg.IsgError) as ei:
        isg.isg_enumerate(isg.isg_graph_create(big.n, big.edges))
    assert ei.value.status == 2
    odd = w.random_graph(15, 15, w.SplitMix64(5), couplings=(-7, 3, 5, 11, 13, 1000))   # 81488 bins
    with pytest.raises(isg.IsgError) as ei:
        isg.isg_enumerate(isg.isg_graph_create(odd.n, odd.edges))
    assert ei.value.status == 2


# ----------------------------------------------------------------------------------- full size
def test_torus_6x6_full_against_frontier_oracle(isg, cuda):
    """6x6 periodic ferromagnet, N = 36, 2^36 configurations, default (benchmark) plan: every one
    of the table's bins equals the oracle's exact frontier programme."""
    lat = w.square(6, 6, True)
    got = gpu_table(isg, cuda, lat)
    ref = oracle.g_frontier(lat.n, lat.edges, max_active=16)
    assert np.array_equal(got, ref)
    check_invariants(got, 36)


def test_torus_6x6_sampled_shards(isg, cuda):
    """Shards of the 6x6 torus in the benchmark's inner-bit split, against the popcount oracle."""
    lat = w.square(6, 6, True)
    g = isg.isg_graph_create(lat.n, lat.edges)
    q = isg.isg_debug_plan(g)["q"]
    for shard in (0, 777, 4095):
        got = isg.isg_enumerate(g, shard_bits=12, shard_lo=shard, shard_hi=shard + 1, inner_bits=q)
        ref = oracle.g_masks(lat.n, lat.edges, shard << 24, (shard + 1) << 24, threads=THREADS)
        assert np.array_equal(got, ref)


def test_cubic_3x3x4_full_invariants_and_shards(isg, cuda):
    """3x3x4 simple cubic torus (Z = 6, 108 bonds), N = 36: full table by invariants and ground
    states, and sampled shards in the benchmark's split against the oracle bit for bit."""
    lat = w.cubic(3, 3, 4, True)
    full = gpu_table(isg, cuda, lat)
    check_invariants(full, 36)
    assert full[0, 0] == 1 and full[0, 36] == 1 and full[0].sum() == 2
    g = isg.isg_graph_create(lat.n, lat.edges)
    q = isg.isg_debug_plan(g)["q"]
    rng = w.SplitMix64(4)
    for shard in sorted({rng.below(4096) for _ in range(6)}):
        got = isg.isg_enumerate(g, shard_bits=12, shard_lo=shard, shard_hi=shard + 1, inner_bits=q)
        ref = oracle.g_masks(lat.n, lat.edges, shard << 24, (shard + 1) << 24, threads=THREADS)
        assert np.array_equal(got, ref)


def test_cubic_3x3x4_full_against_layer_conditioned_oracle(isg, cuda):
    """3x3x4 simple cubic torus, N = 36, in the benchmark's autotuned plan, the default plan (lane
    tables), the quick lane search's and the index order's plans, and by split-and-convolve: every
    bin of every table equals the oracle's frontier programme conditioned on one z layer (2^9 configurations of that
    layer, each with the other 27 spins by the frontier; sites renumbered layer by layer)."""
    import torch
    from relabel import layer_cut
    lat = w.cubic(3, 3, 4, True)
    r, cut = layer_cut(lat)
    assert bin(cut).count("1") == 9
    got = gpu_table(isg, cuda, lat, autotune=1)
    default = gpu_table(isg, cuda, lat)                     # lane tables
    quick = gpu_table(isg, cuda, lat, lane_model=3)         # the quick lane search
    index = gpu_table(isg, cuda, lat, lane_model=2)
    g = isg.isg_graph_create(lat.n, lat.edges)
    assert isg.isg_debug_plan(g)["lane_tables"] == 10
    split = torch.zeros(isg.table_shape(g), dtype=torch.int64, device=cuda)
    isg.isg_enumerate_split(g, split)
    ref = oracle.g_frontier_cut(r.n, r.edges, cut, max_active=20, threads=THREADS)
    assert np.array_equal(got, ref)
    assert np.array_equal(default, ref)
    assert np.array_equal(quick, ref)
    assert np.array_equal(index, ref)
    assert np.array_equal(split.cpu().numpy(), ref)
    isg.isg_device_status()


@pytest.mark.slow
def test_cubic_3x3x4_full_against_popcount_oracle(isg, cuda):
    """3x3x4 simple cubic torus, N = 36, in the benchmark's autotuned plan, the quick lane search's
    plan, the index order's plan, and by split-and-convolve: every bin of every table
    equals the popcount oracle's table over all 2^36 configurations (O1 on
    all host cores; minutes of CPU time): the plainest definition, beside the layer-conditioned
    frontier programme of the test above."""
    import torch
    lat = w.cubic(3, 3, 4, True)
    got = gpu_table(isg, cuda, lat, autotune=1)
    default = gpu_table(isg, cuda, lat, lane_model=3)       # the quick lane search's plan
    index = gpu_table(isg, cuda, lat, lane_model=2)         # the index order's
    g = isg.isg_graph_create(lat.n, lat.edges)
    split = torch.zeros(isg.table_shape(g), dtype=torch.int64, device=cuda)
    isg.isg_enumerate_split(g, split)
    ref = oracle.g_masks(lat.n, lat.edges, threads=THREADS)
    assert np.array_equal(got, ref)
    assert np.array_equal(default, ref)
    assert np.array_equal(index, ref)
    assert np.array_equal(split.cpu().numpy(), ref)
    isg.isg_device_status()


def test_largest_default_size_n40(isg, cuda):
    """N = 40 (the default max_spins): the 5x8 torus with four coupling values, 2^40
    configurations; every bin against the oracle's frontier programme conditioned on one row of
    five spins (sites renumbered along the short side), and the invariants at full size."""
    from relabel import layer_cut
    lat = w.with_random_couplings(w.square(5, 8, True), w.SplitMix64(40), (-2, -1, 1, 2))
    got = gpu_table(isg, cuda, lat)
    check_invariants(got, 40)
    r, cut = layer_cut(lat)
    assert np.array_equal(got, oracle.g_frontier_cut(r.n, r.edges, cut, max_active=20, threads=THREADS))


def test_torus_5x8_n40_lane_tables(isg, cuda):
    """N = 40 ferromagnetic 5x8 torus (2^40 configurations) in the default plan, lane tables: every
    bin against the oracle's frontier programme conditioned on one row, every energy count exactly
    as Kaufman's closed form gives it, and the invariants."""
    from closed_forms import kaufman_energy_counts
    from relabel import layer_cut
    lat = w.square(5, 8, True)
    g = isg.isg_graph_create(lat.n, lat.edges)
    assert isg.isg_debug_plan(g)["lane_tables"] == 10
    got = gpu_table(isg, cuda, lat)
    check_invariants(got, 40)
    assert [int(x) for x in got.sum(axis=1)] == kaufman_energy_counts(5, 8)
    r, cut = layer_cut(lat)
    assert np.array_equal(got, oracle.g_frontier_cut(r.n, r.edges, cut, max_active=20, threads=THREADS))
    isg.isg_device_status()


def test_lane_tables_odd_energy_stride(isg, cuda):
    """Graphs whose energy stride G has an odd factor (J = 3 rings and a J = +-3 triangular torus:
    G = 12), where the lane tables' row stride must make 8 R / G whole: the oracle's tables, with
    a clean self-check."""
    cases = [w.Lattice(17, np.array([(i, (i + 1) % 17, 3) for i in range(17)], np.int64), "ring17-J3"),
             w.Lattice(23, np.array([(i, (i + 1) % 23, 3) for i in range(23)], np.int64), "ring23-J3"),
             w.with_random_couplings(w.triangular(4, 5, True), w.SplitMix64(9), (-3, 3))]
    for lat in cases:
        g = isg.isg_graph_create(lat.n, lat.edges)
        p = isg.isg_debug_plan(g)
        assert p["lane_tables"] == 10 and p["G"] == 12 and p["stride"] % 96 == 0, lat.name
        assert np.array_equal(gpu_table(isg, cuda, lat), oracle.g_masks(lat.n, lat.edges, threads=THREADS)), lat.name
        assert np.array_equal(isg.isg_enumerate(g), oracle.g_masks(lat.n, lat.edges, threads=THREADS)), lat.name
    isg.isg_device_status()


def test_packed_lane_tables_across_sizes(isg, cuda):
    """Packed lane tables (the ten sub-tables side by side in each row, in an order searched per
    residue of N - 5 mod 32) on +-1/+-2 graphs of 16 to 26 spins, one packed order each: the
    oracle's tables."""
    rng = w.SplitMix64(44)
    seen = set()
    for n in range(16, 27):
        lat = w.random_graph(n, 2 * n, rng, couplings=(-2, -1, 1, 2))
        g = isg.isg_graph_create(lat.n, lat.edges)
        L = isg.isg_debug_lane_layout(g)
        assert L["n_sub"] == 10 and L["packed"], lat.name
        seen.add((n - 5) % 32)
        assert np.array_equal(gpu_table(isg, cuda, lat), oracle.g_masks(lat.n, lat.edges, threads=THREADS)), lat.name
    assert len(seen) == 11
    isg.isg_device_status()


@pytest.mark.parametrize("kind", ["square", "triangular"])
def test_packed_lane_tables_n36_two_coupling_classes(isg, cuda, kind):
    """36-spin tori with J in {-2, -1, 1, 2} (114 and 163 energy rows), whose lane tables fit
    shared memory only packed: in the default plan, every bin against the oracle's frontier
    programme (sites renumbered along the short side) and the invariants."""
    from relabel import frontier_table
    lat = w.with_random_couplings(getattr(w, kind)(6, 6, True), w.SplitMix64(3), (-2, -1, 1, 2))
    g = isg.isg_graph_create(lat.n, lat.edges)
    assert isg.isg_debug_plan(g)["lane_tables"] == 10 and isg.isg_debug_lane_layout(g)["packed"]
    got = gpu_table(isg, cuda, lat)
    assert int(got.sum()) == 2 ** 36
    for m in range(37):
        assert int(got[:, m].sum()) == math.comb(36, m)
    assert np.array_equal(got, got[:, ::-1])
    assert np.array_equal(got, frontier_table(lat, THREADS))
    isg.isg_device_status()


def test_autotune_torus_6x6(isg, cuda):
    """The autotuner's choice (cached per graph; the lane spins of the bank-conflict model or of the
    index order, or lane tables, whichever timed fastest) gives the same table as the oracle's frontier programme,
    and so does the model's plan forced; a second isg_autotune call returns the cached fields."""
    import torch
    lat = w.square(6, 6, True)
    g = isg.isg_graph_create(lat.n, lat.edges)
    t1 = isg.isg_autotune(g)
    t2 = isg.isg_autotune(g)
    assert t1 == t2 and t1["block_threads"] > 0 and t1["lane_model"] in (1, 2, 4)
    assert t1["stride_residue"] > 0 or t1["lane_model"] in (1, 4)   # the model's stride; lane tables' multiple of 32
    out = torch.zeros(isg.table_shape(g), dtype=torch.int64, device=cuda)
    isg.isg_enumerate(g, out, autotune=1)
    forced = torch.zeros_like(out)
    isg.isg_enumerate(g, forced, lane_model=1)
    torch.cuda.synchronize()
    ref = oracle.g_frontier(lat.n, lat.edges, max_active=16)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert np.array_equal(forced.cpu().numpy(), ref)
    isg.isg_device_status()


def test_checkpoint_and_resume(isg, cuda, tmp_path):
    """A long enumeration is resumable: shards [0, 5) of 2^4 into a host table, saved to disk,
    reloaded, then shards [5, 16) added with accumulate, equal the full oracle table."""
    lat = w.with_random_couplings(w.triangular(4, 5, True), w.SplitMix64(17), (-2, -1, 1, 2))
    g = isg.isg_graph_create(lat.n, lat.edges)
    part = np.zeros(isg.table_shape(g), dtype=np.int64)
    isg.isg_enumerate(g, part, shard_bits=4, shard_lo=0, shard_hi=5, accumulate=1)
    np.save(tmp_path / "checkpoint.npy", part)
    resumed = np.load(tmp_path / "checkpoint.npy")
    isg.isg_enumerate(g, resumed, shard_bits=4, shard_lo=5, shard_hi=16, accumulate=1)
    assert np.array_equal(resumed, oracle.g_masks(lat.n, lat.edges, threads=THREADS))


def test_device_status_clean_after_device_output_calls(isg, cuda):
    """Device-output calls record their kernels' self-check in the device's word: after a run of
    them (the Gray walk with and without symmetry, split-and-convolve, the no-allocation call) the
    word is clear, isg_device_status reports it so, and the tables equal the oracle's."""
    import torch
    isg.isg_device_status(clear=True)
    lat = w.with_random_couplings(w.triangular(4, 6, True), w.SplitMix64(31), (-2, -1, 1, 2))
    gh = isg.isg_graph_create(lat.n, lat.edges)
    ref = oracle.g_masks(lat.n, lat.edges, threads=THREADS)
    outs = [torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=cuda) for _ in range(4)]
    isg.isg_enumerate(gh, outs[0])
    isg.isg_enumerate(gh, outs[1], symmetry=1)
    isg.isg_enumerate_split(gh, outs[2], boundary=0x3F)           # the first row: one component of 18
    isg.isg_enumerate_noalloc(gh, outs[3])
    isg.isg_device_status()
    for o in outs:
        assert np.array_equal(o.cpu().numpy(), ref)
    isg.isg_device_status(clear=False)


def test_lane_model_with_symmetry_and_rank_shares_torus_6x6(isg, cuda):
    """Lane-model plans where the top spin (symmetry halving) or the top shard bits (rank shares)
    are fixed, so the lane spins come from the remaining free spins: the 6x6 torus's full table
    from the model's plan with symmetry, and from two autotuned rank shares summed, equals the
    oracle's frontier programme."""
    import torch
    lat = w.square(6, 6, True)
    g = isg.isg_graph_create(lat.n, lat.edges)
    ref = oracle.g_frontier(lat.n, lat.edges, max_active=16)
    sym = torch.zeros(isg.table_shape(g), dtype=torch.int64, device=cuda)
    isg.isg_enumerate(g, sym, lane_model=1, symmetry=1)
    ranks = torch.zeros_like(sym)
    for r in range(2):
        isg.isg_enumerate_rank(g, r, 2, ranks, autotune=1, accumulate=1)
    torch.cuda.synchronize()
    assert np.array_equal(sym.cpu().numpy(), ref)
    assert np.array_equal(ranks.cpu().numpy(), ref)
    assert isg.isg_debug_plan(g, lane_model=1, symmetry=0, shard_bits=1, shard_lo=1, shard_hi=2)["lane_model"] == 1
    isg.isg_device_status()


def test_concurrent_host_buffer_calls(isg, cuda):
    """Host-buffer calls from several threads at once, each on its own stream (the library releases
    the interpreter during a call): their pinned staging buffers come from one shared pool, and every
    table and every thermodynamic output equals the single-threaded result."""
    import threading
    import torch
    lats = [w.square(4, 5, True), w.triangular(4, 4, True), w.cubic(2, 2, 4, True),
            w.with_random_couplings(w.square(4, 4, True), w.SplitMix64(5), (-2, -1, 1, 2))]
    graphs = [isg.isg_graph_create(l.n, l.edges) for l in lats]
    refs = [oracle.g_masks(l.n, l.edges) for l in lats]
    T, h = np.linspace(0.5, 5, 40), np.array([0.0, 0.5])
    thermo_refs = [isg.isg_thermo(r, g, T, h, isg.ISG_FP64) for r, g in zip(refs, graphs)]
    errors = []

    def worker(k):
        st = torch.cuda.Stream()
        try:
            for rep in range(6):
                i = (k + rep) % len(lats)
                tab = isg.isg_enumerate(graphs[i], None, st)
                if not np.array_equal(tab, refs[i]):
                    errors.append(("table", k, i))
                out = isg.isg_thermo(tab, graphs[i], T, h, isg.ISG_FP64, st)
                if not all(np.array_equal(a, b) for a, b in zip(out, thermo_refs[i])):
                    errors.append(("thermo", k, i))
        except Exception as e:                       # reported below, not lost in the thread
            errors.append(("raised", k, repr(e)))

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(6)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors

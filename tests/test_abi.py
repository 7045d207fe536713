"""The C ABI on the CPU: the library loads, exports every declared entry point, validates its
inputs, and its kernels' per-thread walk (run on the host by isg_debug_emulate) reproduces the
oracle bit for bit over many plans. No GPU is used."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_1110_2561_gb300 import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"ISG_API\s+[\w\s\*]+?\b(isg_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(isg):
    names = declared_functions()
    assert "isg_enumerate" in names and "isg_thermo" in names and "isg_graph_create" in names
    out = subprocess.run(["nm", "-D", "--defined-only", isg.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (isg_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    lib = isg.lib()
    for n in names:
        assert getattr(lib, n) is not None


def test_version(isg):
    assert "sm_103a" in isg.isg_version()


@pytest.mark.parametrize("n,edges,msg", [
    (0, [], "n_spins"), (65, [], "n_spins"), (3, [(0, 3, 1)], "out of range"), (3, [(1, 1, 1)], "self loop"),
    (3, [(0, 1, 0)], "J = 0"), (3, [(0, 1, (1 << 20) + 1)], "2^20"), (3, [(0, 1, 1 << 20), (0, 1, 1 << 20)], "2^20")])
def test_graph_validation(isg, n, edges, msg):
    with pytest.raises(isg.IsgError) as ei:
        isg.isg_graph_create(n, edges)
    assert ei.value.status == 1 and msg in str(ei.value)


def test_bins_geometry(isg):
    for lat in [w.square(4, 4, True), w.square(4, 4, False), w.random_graph(9, 20, w.SplitMix64(2))]:
        g = isg.isg_graph_create(lat.n, lat.edges)
        e_min, n_e, n_m = oracle.bins(lat.n, lat.edges)
        assert isg.isg_graph_bins(g) == (e_min, 2, n_e, -lat.n, n_m)


def test_duplicate_bonds_summed(isg):
    g = isg.isg_graph_create(3, [(0, 1, 1), (1, 0, 1), (1, 2, 3), (2, 1, -3)])
    assert isg.isg_graph_size(g) == (3, 1)
    assert isg.isg_graph_bins(g)[:3] == (-2, 2, 3)


def test_options_validation(isg):
    g = isg.isg_graph_create(16, w.square(4, 4, True).edges)
    for bad in [dict(shard_bits=17), dict(shard_bits=2, shard_lo=3, shard_hi=2), dict(shard_bits=2, shard_lo=0, shard_hi=5),
                dict(low_bits=8), dict(inner_bits=12), dict(block_threads=48), dict(copies=99)]:
        with pytest.raises(isg.IsgError) as ei:
            isg.isg_debug_plan(g, **bad)
        assert ei.value.status == 1, bad
    with pytest.raises(isg.IsgError) as ei:
        isg.isg_debug_plan(g, max_spins=15)
    assert ei.value.status == 2


def test_plan_torus_6x6(isg):
    """The 6x6 torus plan: energy stride 4 compacts 73 energy bins to 37; the low block is an
    independent set of 7 spins; the inner walk and task count cover 2^36 configurations."""
    g = isg.isg_graph_create(36, w.square(6, 6, True).edges)
    p = isg.isg_debug_plan(g)
    assert p["small"] == 0 and p["G"] == 4 and p["n_e_compact"] == 37 and p["b"] == 7
    assert p["tasks"] * 32 << p["q"] == 1 << 36
    assert p["flush_rounds"] >= 1


EMU_GRAPHS = [w.square(4, 4, True), w.square(4, 4, False), w.square(3, 5, True), w.triangular(4, 4, True),
              w.cubic(2, 2, 4, True), w.ring(13),
              w.with_random_couplings(w.square(4, 4, True), w.SplitMix64(1), (-1, 1)),
              w.with_random_couplings(w.triangular(3, 5, False), w.SplitMix64(2), (-2, -1, 1, 2)),
              w.random_graph(14, 30, w.SplitMix64(3)), w.random_graph(13, 60, w.SplitMix64(4)),
              w.random_graph(12, 12, w.SplitMix64(5), couplings=(-7, 3, 5, 11, 13, 1000)),
              w.induced_lattice("cubic", 17, True, w.SplitMix64(6)), w.lattice("square", (1, 12), True)]
EMU_PLANS = [{}, dict(inner_bits=6), dict(low_bits=1, inner_bits=3), dict(low_bits=3, inner_bits=5),
             dict(low_bits=2, inner_bits=2), dict(shard_bits=2, shard_lo=1, shard_hi=3), dict(shard_bits=4, shard_lo=9, shard_hi=10),
             dict(bin_stride=64), dict(bin_stride=100, low_bits=4), dict(low_bits=7, inner_bits=8),
             dict(symmetry=1), dict(symmetry=1, low_bits=3, inner_bits=4),
             dict(lane_model=1), dict(lane_model=1, inner_bits=6), dict(lane_model=1, low_bits=3, inner_bits=5),
             dict(lane_model=1, shard_bits=2, shard_lo=1, shard_hi=3), dict(lane_model=1, symmetry=1),
             dict(lane_model=1, stride_residue=13), dict(lane_model=2, autotune=0), dict(lane_model=3)]


@pytest.mark.parametrize("lat", EMU_GRAPHS, ids=lambda l: l.name)
def test_emulated_walk_matches_oracle(isg, lat):
    """Every plan of the GPU walk, run on the host with bounds-checked counters, equals the oracle."""
    g = isg.isg_graph_create(lat.n, lat.edges)
    full = oracle.g_masks(lat.n, lat.edges)
    for kw in EMU_PLANS:
        if "shard_bits" in kw:
            k = kw["shard_bits"]
            ref = oracle.g_masks(lat.n, lat.edges, kw["shard_lo"] << (lat.n - k), kw["shard_hi"] << (lat.n - k))
        else:
            ref = full
        try:
            got = isg.isg_debug_emulate(g, **kw)
        except isg.IsgError as e:       # a forced plan this graph cannot take (e.g. no independent set)
            assert e.status in (1, 2), (kw, e)
            continue
        assert np.array_equal(got, ref), kw


def test_symmetry_rejects_shards(isg):
    g = isg.isg_graph_create(16, w.square(4, 4, True).edges)
    with pytest.raises(isg.IsgError) as ei:
        isg.isg_debug_emulate(g, symmetry=1, shard_bits=1, shard_hi=1)
    assert ei.value.status == 1


def test_emulated_accumulate(isg):
    lat = w.square(3, 4, True)
    g = isg.isg_graph_create(lat.n, lat.edges)
    ref = oracle.g_masks(lat.n, lat.edges)
    a = isg.isg_debug_emulate(g, shard_bits=1, shard_lo=0, shard_hi=1)
    b = isg.isg_debug_emulate(g, shard_bits=1, shard_lo=1, shard_hi=2)
    assert np.array_equal(a + b, ref)


def test_smoke_calls_are_valid_plans(isg):
    """The calls __graft_entry__.smoke() makes on the GPU pass the host-side planning: the 4x4 free
    lattice goes through the main Gray-walk kernel (not the small-graph kernel), and the split
    call's boundary (the second row) is admissible."""
    from paper_1110_2561_gb300 import workloads as w
    lat = w.square(4, 4, False)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    assert isg.isg_debug_plan(gh)["small"] == 0
    p = isg.isg_split_plan(gh, 0xF0)
    assert p["boundary"] == 0xF0 and p["components"] == 2


def test_self_check_word_reported_through_the_status_path(isg):
    """The kernels' self-check (each walk's tracked last bin against its recomputation from
    scratch) on the host emulation, with a mistake planted in the program: a wrong field constant
    on the spin at the top inner position, which flips once per walk, must set bit 0 of the word,
    and the library must report that word as ISG_ERR_INTERNAL with the message that the
    host-output calls and isg_device_status give for it. Without a planted mistake the same walk
    reports nothing and gives the oracle's table."""
    lat = w.with_random_couplings(w.square(4, 5, True), w.SplitMix64(1), (-1, 1))
    g = isg.isg_graph_create(lat.n, lat.edges)
    opt = dict(low_bits=3, inner_bits=9)
    plan = isg.isg_debug_plan(g, **opt)
    top = plan["q"] - 1
    st, word, msg, tab = isg.isg_debug_emulate_planted(g, top, 0, **opt)
    assert (st, word, msg) == (0, 0, "")
    assert np.array_equal(tab, oracle.g_masks(lat.n, lat.edges))
    for delta in (plan["G"], -plan["G"], 3 * plan["G"]):
        st, word, msg, _ = isg.isg_debug_emulate_planted(g, top, delta, **opt)
        assert st == 8 and word & 1, delta
        assert "self-check failed" in msg and "tracked bin differed from its recomputation" in msg
    # the same report through isg_debug_emulate's own path (a graph whose walk is consistent)
    with pytest.raises(isg.IsgError) as ei:
        isg.isg_debug_emulate(isg.isg_graph_create(lat.n, lat.edges), shard_bits=lat.n + 1)
    assert ei.value.status == 1


def test_lane_model_plans(isg):
    """The bank-conflict model's lane spins (options.lane_model = 1): five spins outside the low
    block, a stride in [N + 1, N + 32], and a modelled cost no worse than the index order's. On the
    6x6 torus a spin with its four neighbours makes every warp reduction conflict-free under the
    model; on the 3x3x4 torus the model's set is clearly better than the index order's."""
    for lat, want in ((w.square(6, 6, True), 1.0), (w.cubic(3, 3, 4, True), None)):
        g = isg.isg_graph_create(lat.n, lat.edges)
        p = isg.isg_debug_plan(g, lane_model=1)
        q = isg.isg_debug_plan(g, lane_model=2)
        assert p["lane_model"] == 1 and q["lane_model"] == 0
        lanes = [i for i in range(lat.n) if (p["lane_mask"] >> i) & 1]
        assert len(lanes) == 5
        assert lat.n + 1 <= p["stride"] <= lat.n + 32
        assert p["lane_cost"] <= p["lane_cost_index_order"]
        if want is not None:
            assert p["lane_cost"] == want
        else:
            assert p["lane_cost"] < 0.95 * p["lane_cost_index_order"]
        # the index order keeps the five free spins after the inner ones
        assert [i for i in range(lat.n) if (q["lane_mask"] >> i) & 1] != lanes or p["lane_cost"] == p["lane_cost_index_order"]
    quick = isg.isg_debug_plan(g, lane_model=3)          # the quick search: still a valid, better set
    assert quick["lane_model"] == 1 and quick["lane_cost"] <= quick["lane_cost_index_order"]
    with pytest.raises(isg.IsgError) as ei:
        isg.isg_debug_plan(g, lane_model=5)
    assert ei.value.status == 1


def test_lane_model_against_sampled_reductions(isg):
    """The bank-conflict model's expected wavefronts per warp reduction (lanes.cpp) against the
    wavefronts of sampled reductions of the actual plan (isg_debug_lane_banks: the 32 lanes' word
    addresses at one step of a task, the most distinct addresses in one bank)."""
    rng = w.SplitMix64(17)
    for lat in (w.square(6, 6, True), w.cubic(3, 3, 4, True), w.with_random_couplings(w.square(5, 6, True), rng, (-1, 1)),
                w.triangular(5, 6, True)):
        g = isg.isg_graph_create(lat.n, lat.edges)
        for lm in (1, 3):
            p = isg.isg_debug_plan(g, lane_model=lm)
            if not p["lane_model"]:
                continue
            mean, worst = isg.isg_debug_lane_banks(g, samples=6000, seed=3, lane_model=lm)
            assert abs(mean - p["lane_cost"]) <= 0.06, (lat.name, lm, mean, p["lane_cost"])
            assert 1 <= worst <= 32


def check_lane_layout(isg, g, lat, **options):
    """The lane-table layout of the plan, checked from its definition: every (sub-table, row,
    column) word is distinct and inside the copy; lane l's columns popcount(l) + [0, N - 5] lie in
    its sub-table's range; the 32 lanes fall in 32 banks at any column; the row stride is a
    multiple of 32 with 8 R / G whole; the copy is no larger than ten separate padded blocks."""
    L = isg.isg_debug_lane_layout(g, **options)
    p = isg.isg_debug_plan(g, **options)
    n, rows, G, R = lat.n, p["n_e_compact"], p["G"], L["stride"]
    assert L["n_sub"] == 10 and R % 32 == 0 and (8 * R) % G == 0 and R >= n + 1
    words = np.concatenate([off + np.arange(rows)[:, None] * R + np.arange(lo, hi + 1)[None, :]
                            for off, lo, hi in zip(L["sub_off"], L["m_lo"], L["m_hi"])], axis=None)
    assert words.min() >= 0 and words.max() < L["copy_words"]
    assert len(np.unique(words)) == len(words)
    pc = np.array([bin(l).count("1") for l in range(32)])
    sub = L["lane_sub"]
    assert np.array_equal(L["lane_word"], L["sub_off"][sub])
    assert np.all(L["m_lo"][sub] <= pc) and np.all(pc + n - 5 <= L["m_hi"][sub])
    assert len(set((L["lane_word"] + pc) % 32)) == 32
    unit = 32
    while (8 * unit) % G:
        unit += 32
    separate = 10 * (rows * ((n + 1 + unit - 1) // unit * unit) + 32)
    assert L["copy_words"] <= separate
    assert p["smem_bytes"] == p["blob_bytes"] + p["copies"] * L["copy_words"] * 4
    return L


def _ring(n, J):
    return w.Lattice(n, np.array([(i, (i + 1) % n, J) for i in range(n)], np.int64), f"ring{n}-J{J}")


def test_lane_table_layouts_across_sizes(isg):
    """Lane-table layouts for N = 11 .. 62 (every residue of N - 5 mod 32, which sets the packed
    order) and energy strides G with odd factors (J = 3 rings: G = 12 where 8 (N + 1) allows it),
    each checked from its definition; packed wherever it takes fewer words than ten blocks."""
    packed = 0
    for n in range(11, 63):
        for J in (1, 3):
            lat = _ring(n, J)
            g = isg.isg_graph_create(n, lat.edges)
            packed += check_lane_layout(isg, g, lat, lane_model=4, max_spins=62)["packed"]
    assert packed >= 90
    for lat in (w.with_random_couplings(w.triangular(6, 6, True), w.SplitMix64(3), (-2, -1, 1, 2)),
                w.with_random_couplings(w.cubic(3, 3, 4, True), w.SplitMix64(3), (-2, -1, 1, 2))):
        g = isg.isg_graph_create(lat.n, lat.edges)
        assert isg.isg_debug_plan(g)["n_e_compact"] == 163
        assert isg.isg_debug_plan(g)["lane_tables"] == 10          # packed, they fit
        assert check_lane_layout(isg, g, lat)["packed"]


@pytest.mark.parametrize("lat", [w.cubic(3, 3, 4, True), w.square(6, 6, True), w.triangular(5, 6, True),
                                 w.with_random_couplings(w.square(5, 6, True), w.SplitMix64(4), (-2, -1, 1, 2)),
                                 w.random_graph(30, 90, w.SplitMix64(5))], ids=lambda l: l.name)
def test_lane_tables_make_every_reduction_conflict_free(isg, lat):
    """Lane tables (options.lane_model = 4): ten sub-tables per copy and a row stride that is a
    multiple of 32, so each lane's bank is its up count plus its sub-table's offset. Every sampled
    warp reduction of the plan takes exactly one wavefront, whatever the graph and couplings."""
    g = isg.isg_graph_create(lat.n, lat.edges)
    p = isg.isg_debug_plan(g, lane_model=4)
    assert p["lane_tables"] == 10
    check_lane_layout(isg, g, lat, lane_model=4)
    mean, worst = isg.isg_debug_lane_banks(g, samples=3000, seed=5, lane_model=4)
    assert mean == 1.0 and worst == 1
    for sym in (0, 1):
        mean, worst = isg.isg_debug_lane_banks(g, samples=500, seed=6, lane_model=4, symmetry=sym)
        assert worst == 1


def test_lane_tables_emulated_against_the_oracle(isg):
    """The kernel's walk on the host with lane tables (every address checked to lie among its own
    lane's sub-table bins; the flush sums the ten sub-tables): the oracle's table, whole, halved by
    the spin flip, in a shard range, and in a forced small shape with two copies."""
    rng = w.SplitMix64(9)
    for lat in (w.square(4, 5, True), w.cubic(2, 2, 4, True), w.with_random_couplings(w.square(4, 5, True), rng, (-2, -1, 1, 2)),
                w.triangular(4, 4, False), w.random_graph(18, 40, rng), _ring(17, 3),
                w.with_random_couplings(w.triangular(4, 5, True), rng, (-3, 3)), w.random_graph(19, 50, rng),
                w.with_random_couplings(w.square(3, 7, False), rng, (-2, -1, 1, 2)), w.random_graph(22, 44, rng)):
        g = isg.isg_graph_create(lat.n, lat.edges)
        ref = oracle.g_edges(lat.n, lat.edges)
        assert np.array_equal(isg.isg_debug_emulate(g, lane_model=4), ref)
        assert np.array_equal(isg.isg_debug_emulate(g, lane_model=4, symmetry=1), ref)
        assert np.array_equal(isg.isg_debug_emulate(g, lane_model=4, inner_bits=6, low_bits=3, block_threads=64, copies=2), ref)
        part = oracle.g_edges(lat.n, lat.edges, 1 << (lat.n - 2), 3 << (lat.n - 2))
        assert np.array_equal(isg.isg_debug_emulate(g, lane_model=4, shard_bits=2, shard_lo=1, shard_hi=3), part)


def test_packed_lane_tables_emulated_on_shards_of_large_graphs(isg):
    """Lane tables of 27 to 40 spins (fourteen residues of N - 5 mod 32: twelve packed orders, and
    the padded blocks at 30 and 31 spins, where they are smaller) on graphs with J in
    {-2, -1, 1, 2} or {-1, 1}: the kernel's walk on the host over one shard of 2^18
    configurations (every address checked against its lane's own sub-table columns) equals the
    oracle's table of the same range. A draw whose energy rows fit no lane-table layout would be
    refused with TOO_LARGE; at least twelve sizes run."""
    rng = w.SplitMix64(2740)
    done = 0
    for n in range(27, 41):
        kind = ("square", "triangular", "cubic")[n % 3]
        J = (-2, -1, 1, 2) if n % 2 else (-1, 1)
        lat = w.induced_lattice(kind, n, bool(n % 4 < 2), rng, couplings=J)
        g = isg.isg_graph_create(lat.n, lat.edges)
        k = n - 18
        lo = rng.below(1 << k)
        opts = dict(lane_model=4, shard_bits=k, shard_lo=lo, shard_hi=lo + 1)
        try:
            L = isg.isg_debug_lane_layout(g, **opts)
        except isg.IsgError as e:                  # too many energy rows for any lane-table layout
            assert e.status == 2, (lat.name, str(e))
            continue
        assert L["n_sub"] == 10 and L["packed"] == (n not in (30, 31)), lat.name   # blocks are smaller at 30, 31
        got = isg.isg_debug_emulate(g, **opts)
        assert np.array_equal(got, oracle.g_masks(n, lat.edges, lo << 18, (lo + 1) << 18)), lat.name
        done += 1
    assert done >= 12


def test_lane_tables_rejects(isg):
    lat = w.with_random_couplings(w.triangular(5, 8, True), w.SplitMix64(40), (-2, -1, 1, 2))
    g = isg.isg_graph_create(lat.n, lat.edges)
    with pytest.raises(isg.IsgError) as ei:                    # about 180 rows of 416 words
        isg.isg_debug_plan(g, lane_model=4)
    assert ei.value.status == 2
    t = w.square(6, 6, True)
    gt = isg.isg_graph_create(t.n, t.edges)
    with pytest.raises(isg.IsgError) as ei:
        isg.isg_debug_plan(gt, lane_model=4, bin_stride=45)
    assert ei.value.status == 1
    assert isg.isg_debug_plan(gt, lane_model=4, bin_stride=96)["stride"] == 96


def test_lane_model_is_deterministic_and_sign_free(isg):
    """The lane model's choice depends only on the graph's structure: the same lattice built twice
    (separate handles), and a copy with every coupling's sign flipped, get the same lane spins and
    stride; a thorough and a quick search are both repeatable."""
    lat = w.square(6, 6, True)
    neg = w.Lattice(lat.n, lat.edges * np.array([1, 1, -1]), "torus6x6-antiferro")
    plans = []
    for l in (lat, lat, neg):
        g = isg.isg_graph_create(l.n, l.edges)
        plans.append({k: v for k, v in isg.isg_debug_plan(g, lane_model=1).items() if k in ("lane_mask", "stride")})
    assert plans[0] == plans[1] == plans[2]
    g = isg.isg_graph_create(lat.n, lat.edges)
    q1 = isg.isg_debug_plan(g, lane_model=3)
    q2 = isg.isg_debug_plan(isg.isg_graph_create(lat.n, lat.edges), lane_model=3)
    assert q1 == q2

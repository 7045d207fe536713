"""Split-and-convolve enumeration, host side (no GPU): the planner's boundary sets and the
emulation of the split kernel's per-warp work against the oracle's full enumeration."""
import numpy as np
import pytest

import oracle
from paper_1110_2561_gb300 import workloads as w


def mask(idx):
    m = 0
    for i in idx:
        m |= 1 << i
    return m


def components_without(lat, S):
    """Connected components of the graph minus the spins of mask S (plain BFS, independent of the library)."""
    adj = [set() for _ in range(lat.n)]
    for i, j, J in lat.edges:
        if J:
            adj[int(i)].add(int(j))
            adj[int(j)].add(int(i))
    seen, comps = set(), []
    for v in range(lat.n):
        if (S >> v) & 1 or v in seen:
            continue
        stack, comp = [v], set()
        while stack:
            u = stack.pop()
            if u in comp:
                continue
            comp.add(u)
            stack.extend(x for x in adj[u] if not (S >> x) & 1 and x not in comp)
        seen |= comp
        comps.append(comp)
    return comps


CASES = [
    (w.square(4, 4, True), mask(range(0, 4)) | mask(range(8, 12))),       # two rows: Table 1's lattice
    (w.square(4, 4, False), mask(range(4, 8))),
    (w.ring(10), mask([0, 5])),
    (w.square(4, 5, True), 0),
    (w.square(5, 5, False), 0),
    (w.with_random_couplings(w.square(4, 5, True), w.SplitMix64(7), (-1, 1)), 0),
    (w.random_graph(20, 40, w.SplitMix64(3)), 0),
    (w.with_random_couplings(w.triangular(4, 5, True), w.SplitMix64(9), (-2, -1, 1, 2)), 0),
    (w.cubic(2, 3, 4, True), 0),
    (w.Lattice(7, np.zeros((0, 3), np.int64)), 0),                        # no bonds: seven components
    (w.square(3, 4, True), mask(range(12))),                               # everything boundary
    # components of 16 or more spins: walker lane spins and row strides chosen by the conflict model
    (w.square(4, 5, False), mask([0, 1, 2, 3])),                           # one component of 16
    (w.with_random_couplings(w.square(4, 5, True), w.SplitMix64(11), (-1, 1)), mask(range(0, 5)) | mask([10, 11, 12])),
    (w.with_random_couplings(w.triangular(3, 6, False), w.SplitMix64(12), (-2, -1, 1, 2)), mask([0])),   # 17 spins
]


@pytest.mark.parametrize("lat,boundary", CASES, ids=[c[0].name or "free-spins" for c in CASES])
def test_emulated_split_matches_oracle(isg, lat, boundary):
    gh = isg.isg_graph_create(lat.n, lat.edges)
    got = isg.isg_debug_emulate_split(gh, boundary)
    assert np.array_equal(got, oracle.g_masks(lat.n, lat.edges))


def test_table1_through_split(isg, table1_triples):
    """Table 1 (Sec. 4) from the emulated split with rows 0 and 2 as the boundary."""
    lat = w.square(4, 4, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = isg.isg_debug_emulate_split(gh, mask(range(0, 4)) | mask(range(8, 12)))
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    got = {(int(g[e, m]), -lat.n + 2 * m, e_min + 2 * e) for e, m in zip(*np.nonzero(g))}
    assert got == set(table1_triples)


@pytest.mark.parametrize("lat", [w.square(6, 6, True), w.square(7, 7, True), w.cubic(3, 3, 4, True),
                                 w.ea_instances()[0], w.triangular(6, 6, True)], ids=lambda l: l.name)
def test_plan_is_a_separator_and_cheaper(isg, lat):
    """The chosen boundary leaves components with no bond between them (checked here by a plain
    BFS), each of at most 30 spins, and the modelled work is below the full enumeration's."""
    gh = isg.isg_graph_create(lat.n, lat.edges)
    p = isg.isg_split_plan(gh)
    comps = components_without(lat, p["boundary"])
    assert len(comps) == p["components"] and max(len(c) for c in comps) == p["largest_component"] <= 30
    assert p["visits"] == 2.0 ** (p["boundary_spins"] - 1) * sum(2.0 ** len(c) for c in comps)
    assert p["work_ratio"] < 1
    assert p["visits"] < 2.0 ** lat.n / 10


def test_plan_torus_6x6_two_rows(isg):
    lat = w.square(6, 6, True)
    p = isg.isg_split_plan(isg.isg_graph_create(lat.n, lat.edges))
    assert p["boundary_spins"] == 12 and p["components"] == 2 and p["largest_component"] <= 13
    assert p["visits"] <= 2.0 ** 11 * (2.0 ** 11 + 2.0 ** 13) and p["work_ratio"] < 0.02


def test_split_rejections(isg):
    lat = w.square(6, 6, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    with pytest.raises(isg.IsgError, match="INVALID"):
        isg.isg_split_plan(gh, 1 << 40)                      # a spin beyond N
    with pytest.raises(isg.IsgError, match="TOO_LARGE"):
        isg.isg_split_plan(gh, 1)                            # leaves a 35-spin component
    many = w.Lattice(4, np.array([[0, 1, 1], [1, 2, 2], [2, 3, 3], [0, 3, 4], [0, 2, 5], [1, 3, 6],
                                  ], np.int64))
    assert isg.isg_split_plan(isg.isg_graph_create(many.n, many.edges), 0)["components"] >= 1
    # more than 16 distinct couplings
    edges = np.array([[i, j, 1 + i * 8 + j] for i in range(8) for j in range(i + 1, 8)], np.int64)
    with pytest.raises(isg.IsgError, match="TOO_LARGE"):
        isg.isg_split_plan(isg.isg_graph_create(8, edges), 0)


def _random_cases(count=40, seed=20260):
    """Seeded random graphs of 6..18 spins: sparse and dense, couplings from several alphabets
    (ferromagnetic, antiferromagnetic, +-J, +-1/+-2, wide), with isolated spins and disconnected
    pieces, each with a random boundary mask (possibly empty or everything)."""
    rng = w.SplitMix64(seed)
    alphabets = [(1,), (-1,), (-1, 1), (-2, -1, 1, 2), (-7, 3, 5, 11)]
    out = []
    for k in range(count):
        n = 6 + rng.below(13)
        m = rng.below(3 * n)
        lat = w.random_graph(n, m, rng, alphabets[k % len(alphabets)])
        r = rng.below(4)
        if r == 0:
            boundary = 0                                   # the planner's choice
        elif r == 1:
            boundary = (1 << n) - 1                        # every spin boundary
        else:
            boundary = rng.below(1 << n)                   # an arbitrary set (0: the planner's)
        out.append((lat, boundary))
    return out


@pytest.mark.parametrize("k", range(40))
def test_emulated_split_random_graphs(isg, k):
    lat, boundary = _random_cases()[k]
    gh = isg.isg_graph_create(lat.n, lat.edges)
    try:
        got = isg.isg_debug_emulate_split(gh, boundary)
    except isg.IsgError as e:
        # an arbitrary set may leave a component over 30 spins or too many classes: refused, not wrong
        assert "TOO_LARGE" in str(e)
        return
    assert np.array_equal(got, oracle.g_edges(lat.n, lat.edges))


@pytest.mark.parametrize("lat", [w.square(6, 6, True), w.with_random_couplings(w.square(5, 6, True), w.SplitMix64(4), (-1, 1))],
                         ids=lambda l: l.name)
def test_emulated_split_low_block(isg, lat):
    """Lattices whose components are large enough for a low block (walked with its fields held
    fixed and its configurations unrolled): the emulated kernel equals the frontier oracle."""
    gh = isg.isg_graph_create(lat.n, lat.edges)
    assert isg.isg_split_plan(gh)["largest_component"] >= 12
    assert np.array_equal(isg.isg_debug_emulate_split(gh), oracle.g_frontier(lat.n, lat.edges, 16))

"""Pins of the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each pin is chosen so that a plausible slip in the oracle -- a dropped bond, a wrong sign on E
or M, a transposed bin index, a wrong power of T -- fails at least one of them (the mutation
tests in test_oracle_mutants.py check exactly that).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1110_2561_gb300 import workloads as w
from closed_forms import (brute_force_g, brute_force_g_range, brute_force_magnetisation, free_spin_moments,
                          free_spins, golden_max, kaufman_C, kaufman_C_peak, kaufman_energy_counts, kaufman_logz,
                          ring_joint_count, ring_logz, ring_M2)

THREADS = os.cpu_count() or 1


def as_dict(g: np.ndarray, n: int, e_min: int):
    out = {}
    for e, m in zip(*np.nonzero(g)):
        out[(e_min + 2 * int(e), -n + 2 * int(m))] = int(g[e, m])
    return out


# --------------------------------------------------------------------------- Table 1 (Sec. 4)
@pytest.mark.parametrize("method", ["edges", "masks", "frontier"])
def test_table1_4x4_periodic(table1_triples, method):
    """Table 1: all 80 printed (Nc, M, E) cells of the 4x4 periodic ferromagnet, and nothing else."""
    lat = w.square(4, 4, True)
    g = {"edges": oracle.g_edges, "masks": oracle.g_masks, "frontier": oracle.g_frontier}[method](lat.n, lat.edges)
    e_min, n_e, n_m = oracle.bins(lat.n, lat.edges)
    assert (e_min, n_e, n_m) == (-32, 33, 17)
    got = as_dict(g, lat.n, e_min)
    want = {(E, M): nc for nc, M, E in table1_triples}
    assert len(want) == 80
    assert got == want
    assert sum(want.values()) == 2 ** 16          # Sec. 4: 65536 configurations


# --------------------------------------------------------------------------- invariants
def graphs_small():
    rng = w.SplitMix64(7)
    out = [w.square(4, 4, False), w.square(3, 5, True), w.triangular(3, 4, True), w.cubic(2, 2, 3, False),
           w.ring(9), w.ring(10, J=-1)]
    for n, ne in [(1, 0), (2, 1), (5, 7), (8, 12), (11, 20), (13, 30)]:
        out.append(w.random_graph(n, ne, rng))
    out.append(w.with_random_couplings(w.square(3, 4, True), rng, (-2, -1, 1, 2)))
    return out


@pytest.mark.parametrize("lat", graphs_small(), ids=lambda l: l.name)
def test_total_and_binomial_columns(lat):
    """Sec. 4 / Sec. 2: sum of g is 2^N and, for fixed M, the sum over E is C(N, (N+M)/2)."""
    g = oracle.g_masks(lat.n, lat.edges)
    assert int(g.sum()) == 2 ** lat.n
    for m in range(lat.n + 1):
        assert int(g[:, m].sum()) == math.comb(lat.n, m)


@pytest.mark.parametrize("lat", graphs_small(), ids=lambda l: l.name)
def test_global_flip_symmetry(lat):
    """Flipping every spin keeps E and negates M: g(E, M) = g(E, -M) for any couplings."""
    g = oracle.g_masks(lat.n, lat.edges)
    assert np.array_equal(g, g[:, ::-1])


@pytest.mark.parametrize("lat", [w.square(4, 4, False), w.square(3, 3, False), w.square(4, 4, True),
                                 w.cubic(2, 3, 2, False), w.triangular(3, 3, False), w.cubic(3, 3, 2, True)],
                         ids=lambda l: l.name)
def test_ferromagnet_ground_states(lat):
    """A connected ferromagnet has exactly two ground states, all up and all down, at E = -sum J."""
    g = oracle.g_masks(lat.n, lat.edges)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    assert e_min == -int(lat.edges[:, 2].sum())
    assert g[0, 0] == 1 and g[0, lat.n] == 1 and int(g[0].sum()) == 2


@pytest.mark.parametrize("lat", [w.square(4, 4, False), w.square(4, 6, True), w.cubic(2, 2, 4, True),
                                 w.square(3, 4, False)], ids=lambda l: l.name)
def test_bipartite_energy_mirror(lat):
    """On a bipartite ferromagnet, flipping one sublattice negates E: the E-marginal is mirrored."""
    g = oracle.g_masks(lat.n, lat.edges)
    marg = g.sum(axis=1)
    assert np.array_equal(marg, marg[::-1])


def test_gauge_invariance_pm_j():
    """+-J: flipping spin i together with the sign of every coupling at i maps configurations one
    to one and keeps E, so the E-marginal is unchanged (M is not)."""
    rng = w.SplitMix64(3)
    lat = w.with_random_couplings(w.square(4, 4, True), rng, (-1, 1))
    base = oracle.g_masks(lat.n, lat.edges).sum(axis=1)
    for site in (0, 5, 15):
        e = lat.edges.copy()
        at = (e[:, 0] == site) | (e[:, 1] == site)
        e[at, 2] *= -1
        assert np.array_equal(oracle.g_masks(lat.n, e).sum(axis=1), base)


@pytest.mark.parametrize("n", [3, 4, 7, 12, 15])
def test_ring_run_counting(n):
    """Periodic chain: a configuration with `up` up spins and 2r runs has 2r unsatisfied bonds,
    so E = -n + 4r, and the count is (n/r) C(up-1, r-1) C(n-up-1, r-1)."""
    lat = w.ring(n)
    g = oracle.g_edges(lat.n, lat.edges)
    e_min, n_e, _ = oracle.bins(lat.n, lat.edges)
    want = np.zeros_like(g)
    for up in range(n + 1):
        for r in range(0, n // 2 + 1):
            c = ring_joint_count(n, up, r)
            if c:
                want[(-n + 4 * r - e_min) // 2, up] += c
    assert np.array_equal(g, want)


@pytest.mark.parametrize("seed", range(6))
def test_second_language_brute_force(seed):
    """Random multigraphs (duplicate edges, J in {-2,-1,1,2}, isolated spins) against a pure-Python
    brute force of the definition."""
    rng = w.SplitMix64(100 + seed)
    n = 3 + rng.below(9)
    lat = w.random_graph(n, rng.below(2 * n + 1), rng)
    g = oracle.g_edges(lat.n, lat.edges)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    want = brute_force_g(lat.n, [tuple(int(x) for x in r) for r in lat.edges])
    want = {k: v for k, v in want.items() if v}
    assert as_dict(g, lat.n, e_min) == want


@pytest.mark.parametrize("lat", graphs_small() + [w.square(4, 5, True), w.triangular(4, 4, True),
                                                  w.square(5, 4, False)], ids=lambda l: l.name)
def test_three_oracles_agree(lat):
    """The bond loop, the popcount form and the frontier programme give the same table."""
    g0 = oracle.g_edges(lat.n, lat.edges)
    assert np.array_equal(g0, oracle.g_masks(lat.n, lat.edges, threads=3))
    assert np.array_equal(g0, oracle.g_frontier(lat.n, lat.edges))


def test_ranges_partition():
    """g over all configurations is the sum of g over any partition of [0, 2^N) into ranges."""
    lat = w.with_random_couplings(w.square(3, 5, True), w.SplitMix64(9), (-2, -1, 1, 2))
    full = oracle.g_masks(lat.n, lat.edges)
    cuts = [0, 1, 777, 4096, 20000, 2 ** 15]
    parts = sum(oracle.g_edges(lat.n, lat.edges, a, b) for a, b in zip(cuts[:-1], cuts[1:]))
    assert np.array_equal(parts, full)


@pytest.mark.parametrize("lo,hi", [(0, 1), (5, 6), (37, 301), (1000, 4096), (3001, 3001)])
def test_range_semantics(lo, hi):
    """A range [lo, hi) holds exactly the configuration words lo..hi-1, spin i being bit i."""
    rg = w.random_graph(12, 20, w.SplitMix64(11))
    want = brute_force_g_range(rg.n, [tuple(int(x) for x in r) for r in rg.edges], lo, hi)
    e_min, _, _ = oracle.bins(rg.n, rg.edges)
    for fn in (oracle.g_edges, oracle.g_masks):
        assert as_dict(fn(rg.n, rg.edges, lo, hi), rg.n, e_min) == want


def test_duplicate_edges_are_summed():
    """Listing a bond twice with J = 1 equals one bond with J = 2; opposite couplings cancel."""
    two = oracle.g_masks(3, [(0, 1, 1), (1, 0, 1), (1, 2, 1)])
    one = oracle.g_masks(3, [(0, 1, 2), (1, 2, 1)])
    assert np.array_equal(two, one)
    cancel = oracle.g_masks(3, [(0, 1, 2), (0, 1, -2), (1, 2, 1)])
    assert np.array_equal(cancel, oracle.g_masks(3, [(1, 2, 1)]))


def test_invalid_graphs_rejected():
    with pytest.raises(ValueError):
        oracle.g_edges(3, [(0, 0, 1)])
    with pytest.raises(ValueError):
        oracle.g_edges(3, [(0, 3, 1)])
    with pytest.raises(ValueError):
        oracle.g_edges(0, [])


def test_frontier_large_lattices_invariants():
    """The frontier programme reaches the 6x6 torus (2^36 configurations) exactly: total, binomial
    columns, the flip and bipartite mirrors, the two ground states and Kaufman's Z."""
    lat = w.square(6, 6, True)
    g = oracle.g_frontier(lat.n, lat.edges, max_active=16)
    assert int(g.sum()) == 2 ** 36
    for m in range(37):
        assert int(g[:, m].sum()) == math.comb(36, m)
    assert np.array_equal(g, g[:, ::-1])
    assert np.array_equal(g.sum(1), g.sum(1)[::-1])
    assert g[0, 0] == 1 and g[0, 36] == 1 and g[0].sum() == 2
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    T = np.linspace(0.5, 5, 16)
    lz = oracle.thermo(lat.n, e_min, g, T, [0.0])[0][:, 0]
    for t, l in zip(T, lz):
        assert abs(l - kaufman_logz(6, 6, t)) <= 1e-13 * abs(l)


# --------------------------------------------------------------------------- conditioned frontier
def _mask(sites):
    out = 0
    for i in sites:
        out |= 1 << i
    return out


@pytest.mark.parametrize("seed", range(8))
def test_frontier_cut_brute_force(seed):
    """The frontier programme conditioned on a cut set, on random multigraphs (couplings in
    {-2,-1,1,2}, duplicate edges, isolated spins) with an empty, a full and two random cut sets,
    against the pure-Python brute force of the definition."""
    rng = w.SplitMix64(300 + seed)
    n = 2 + rng.below(10)
    lat = w.random_graph(n, rng.below(2 * n + 1), rng)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    want = {k: v for k, v in brute_force_g(lat.n, [tuple(int(x) for x in r) for r in lat.edges]).items() if v}
    full = (1 << n) - 1
    for cut in (0, full, rng.next_u64() & full, rng.next_u64() & full):
        assert as_dict(oracle.g_frontier_cut(lat.n, lat.edges, cut, threads=2), lat.n, e_min) == want, cut


@pytest.mark.parametrize("cut", [_mask(range(4)), _mask(i for i in range(16) if (i // 4 + i % 4) % 2 == 0),
                                 _mask([0, 5, 10, 15]), _mask(range(16))], ids=["row", "checkerboard", "diagonal", "all"])
def test_frontier_cut_table1(table1_triples, cut):
    """Table 1 (Sec. 4) through the conditioned programme, for cut sets of several shapes."""
    lat = w.square(4, 4, True)
    g = oracle.g_frontier_cut(lat.n, lat.edges, cut)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    assert as_dict(g, lat.n, e_min) == {(E, M): nc for nc, M, E in table1_triples}


def test_frontier_cut_rejects():
    lat = w.square(4, 4, True)
    with pytest.raises(ValueError):
        oracle.g_frontier_cut(lat.n, lat.edges, 1 << 16)          # a cut spin outside the graph
    with pytest.raises(ValueError):
        oracle.g_frontier_cut(lat.n, lat.edges, 0, max_active=2)  # the rest's frontier is wider


@pytest.mark.parametrize("m,n", [(3, 3), (4, 4), (3, 5), (5, 4), (4, 6)])
def test_exact_energy_counts_kaufman(m, n):
    """The energy marginal of g, bin for bin, against the exact counts that Kaufman's closed form
    alone gives (the coefficients of Z as a polynomial in exp(-2K)), from every oracle."""
    lat = w.square(m, n, True)
    want = kaufman_energy_counts(m, n)
    assert sum(want) == 2 ** (m * n)
    tables = [oracle.g_frontier(lat.n, lat.edges), oracle.g_frontier_cut(lat.n, lat.edges, _mask(range(n)))]
    if m * n <= 20:
        tables.append(oracle.g_masks(lat.n, lat.edges, threads=THREADS))
    for g in tables:
        assert [int(x) for x in g.sum(axis=1)] == want


def _torus_pins(g, m, n):
    N = m * n
    assert sum(int(v) for v in g.ravel()) == 2 ** N
    assert all(sum(int(v) for v in g[:, k]) == math.comb(N, k) for k in range(N + 1))
    assert np.array_equal(g, g[:, ::-1])
    assert [int(x) for x in g.sum(axis=1)] == kaufman_energy_counts(m, n)
    assert int(g[0, 0]) == 1 and int(g[0, N]) == 1 and not g[0, 1:N].any()


def test_frontier_cut_torus_7x7():
    """The 7x7 torus (N = 49) by the programme conditioned on one row: every energy count exactly
    as Kaufman's closed form gives it, every spin-excess column C(49, m), the M -> -M mirror and
    the two ground states."""
    lat = w.square(7, 7, True)
    _torus_pins(oracle.g_frontier_cut(lat.n, lat.edges, _mask(range(7)), max_active=16, threads=THREADS), 7, 7)


def test_frontier_cut_torus_5x8():
    """The 5x8 torus (N = 40) by the programme conditioned on its first row of five spins, after
    renumbering the sites along the short side: the same pins as the 7x7 torus."""
    from relabel import layer_cut
    lat = w.square(5, 8, True)
    r, cut = layer_cut(lat)
    _torus_pins(oracle.g_frontier_cut(r.n, r.edges, cut, max_active=16, threads=THREADS), 5, 8)


def test_frontier_cut_torus_8x8():
    """The 8x8 torus (N = 64, 2^64 configurations) by the programme conditioned on one row (2^8
    rest programmes of 56 spins): the same pins as the 7x7 torus; the table's largest count is
    2.6e18 and its sum 2^64 (checked in Python integers)."""
    lat = w.square(8, 8, True)
    _torus_pins(oracle.g_frontier_cut(lat.n, lat.edges, _mask(range(8)), max_active=18, threads=THREADS), 8, 8)


# --------------------------------------------------------------------------- thermodynamics
@pytest.mark.parametrize("m,n", [(3, 3), (3, 4), (4, 4), (4, 5), (5, 3)])
def test_thermo_kaufman(m, n):
    """Eq. (2) from g on m x n tori against Kaufman's closed form at h = 0."""
    lat = w.square(m, n, True)
    g = oracle.g_masks(lat.n, lat.edges)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    T = np.linspace(0.5, 5, 25)
    lz = oracle.thermo(lat.n, e_min, g, T, [0.0])[0][:, 0]
    for t, l in zip(T, lz):
        assert abs(l - kaufman_logz(m, n, t)) <= 1e-13 * abs(l)


@pytest.mark.parametrize("n", [3, 8, 13])
def test_thermo_ring_in_field(n):
    """Periodic chain in a field against the 2 x 2 transfer matrix (covers the sign of h M)."""
    lat = w.ring(n)
    g = oracle.g_edges(lat.n, lat.edges)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    T = np.array([0.5, 1.0, 2.3, 5.0])
    h = np.array([-1.5, -0.2, 0.0, 0.7, 2.0])
    lz = oracle.thermo(lat.n, e_min, g, T, h)[0]
    for a, t in enumerate(T):
        for b, f in enumerate(h):
            assert abs(lz[a, b] - ring_logz(n, t, f)) <= 1e-13 * max(1.0, abs(lz[a, b]))


def test_thermo_free_spins():
    """No bonds: Z = (2 cosh(h/T))^N, <M> = N tanh(h/T), chi = N/T sech^2(h/T), <H> = -h <M>,
    C = h^2 chi / T."""
    n = 7
    g = oracle.g_edges(n, np.zeros((0, 3), dtype=np.int64))
    T = np.array([0.4, 1.0, 3.0])
    h = np.array([-2.0, 0.0, 0.5])
    lz, E, M, C, chi = oracle.thermo(n, 0, g, T, h)
    for a, t in enumerate(T):
        for b, f in enumerate(h):
            l0, m0, x0 = free_spins(n, t, f)
            assert lz[a, b] == pytest.approx(l0, rel=1e-14, abs=1e-14)
            assert M[a, b] == pytest.approx(m0, rel=1e-13, abs=1e-13)
            assert chi[a, b] == pytest.approx(x0, rel=1e-13)
            assert E[a, b] == pytest.approx(-f * m0, rel=1e-13, abs=1e-13)
            assert C[a, b] == pytest.approx(f * f * x0 / t, rel=1e-12, abs=1e-14)


def test_thermo_derivative_identities():
    """<H> = T^2 d lnZ/dT, <M> = T d lnZ/dh, C = d<H>/dT, chi = d<M>/dh (central differences)."""
    lat = w.with_random_couplings(w.triangular(3, 4, True), w.SplitMix64(5), (-2, -1, 1, 2))
    g = oracle.g_masks(lat.n, lat.edges)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    d = 1e-4
    for t, f in [(0.8, 0.3), (1.7, -0.9), (3.0, 0.0)]:
        lz, E, M, C, chi = (x[0, 0] for x in oracle.thermo(lat.n, e_min, g, [t], [f]))
        lzT = oracle.thermo(lat.n, e_min, g, [t - d, t + d], [f])
        lzh = oracle.thermo(lat.n, e_min, g, [t], [f - d, f + d])
        dT = (lzT[0][1, 0] - lzT[0][0, 0]) / (2 * d)
        dh = (lzh[0][0, 1] - lzh[0][0, 0]) / (2 * d)
        assert E == pytest.approx(t * t * dT, rel=1e-6, abs=1e-6)
        assert M == pytest.approx(t * dh, rel=1e-6, abs=1e-6)
        assert C == pytest.approx((lzT[1][1, 0] - lzT[1][0, 0]) / (2 * d), rel=1e-5, abs=1e-6)
        assert chi == pytest.approx((lzh[2][0, 1] - lzh[2][0, 0]) / (2 * d), rel=1e-5, abs=1e-6)


def test_specific_heat_peak_against_kaufman():
    """The oracle's specific heat C(T) on the 6x6 torus (frontier table) peaks where Kaufman's
    closed form does (C from second differences of ln Z), and its values agree there."""
    lat = w.square(6, 6, True)
    g = oracle.g_frontier(lat.n, lat.edges, max_active=16)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    c_oracle = lambda t: oracle.thermo(lat.n, e_min, g, [t], [0.0])[3][0, 0]
    t_or = golden_max(c_oracle, 1.5, 3.5)
    assert abs(t_or - kaufman_C_peak(6, 6, t_or)) <= 1e-5
    assert abs(c_oracle(t_or) - kaufman_C(6, 6, t_or)) <= 1e-5 * c_oracle(t_or)


# --------------------------------------------------------------------------- magnetisation
def test_magnetisation_free_spins():
    """No bonds: the number of up spins is binomial(N, (1 + tanh(h/T))/2); <|M|> from the
    binomial sum, <M^2> and <M^4> from the cumulants of one spin."""
    n = 9
    g = oracle.g_edges(n, np.zeros((0, 3), dtype=np.int64))
    T = np.array([0.3, 1.0, 4.0])
    h = np.array([-1.2, 0.0, 0.35])
    a, m2, m4, u = oracle.magnetisation(n, 0, g, T, h)
    for i, t in enumerate(T):
        for j, f in enumerate(h):
            a0, m20, m40 = free_spin_moments(n, t, f)
            assert a[i, j] == pytest.approx(a0, rel=1e-13)
            assert m2[i, j] == pytest.approx(m20, rel=1e-13)
            assert m4[i, j] == pytest.approx(m40, rel=1e-12)
            assert u[i, j] == pytest.approx(1 - m40 / (3 * m20 * m20), rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("n", [4, 9, 14])
def test_magnetisation_ring(n):
    """Periodic chain at h = 0: <M^2> = n sum_r (t^r + t^(n-r)) / (1 + t^n), t = tanh(1/T)."""
    lat = w.ring(n)
    g = oracle.g_edges(lat.n, lat.edges)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    T = np.array([0.4, 1.1, 2.5, 6.0])
    m2 = oracle.magnetisation(lat.n, e_min, g, T, [0.0])[1][:, 0]
    for t, v in zip(T, m2):
        assert v == pytest.approx(ring_M2(n, t), rel=1e-13)


@pytest.mark.parametrize("seed", [3, 8])
def test_magnetisation_brute_force(seed):
    """Random couplings in {-2, -1, 1, 2} on 11 spins: every moment against a direct sum over the
    2^11 configurations with their Boltzmann weights (no table in between), in a field too."""
    lat = w.random_graph(11, 20, w.SplitMix64(seed))
    edges = [tuple(int(x) for x in r) for r in lat.edges]
    g = oracle.g_edges(lat.n, lat.edges)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    for t, f in [(0.7, 0.0), (1.9, -0.4), (3.3, 1.1)]:
        a, m2, m4, u = (x[0, 0] for x in oracle.magnetisation(lat.n, e_min, g, [t], [f]))
        a0, m20, m40 = brute_force_magnetisation(lat.n, edges, t, f)
        assert (a, m2, m4) == pytest.approx((a0, m20, m40), rel=1e-12)
        assert u == pytest.approx(1 - m40 / (3 * m20 * m20), rel=1e-12)


def test_magnetisation_limits_and_chi():
    """4x4 ferromagnet: ordered at low T (<|M|> -> N, Binder cumulant -> 2/3), free at high T
    (cumulant -> 2/(3N)); at any (T, h), <M^2> - <M>^2 = T chi from the thermodynamics."""
    lat = w.square(4, 4, True)
    g = oracle.g_edges(lat.n, lat.edges)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    a, m2, m4, u = oracle.magnetisation(lat.n, e_min, g, [0.05, 1e7], [0.0])
    assert a[0, 0] == pytest.approx(16, rel=1e-12) and u[0, 0] == pytest.approx(2 / 3, rel=1e-12)
    assert u[1, 0] == pytest.approx(2 / (3 * 16), rel=1e-5)
    T, h = [0.9, 2.27, 4.0], [-0.5, 0.0, 0.3]
    _, _, M, _, chi = oracle.thermo(lat.n, e_min, g, T, h)
    m2 = oracle.magnetisation(lat.n, e_min, g, T, h)[1]
    assert np.allclose(m2 - M * M, np.array(T)[:, None] * chi, rtol=1e-11, atol=1e-11)

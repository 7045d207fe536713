"""GPU thermodynamics (isg_thermo) against the oracle's direct evaluation of Eq. (2), and the
FP32 path against the FP64 path within the stated bounds."""
import numpy as np
import pytest

import oracle
from paper_1110_2561_gb300 import workloads as w
from closed_forms import golden_max, kaufman_C_peak, kaufman_logz

pytestmark = pytest.mark.gpu


def rel_close(a, b, rtol, atol):
    return np.all(np.abs(a - b) <= rtol * np.abs(b) + atol)


def fp64_vs_oracle(isg, lat, T, h, sample=None):
    g_ref = oracle.g_masks(lat.n, lat.edges) if lat.n <= 24 else oracle.g_frontier(lat.n, lat.edges, 16)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    got = isg.isg_thermo(g_ref, gh, T, h, isg.ISG_FP64)
    ref = oracle.thermo(lat.n, e_min, g_ref, T, h)
    names = ["logZ", "E", "M", "C", "chi"]
    for k, (a, b) in enumerate(zip(got, ref)):
        # <M> vanishes at h = 0 by symmetry: absolute tolerance 1e-12 N there
        assert rel_close(a, b, 1e-12, 1e-12 * lat.n), (names[k], np.max(np.abs(a - b) / (np.abs(b) + 1e-300)))
    return got, g_ref, gh


@pytest.mark.parametrize("lat", [w.square(4, 4, False), w.ring(11), w.with_random_couplings(w.triangular(3, 5, True), w.SplitMix64(3), (-2, -1, 1, 2)),
                                 w.Lattice(6, np.zeros((0, 3), np.int64))], ids=lambda l: l.name or "free")
def test_fp64_small(isg, cuda, lat):
    T = np.linspace(0.5, 5, 64)
    h = np.array([-2.0, -0.3, 0.0, 0.1, 1.7])
    fp64_vs_oracle(isg, lat, T, h)


def test_exchange_energy_from_the_outputs(isg, cuda):
    """The mean exchange energy <E_J> = <H> + h <M> (H = E_J - h M, Eq. 1) from the FP64 outputs,
    against the exchange energy averaged directly over the oracle's table (every bin's E_J with
    the Boltzmann weight of its H, in long double)."""
    lat = w.with_random_couplings(w.square(4, 4, True), w.SplitMix64(31), (-2, -1, 1, 2))
    g = oracle.g_masks(lat.n, lat.edges)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    T = np.array([0.6, 1.3, 2.5, 4.0])
    h = np.array([-1.5, 0.0, 0.4, 2.0])
    _, E, M, _, _ = isg.isg_thermo(g, gh, T, h, isg.ISG_FP64)
    Ev = (e_min + 2 * np.arange(g.shape[0], dtype=np.longdouble))[:, None]
    Mv = (-lat.n + 2 * np.arange(g.shape[1], dtype=np.longdouble))[None, :]
    gl = g.astype(np.longdouble)
    for a, t in enumerate(T):
        for b, f in enumerate(h):
            x = -(Ev - f * Mv) / t
            wgt = np.where(gl > 0, gl * np.exp(x - x[gl > 0].max()), 0)
            want = float((wgt * Ev).sum() / wgt.sum())
            got = E[a, b] + f * M[a, b]
            # the bounds of the two outputs: 1e-12 relative on <H>, 1e-12 N on <M> (times |h|)
            assert abs(got - want) <= 1e-12 * (abs(E[a, b]) + (abs(f) + 1) * lat.n), (t, f, got, want)


def test_config_4x4_free_fp64(isg, cuda):
    """4x4 free ferromagnet, 64 temperatures in [0.5, 5] at h = 0, FP64."""
    fp64_vs_oracle(isg, w.square(4, 4, False), np.linspace(0.5, 5, 64), np.array([0.0]))


def test_torus_6x6_kaufman(isg, cuda):
    """6x6 torus: ln Z from the GPU table and GPU thermodynamics against Kaufman's closed form on
    256 temperatures in [0.5, 5], h = 0, FP64."""
    import torch
    lat = w.square(6, 6, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=cuda)
    isg.isg_enumerate(gh, g)
    T = np.linspace(0.5, 5, 256)
    lz = isg.isg_thermo(g, gh, T, [0.0], isg.ISG_FP64)[0][:, 0]
    ref = np.array([kaufman_logz(6, 6, t) for t in T])
    assert np.max(np.abs(lz - ref) / np.abs(ref)) <= 1e-12


def test_cubic_grid_fp32_vs_fp64(isg, cuda):
    """3x3x4 cubic torus on the 512 x 256 (T, h) grid: FP64 against the oracle on sampled points,
    FP32 against FP64 everywhere within the bounds |dlnZ| <= 2e-5, |d<E>| <= 1e-5 (S + N |h|max),
    |d<M>| <= 1e-5 N, C and chi within 1e-3 relative (or 1e-3 of the grid maximum)."""
    lat = w.cubic(3, 3, 4, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = isg.isg_enumerate(gh)
    T = np.linspace(0.5, 8, 512)
    h = np.linspace(-2, 2, 256)
    d = isg.isg_thermo(g, gh, T, h, isg.ISG_FP64)
    f = isg.isg_thermo(g, gh, T, h, isg.ISG_FP32)
    rng = w.SplitMix64(12)
    pts = [(rng.below(512), rng.below(256)) for _ in range(24)]
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    for a, b in pts:
        ref = oracle.thermo(lat.n, e_min, g, T[a:a + 1], h[b:b + 1])
        for k in range(5):
            assert abs(d[k][a, b] - ref[k][0, 0]) <= 1e-12 * abs(ref[k][0, 0]) + 1e-12 * lat.n, (k, a, b)
    S, N = 108, 36
    assert np.max(np.abs(f[0] - d[0])) <= 2e-5
    assert np.max(np.abs(f[1] - d[1])) <= 1e-5 * (S + N * 2)
    assert np.max(np.abs(f[2] - d[2])) <= 1e-5 * N
    for k in (3, 4):
        scale = np.max(np.abs(d[k]))
        err = np.abs(f[k] - d[k])
        assert np.all(err <= np.maximum(1e-3 * np.abs(d[k]), 1e-3 * scale)), k


@pytest.mark.parametrize("nT", [1, 5, 19, 40, 75, 76, 77])
def test_fp64_cluster_shapes_torus_6x6(isg, cuda, nT):
    """Grids of at most half as many temperatures as SMs split stage 1 over a thread-block cluster
    per temperature (on 152 SMs: 8 CTAs for 1, 5 and 19 temperatures, 3 for 40, 2 for 75 and 76,
    none for 77). Every shape against the oracle on the 6x6 torus's table, with few fields (a warp
    per point) and many (a thread per point)."""
    lat = w.square(6, 6, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = isg.isg_enumerate(gh)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    T = np.linspace(0.4, 6, nT)
    rows = np.unique(np.linspace(0, nT - 1, min(nT, 4)).astype(int))   # the oracle on sampled rows
    for h, pick in ((np.array([-1.0, 0.0, 0.5]), np.arange(nT)), (np.linspace(-2, 2, 64), rows)):
        got = isg.isg_thermo(g, gh, T, h, isg.ISG_FP64)
        ref = oracle.thermo(lat.n, e_min, g, T[pick], h)
        for k, (a, b) in enumerate(zip(got, ref)):
            assert rel_close(a[pick], b, 1e-12, 1e-12 * lat.n), (k, len(h), np.max(np.abs(a[pick] - b) / (np.abs(b) + 1e-300)))


def test_table_off_energy_sublattice(isg, cuda):
    """On the 4x4 torus every energy is a multiple of 4, so stage 1 walks every other energy bin.
    A table with counts on the other bins (in every other column: the shape of this graph's table,
    not its values) makes those columns fall back to the walk over every bin. FP64 against the
    oracle on a clustered (64 T) and an unclustered (160 T) grid, few and many fields; FP32
    within its ln Z bound of FP64."""
    lat = w.square(4, 4, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = isg.isg_enumerate(gh)
    rng = w.SplitMix64(21)
    n_e, n_m = g.shape
    for m in range(0, n_m, 2):
        for e in range(n_e):
            g[e, m] += rng.below(1000)
    assert np.any(g[1::2, 0] > 0)                     # odd bins are off the sublattice here
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    for T in (np.linspace(0.5, 5, 64), np.linspace(0.3, 8, 160)):
        for h in (np.array([-1.0, 0.0, 0.7]), np.linspace(-2, 2, 64)):
            got = isg.isg_thermo(g, gh, T, h, isg.ISG_FP64)
            pick = np.arange(len(T)) if len(h) < 64 else np.linspace(0, len(T) - 1, 6).astype(int)
            ref = oracle.thermo(lat.n, e_min, g, T[pick], h)          # many fields: sampled rows
            for k, (a, b) in enumerate(zip(got, ref)):
                assert rel_close(a[pick], b, 1e-12, 1e-12 * lat.n), (k, len(T), len(h))
            f = isg.isg_thermo(g, gh, T, h, isg.ISG_FP32)
            assert np.max(np.abs(f[0] - got[0])) <= 2e-5


def test_fp64_extreme_temperatures_and_fields(isg, cuda):
    """S/T up to 3.2e4 and |h/T| N up to 8e5, where the reference bins and dominant columns are
    searched in double rather than float; against the oracle at 1e-12."""
    T = np.array([1e-3, 2e-3, 0.01, 0.05, 0.5, 3.0, 1e3])
    h = np.array([-50.0, -1.0, 0.0, 1e-3, 1.0, 50.0])
    fp64_vs_oracle(isg, w.square(4, 4, True), T, h)
    fp64_vs_oracle(isg, w.with_random_couplings(w.triangular(3, 4, True), w.SplitMix64(5), (-2, -1, 1, 2)), T, h)


@pytest.mark.parametrize("nT,nh", [(1000, 25), (20, 1010)])
def test_fp64_grids_beyond_kernel_parameters(isg, cuda, nT, nh):
    """T and h grids of more than 1024 values together are copied to the device instead of
    travelling in the kernel parameters: 1000 x 25 (a CTA per temperature, a warp per point) and
    20 x 1010 (a cluster per temperature, a thread per point), 4x4 torus, against the oracle."""
    lat = w.square(4, 4, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = isg.isg_enumerate(gh)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    T = np.linspace(0.3, 7, nT)
    h = np.linspace(-3, 3, nh)
    got = isg.isg_thermo(g, gh, T, h, isg.ISG_FP64)
    ref = oracle.thermo(lat.n, e_min, g, T, h)
    for k, (a, b) in enumerate(zip(got, ref)):
        assert rel_close(a, b, 1e-12, 1e-12 * lat.n), (k, np.max(np.abs(a - b) / (np.abs(b) + 1e-300)))


def test_fp64_torus_8x8_clusters(isg, cuda):
    """The largest table (8x8 torus, N = 64: 129 x 65 bins, from split-and-convolve) on grids of
    3 and 40 temperatures, split over clusters of 8 and 3 CTAs on 152 SMs, with a warp per point
    and (3 temperatures) a thread per point, against the oracle."""
    import torch
    lat = w.square(8, 8, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=cuda)
    isg.isg_enumerate_split(gh, g)
    g_host = g.cpu().numpy()
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    for T, h in ((np.linspace(1.5, 4, 3), np.array([0.0, 0.3])), (np.linspace(1.5, 4, 3), np.linspace(-1, 1, 64)),
                 (np.linspace(1.5, 4, 40), np.array([0.0, 0.3]))):
        got = isg.isg_thermo(g, gh, T, h, isg.ISG_FP64)
        ref = oracle.thermo(lat.n, e_min, g_host, T, h)
        for k, (a, b) in enumerate(zip(got, ref)):
            assert rel_close(a, b, 1e-12, 1e-12 * lat.n), (k, len(T), len(h))


def test_fp32_torus_8x8_within_bounds(isg, cuda):
    """FP32 against FP64 on the largest table (8x8 torus, 129 x 65 bins, from split-and-convolve)
    on a clustered grid (40 T) and an unclustered one (200 T), few and many fields, within the
    stated bounds: |d ln Z| <= 2e-5, |d<E>| <= 1e-5 (S + N |h|max), |d<M>| <= 1e-5 N, C and chi
    within 1e-3 relative or 1e-3 of the grid maximum."""
    import torch
    lat = w.square(8, 8, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=cuda)
    isg.isg_enumerate_split(gh, g)
    S, N = 128, 64
    for T in (np.linspace(1.0, 6, 40), np.linspace(0.5, 8, 200)):
        for h in (np.array([0.0, 0.2]), np.linspace(-1, 1, 64)):
            d = isg.isg_thermo(g, gh, T, h, isg.ISG_FP64)
            f = isg.isg_thermo(g, gh, T, h, isg.ISG_FP32)
            hmax = float(np.max(np.abs(h)))
            assert np.max(np.abs(f[0] - d[0])) <= 2e-5
            assert np.max(np.abs(f[1] - d[1])) <= 1e-5 * (S + N * hmax)
            assert np.max(np.abs(f[2] - d[2])) <= 1e-5 * N
            for k in (3, 4):
                scale = np.max(np.abs(d[k]))
                assert np.all(np.abs(f[k] - d[k]) <= np.maximum(1e-3 * np.abs(d[k]), 1e-3 * scale)), (k, len(T), len(h))


def test_thermo_device_outputs(isg, cuda):
    import torch
    lat = w.square(4, 4, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=cuda)
    isg.isg_enumerate(gh, g)
    T = np.linspace(1, 3, 7)
    h = np.linspace(-1, 1, 5)
    outs = tuple(torch.empty((7, 5), dtype=torch.float64, device=cuda) for _ in range(5))
    isg.isg_thermo(g, gh, T, h, isg.ISG_FP64, out=outs)
    torch.cuda.synchronize()
    ref = isg.isg_thermo(g.cpu().numpy(), gh, T, h, isg.ISG_FP64)
    for a, b in zip(outs, ref):
        assert np.array_equal(a.cpu().numpy(), b)


def test_thermo_rejects_bad_grid(isg, cuda):
    gh = isg.isg_graph_create(4, w.ring(4).edges)
    g = np.zeros(isg.table_shape(gh), np.int64)
    with pytest.raises(isg.IsgError):
        isg.isg_thermo(g, gh, [0.0], [0.0])
    with pytest.raises(isg.IsgError):
        isg.isg_thermo(g, gh, [1.0], [np.nan])


def test_specific_heat_peak(isg, cuda):
    """isg_specific_heat_peak on the 6x6 torus equals the oracle's peak (golden-section search on
    its C(T)) and Kaufman's; on a triangular +-J lattice in a field too. In FP32 the location is
    limited by the float error of C (~1e-6 relative) on a flat maximum: within 1e-4 relative."""
    lat = w.square(6, 6, True)
    g = oracle.g_frontier(lat.n, lat.edges, max_active=16)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    t_gpu, c_gpu = isg.isg_specific_heat_peak(g, gh, 0.0, 1.0, 4.0)
    c_oracle = lambda t: oracle.thermo(lat.n, e_min, g, [t], [0.0])[3][0, 0]
    t_or = golden_max(c_oracle, 1.5, 3.5, tol=1e-11)
    assert abs(t_gpu - t_or) <= 1e-7 * t_or
    assert abs(c_gpu - c_oracle(t_gpu)) <= 1e-12 * c_gpu
    assert abs(t_gpu - kaufman_C_peak(6, 6, t_gpu)) <= 1e-5
    t32, _ = isg.isg_specific_heat_peak(g, gh, 0.0, 1.0, 4.0, isg.ISG_FP32)
    assert abs(t32 - t_or) <= 1e-4 * t_or
    tri = w.with_random_couplings(w.triangular(3, 4, True), w.SplitMix64(6), (-1, 1))
    gt = oracle.g_masks(tri.n, tri.edges)
    ht = isg.isg_graph_create(tri.n, tri.edges)
    et, _, _ = oracle.bins(tri.n, tri.edges)
    t_gpu, _ = isg.isg_specific_heat_peak(gt, ht, 0.3, 0.2, 6.0)
    c_or = lambda t: oracle.thermo(tri.n, et, gt, [t], [0.3])[3][0, 0]
    grid = np.linspace(0.2, 6.0, 400)
    t0 = grid[int(np.argmax([c_or(t) for t in grid]))]
    t_or = golden_max(c_or, t0 - 0.03, t0 + 0.03, tol=1e-11)
    assert abs(t_gpu - t_or) <= 1e-7 * t_or


# --------------------------------------------------------------------------- magnetisation
MAG_NAMES = ["absM", "M2", "M4", "binder"]


@pytest.mark.parametrize("lat", [w.square(4, 4, False), w.ring(11), w.with_random_couplings(w.triangular(3, 5, True), w.SplitMix64(3), (-2, -1, 1, 2)),
                                 w.Lattice(6, np.zeros((0, 3), np.int64))], ids=lambda l: l.name or "free")
def test_magnetisation_fp64_small(isg, cuda, lat):
    """<|M|>, <M^2>, <M^4>, Binder's cumulant against the oracle at 1e-12 relative, FP64."""
    g = oracle.g_masks(lat.n, lat.edges)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    T = np.linspace(0.3, 6, 48)
    h = np.array([-1.5, -0.2, 0.0, 0.4, 2.0])
    got = isg.isg_magnetisation(g, gh, T, h, isg.ISG_FP64)
    ref = oracle.magnetisation(lat.n, e_min, g, T, h)
    for k, (a, b) in enumerate(zip(got, ref)):
        assert rel_close(a, b, 1e-12, 1e-13), (MAG_NAMES[k], np.max(np.abs(a - b) / np.abs(b)))


def test_magnetisation_cubic_grid(isg, cuda):
    """3x3x4 cubic torus on the 512 x 256 (T, h) grid: FP64 against the oracle on sampled points
    (1e-12 relative); FP32 against FP64 everywhere: <|M|>, <M^2>, <M^4> within 1e-5 relative,
    Binder's cumulant within 1e-5 absolute (it is a difference of two O(1) terms)."""
    lat = w.cubic(3, 3, 4, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = isg.isg_enumerate(gh)
    T = np.linspace(0.5, 8, 512)
    h = np.linspace(-2, 2, 256)
    d = isg.isg_magnetisation(g, gh, T, h, isg.ISG_FP64)
    f = isg.isg_magnetisation(g, gh, T, h, isg.ISG_FP32)
    rng = w.SplitMix64(13)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    for _ in range(16):
        a, b = rng.below(512), rng.below(256)
        ref = oracle.magnetisation(lat.n, e_min, g, T[a:a + 1], h[b:b + 1])
        for k in range(4):
            assert abs(d[k][a, b] - ref[k][0, 0]) <= 1e-12 * abs(ref[k][0, 0]) + 1e-13, (MAG_NAMES[k], a, b)
    for k in range(3):
        assert np.max(np.abs(f[k] - d[k]) / d[k]) <= 1e-5, MAG_NAMES[k]
    assert np.max(np.abs(f[3] - d[3])) <= 1e-5


def test_magnetisation_device_outputs(isg, cuda):
    import torch
    lat = w.square(4, 4, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=cuda)
    isg.isg_enumerate(gh, g)
    T = np.linspace(1, 3, 7)
    h = np.linspace(-1, 1, 5)
    outs = tuple(torch.empty((7, 5), dtype=torch.float64, device=cuda) for _ in range(4))
    isg.isg_magnetisation(g, gh, T, h, isg.ISG_FP64, out=(outs[0], None, outs[2], outs[3]))
    torch.cuda.synchronize()
    ref = isg.isg_magnetisation(g.cpu().numpy(), gh, T, h, isg.ISG_FP64)
    for k in (0, 2, 3):
        assert np.array_equal(outs[k].cpu().numpy(), ref[k])


def test_binder_cumulants_cross_near_onsager(isg, cuda):
    """Binder's cumulant of the 4x4 and 6x6 ferromagnetic tori (GPU tables, FP64): the larger
    system is more ordered below the transition and less above it, so the curves cross once on
    [1.5, 3.5], close to the infinite-lattice temperature 2 / ln(1 + sqrt 2) = 2.269."""
    T = np.linspace(1.5, 3.5, 401)
    u = []
    for L in (4, 6):
        lat = w.square(L, L, True)
        gh = isg.isg_graph_create(lat.n, lat.edges)
        u.append(isg.isg_magnetisation(isg.isg_enumerate(gh), gh, T, [0.0], isg.ISG_FP64)[3][:, 0])
    diff = u[1] - u[0]
    sign_changes = np.nonzero(np.diff(np.sign(diff)))[0]
    assert len(sign_changes) == 1
    t_cross = T[sign_changes[0]]
    assert abs(t_cross - 2 / np.log(1 + np.sqrt(2))) < 0.1, t_cross


@pytest.mark.parametrize("lat", [w.square(4, 4, False), w.square(6, 6, True), w.cubic(3, 3, 4, True),
                                 w.with_random_couplings(w.triangular(4, 5, True), w.SplitMix64(9), (-2, -1, 1, 2))],
                         ids=lambda l: l.name)
def test_zero_field_path_against_the_general_path(isg, cuda, lat):
    """Grids whose fields are all zero take the per-energy path (the sum over M once per energy);
    its outputs, thermodynamic and magnetic, equal those of the general kernel (the h = 0 row of a
    grid that also holds a nonzero field) within 1e-12 relative."""
    g = oracle.g_masks(lat.n, lat.edges) if lat.n <= 24 else \
        oracle.g_frontier(lat.n, lat.edges, 16) if lat.meta.get("kind") == "square" else None
    if g is None:
        from relabel import layer_cut
        r, cut = layer_cut(lat)
        g = oracle.g_frontier_cut(r.n, r.edges, cut, max_active=20)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    T = np.linspace(0.4, 6, 97)
    zero = isg.isg_thermo(g, gh, T, [0.0], isg.ISG_FP64)
    gen = isg.isg_thermo(g, gh, T, [0.0, 0.25], isg.ISG_FP64)
    for k, (a, b) in enumerate(zip(zero, gen)):
        assert rel_close(a[:, 0], b[:, 0], 1e-12, 1e-12 * lat.n), k
    mz = isg.isg_magnetisation(g, gh, T, [0.0], isg.ISG_FP64)
    mg = isg.isg_magnetisation(g, gh, T, [0.0, 0.25], isg.ISG_FP64)
    for k, (a, b) in enumerate(zip(mz, mg)):
        assert rel_close(a[:, 0], b[:, 0], 1e-12, 1e-12), k


def test_zero_field_path_on_asymmetric_counts(isg, cuda):
    """The per-energy path on a table of arbitrary counts (no M -> -M symmetry, so <M> is not zero
    and the per-energy variances matter) against the oracle at h = 0, FP64 and FP32 requests."""
    lat = w.square(4, 4, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    rng = np.random.default_rng(7)
    g = oracle.g_masks(lat.n, lat.edges)
    g = np.where(g > 0, g * rng.integers(1, 50, size=g.shape) + rng.integers(0, 3, size=g.shape), 0).astype(np.int64)
    g[:, -1] += 5                                     # a heavier all-up column
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    T = np.linspace(0.5, 5, 31)
    ref = oracle.thermo(lat.n, e_min, g, T, [0.0])
    for prec in (isg.ISG_FP64, isg.ISG_FP32):
        got = isg.isg_thermo(g, gh, T, [0.0], prec)
        for k, (a, b) in enumerate(zip(got, ref)):
            assert rel_close(a, b, 1e-12, 1e-12 * lat.n), (prec, k, np.max(np.abs(a - b) / (np.abs(b) + 1e-300)))


def test_zero_field_path_at_its_size_limit(isg, cuda):
    """Tables of nearly 1024 energy bins (the per-energy path's largest shared-memory block) and of
    more (the general kernel), from graphs with large couplings, at h = 0 against the oracle."""
    for J, expect_fast in (((-23, 17, 29, -31), True), ((-31, 37, 41, -43), False)):
        lat = w.random_graph(18, 36, w.SplitMix64(5), couplings=J)
        gh = isg.isg_graph_create(lat.n, lat.edges)
        n_e = isg.table_shape(gh)[0]
        assert (n_e <= 1024) == expect_fast, n_e
        g = oracle.g_masks(lat.n, lat.edges)
        e_min, _, _ = oracle.bins(lat.n, lat.edges)
        T = np.linspace(2.0, 60.0, 37)
        got = isg.isg_thermo(g, gh, T, [0.0], isg.ISG_FP64)
        ref = oracle.thermo(lat.n, e_min, g, T, [0.0])
        for k, (a, b) in enumerate(zip(got, ref)):
            assert rel_close(a, b, 1e-12, 1e-12 * lat.n), (J, k)


@pytest.mark.parametrize("index", [0, 3])
def test_fp32_within_bounds_on_frustrated_instances(isg, cuda, index):
    """FP32 against FP64 on Edwards-Anderson +-J 5x6 instances (frustrated, many degenerate ground
    states), down to T = 0.2 and across h in [-2, 2]: the stated bounds |dlnZ| <= 2e-5,
    |d<E>| <= 1e-5 (S + N |h|max), |d<M>| <= 1e-5 N, C and chi within 1e-3 relative (or 1e-3 of the
    grid maximum); the FP64 path against the oracle on sampled points."""
    lat = [l for l in w.ea_instances(64) if l.n == 30][index]
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = oracle.g_frontier(lat.n, lat.edges, 16)
    T = np.linspace(0.2, 5, 97)
    h = np.linspace(-2, 2, 65)
    d = isg.isg_thermo(g, gh, T, h, isg.ISG_FP64)
    f = isg.isg_thermo(g, gh, T, h, isg.ISG_FP32)
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    rng = w.SplitMix64(40 + index)
    for _ in range(12):
        a, b = rng.below(len(T)), rng.below(len(h))
        ref = oracle.thermo(lat.n, e_min, g, T[a:a + 1], h[b:b + 1])
        for k in range(5):
            assert abs(d[k][a, b] - ref[k][0, 0]) <= 1e-12 * abs(ref[k][0, 0]) + 1e-12 * lat.n, (k, a, b)
    S, N = int(np.abs(lat.edges[:, 2]).sum()), lat.n
    assert np.max(np.abs(f[0] - d[0])) <= 2e-5
    assert np.max(np.abs(f[1] - d[1])) <= 1e-5 * (S + N * 2)
    assert np.max(np.abs(f[2] - d[2])) <= 1e-5 * N
    for k in (3, 4):
        scale = np.max(np.abs(d[k]))
        err = np.abs(f[k] - d[k])
        assert np.all(err <= np.maximum(1e-3 * np.abs(d[k]), 1e-3 * scale)), k

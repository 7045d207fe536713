"""The request server (continuous batching): every result equals the same graph enumerated
alone, whatever else was in flight; admission limits, cancellation and timeouts are reported on
the host without disturbing the other requests."""
import os
import time

import numpy as np
import pytest

import oracle
from paper_1110_2561_gb300 import workloads as w

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


def alone(isg, lat):
    return isg.isg_enumerate(isg.isg_graph_create(lat.n, lat.edges))


def reference(lat):
    """The oracle's table: the popcount oracle up to 22 spins, else the frontier programme."""
    from relabel import frontier_table
    return oracle.g_masks(lat.n, lat.edges, threads=THREADS) if lat.n <= 22 else frontier_table(lat, THREADS)


def test_mix_equals_alone(isg, cuda):
    """A seeded request stream (N 16..32, square / triangular / cubic, free or periodic, J in
    {-2,-1,1,2}) submitted at once from one thread: each table equals isg_enumerate alone and the
    oracle's (the popcount oracle up to 22 spins, the frontier programme above)."""
    reqs = w.serving_stream(48, n_range=(16, 32), seed=7)
    srv = isg.Server(step_ms=5.0)
    tickets = [(srv.submit(isg.isg_graph_create(r.lattice.n, r.lattice.edges)), r.lattice) for r in reqs]
    for t, lat in tickets:
        srv.wait(t, 60000)
        g, times = srv.result(t)
        assert np.array_equal(g, alone(isg, lat)), lat.name
        assert times[2] >= times[1] >= 0 and times[0] >= 0
        assert np.array_equal(g, reference(lat)), lat.name
    st = srv.stats()
    assert st["tickets"] == 0 and st["admitted"] == 0 and st["steps"] >= 1
    srv.close()


def test_mix_with_split_equals_alone(isg, cuda):
    """With split-and-convolve enabled (split_work_ratio = 0.5), a stream of requests up to N = 36
    (the large ones served by split launches, mixed with tile steps) gives every table equal to
    isg_enumerate alone and to the oracle's; the split planner is consulted on the host for each
    large request."""
    reqs = w.serving_stream(40, n_range=(20, 36), seed=11)
    srv = isg.Server(step_ms=5.0, split_work_ratio=0.5)
    tickets = [(srv.submit(isg.isg_graph_create(r.lattice.n, r.lattice.edges)), r.lattice) for r in reqs]
    n_split = 0
    for t, lat in tickets:
        srv.wait(t, 120000)
        g, _ = srv.result(t)
        assert np.array_equal(g, alone(isg, lat)), lat.name
        assert np.array_equal(g, reference(lat)), lat.name
        gh = isg.isg_graph_create(lat.n, lat.edges)
        try:
            n_split += lat.n >= 24 and isg.isg_split_plan(gh)["work_ratio"] < 0.5
        except isg.IsgError:
            pass
    assert n_split >= 5                          # the stream really exercises the split path
    srv.close()


def test_mix_with_symmetry_equals_alone(isg, cuda):
    """With symmetry = 1 the server enumerates only the configurations with spin N-1 up of every
    tile-served request of 13 or more spins and mirrors the table in the step that carries its last
    tile: every table equals isg_enumerate alone (all 2^N configurations) and the oracle's, and the
    server counts about half the configurations enumerated."""
    reqs = w.serving_stream(40, n_range=(10, 30), seed=13)
    srv = isg.Server(step_ms=5.0, symmetry=1)
    tickets = [(srv.submit(isg.isg_graph_create(r.lattice.n, r.lattice.edges)), r.lattice) for r in reqs]
    for t, lat in tickets:
        srv.wait(t, 60000)
        g, _ = srv.result(t)
        assert np.array_equal(g, alone(isg, lat)), lat.name
        assert np.array_equal(g, reference(lat)), lat.name
    st = srv.stats()
    full = sum(1 << lat.n for _, lat in tickets)
    assert st["configs"] < 0.6 * full
    srv.close()
    with pytest.raises(isg.IsgError):
        isg.Server(symmetry=2)


def test_mix_with_split_and_symmetry_equals_alone(isg, cuda):
    """Both options at once (split_work_ratio = 0.5, symmetry = 1): large requests by split launches,
    the other tile-served ones halved and mirrored, in shared steps. Every table equals
    isg_enumerate alone and the oracle's."""
    reqs = w.serving_stream(32, n_range=(14, 34), seed=17)
    srv = isg.Server(step_ms=5.0, split_work_ratio=0.5, symmetry=1)
    tickets = [(srv.submit(isg.isg_graph_create(r.lattice.n, r.lattice.edges)), r.lattice) for r in reqs]
    for t, lat in tickets:
        srv.wait(t, 120000)
        g, _ = srv.result(t)
        assert np.array_equal(g, alone(isg, lat)), lat.name
        assert np.array_equal(g, reference(lat)), lat.name
    srv.close()


@pytest.mark.parametrize("opts", [{}, dict(symmetry=1), dict(lane_model=0)], ids=["every-configuration", "symmetry",
                                                                               "index-order"])
def test_largest_requests_against_frontier_oracle(isg, cuda, opts):
    """Requests of N = 37 and 38, the top of the request stream's range (square, triangular and
    simple cubic, periodic and free, J in {-2,-1,1,2}), served in one mix (every configuration
    with the default quick lane search, halved by the spin flip, or in index order): every table
    equals the oracle's frontier programme (sites renumbered along the short side), conditioned on
    the first cross-section for the periodic cubic requests (whose own frontier spans two
    cross-sections of 2 x 4 sites and their wrap-around)."""
    from concurrent.futures import ThreadPoolExecutor
    from relabel import layer_cut, short_side_fastest
    rng = w.SplitMix64(3738)
    lats = [w.induced_lattice(kind, n, per, rng) for n in (37, 38) for kind in ("square", "triangular")
            for per in (True, False)] + [w.induced_lattice("cubic", n, False, rng) for n in (37, 38)]
    lats += [w.induced_lattice("cubic", n, True, w.SplitMix64(3700 + n)) for n in (37, 38)]
    srv = isg.Server(step_ms=5.0, **opts)
    tickets = [srv.submit(isg.isg_graph_create(l.n, l.edges)) for l in lats]

    def ref(l):
        if l.meta["kind"] == "cubic" and l.meta["periodic"]:
            r, cut = layer_cut(l)
            return oracle.g_frontier_cut(r.n, r.edges, cut, max_active=20)
        r = short_side_fastest(l)
        return oracle.g_frontier(r.n, r.edges, max_active=20)
    with ThreadPoolExecutor(max_workers=THREADS) as ex:
        refs = list(ex.map(ref, lats))
    for t, l, r in zip(tickets, lats, refs):
        srv.wait(t, 120000)
        g, _ = srv.result(t)
        assert int(r.sum()) == 1 << l.n
        assert np.array_equal(g, r), l.name
    # lane tables fit one CTA for all but the two triangular 38-spin requests (about 180 rows)
    lc = srv.lane_counts()
    assert lc["requests"] == (0 if opts.get("lane_model") == 0 else 10)
    assert lc["launches"] >= lc["requests"]
    srv.close()


@pytest.mark.parametrize("sym", [0, 1], ids=["every-configuration", "symmetry"])
def test_lane_table_requests_across_steps(isg, cuda, sym):
    """36-spin tori with J in {-2,-1,1,2} (lane tables fit one CTA only packed), served by the
    enumeration kernel in task ranges over many 1 ms steps, next to small requests that go to the
    batch kernel in the same steps, with or without the spin-flip halving: every table equals the
    oracle's (the frontier programme for the tori)."""
    rng = w.SplitMix64(36)
    big = [w.with_random_couplings(getattr(w, k)(6, 6, True), w.SplitMix64(3), (-2, -1, 1, 2))
           for k in ("square", "triangular")] + [w.with_random_couplings(w.cubic(3, 3, 4, True), w.SplitMix64(3), (-2, -1, 1, 2))]
    small = [w.induced_lattice(k, n, per, rng) for n in (16, 20) for k in ("square", "triangular") for per in (True, False)]
    lats = [x for pair in zip(big, small) for x in pair] + small[len(big):]
    srv = isg.Server(step_ms=1.0, symmetry=sym)
    tickets = [srv.submit(isg.isg_graph_create(l.n, l.edges)) for l in lats]
    refs = [reference(l) for l in lats]
    for t, l, r in zip(tickets, lats, refs):
        srv.wait(t, 120000)
        g, _ = srv.result(t)
        assert np.array_equal(g, r), l.name
    lc = srv.lane_counts()
    assert lc["requests"] == 3
    assert lc["launches"] >= 6                 # each torus over more than one step
    srv.close()


def test_server_rejects_bad_split_ratio(isg, cuda):
    with pytest.raises(isg.IsgError, match="INVALID"):
        isg.Server(split_work_ratio=1.5)


def test_staggered_arrivals_and_small_arena(isg, cuda):
    """Requests arriving while others run, with an arena that holds only a few tables at a time and
    two admission slots: all finish and match."""
    lats = [w.square(5, 6, True), w.cubic(2, 3, 4, True), w.triangular(4, 5, False), w.square(4, 4, False),
            w.with_random_couplings(w.square(6, 5, True), w.SplitMix64(3), (-1, 1)), w.ring(12)]
    srv = isg.Server(max_inflight=2, arena_bytes=1 << 20, step_ms=2.0)
    tickets = []
    for lat in lats:
        tickets.append((srv.submit(isg.isg_graph_create(lat.n, lat.edges)), lat))
        time.sleep(0.002)
    for t, lat in tickets:
        srv.wait(t)
        assert np.array_equal(srv.result(t)[0], alone(isg, lat)), lat.name
    srv.close()


def test_limits_cancel_timeout(isg, cuda):
    srv = isg.Server(max_inflight=1, max_queued=1, step_ms=1.0)
    big = w.square(5, 8, True)                              # 2^40 configurations: ~0.15 s of steps
    gb = isg.isg_graph_create(big.n, big.edges)
    t1 = srv.submit(gb)
    with pytest.raises(isg.IsgError) as ei:                 # N > max_spins
        srv.submit(isg.isg_graph_create(41, w.random_graph(41, 50, w.SplitMix64(1)).edges))
    assert ei.value.status == 2
    time.sleep(0.01)                                        # let t1 be admitted
    small = w.square(4, 4, True)
    t2 = srv.submit(isg.isg_graph_create(small.n, small.edges))   # waits: the only slot is busy
    with pytest.raises(isg.IsgError) as ei:                 # queue of one is full
        srv.submit(isg.isg_graph_create(small.n, small.edges))
    assert ei.value.status == 6
    with pytest.raises(isg.IsgError) as ei:                 # not finished within 0 ms
        srv.wait(t1, 0)
    assert ei.value.status == 5
    with pytest.raises(isg.IsgError) as ei:
        srv.result(t2)
    assert ei.value.status in (7,)
    srv.cancel(t1)                                          # frees the slot after its steps drain
    srv.wait(t2, 60000)
    assert np.array_equal(srv.result(t2)[0], alone(isg, small))
    with pytest.raises(isg.IsgError):
        srv.poll(t1)                                        # cancelled ticket is gone
    srv.close()


@pytest.mark.parametrize("lane", [0, 1], ids=["tiles", "lane-tables"])
@pytest.mark.parametrize("where", [1, 2], ids=["before-enqueue", "after-launch"])
def test_host_side_step_failure_releases_slots(isg, cuda, where, lane):
    """A host-side failure of an engine step (injected on the host with isg_debug_server_inject; no
    GPU fault): the admitted requests with tiles left fail with ISG_ERR_CUDA, every other request
    finishes with its exact table, every arena slot comes back once no step in flight writes into
    it (no admitted request, no open ticket), and the server keeps serving. With lane_model = 0
    the steps carry batch-kernel tiles of 35-spin requests; with the default, task ranges of the
    enumeration kernel (lane tables) of 36-spin ones, several steps each."""
    if lane:
        lats = [w.with_random_couplings(w.square(6, 6, True), w.SplitMix64(60 + k), (-1, 1)) for k in range(4)]
    else:
        lats = [w.with_random_couplings(w.square(5, 7, True), w.SplitMix64(60 + k), (-1, 1)) for k in range(6)]
    srv = isg.Server(max_inflight=2, arena_bytes=1 << 20, step_ms=0.5, lane_model=lane)
    tickets = [(srv.submit(isg.isg_graph_create(l.n, l.edges)), l) for l in lats]
    srv.inject_failure(where)
    failed = 0
    for t, lat in tickets:
        srv.wait(t, 60000)
        try:
            g, _ = srv.result(t)
        except isg.IsgError as e:
            assert e.status == 4 and "injected" in str(e), str(e)
            failed += 1
            continue
        assert np.array_equal(g, alone(isg, lat)), lat.name
    assert failed >= 1
    assert srv.lane_counts()["requests"] == (len(lats) if lane else 0)
    t0 = time.time()
    while (srv.stats()["admitted"] or srv.stats()["tickets"]) and time.time() - t0 < 10:
        time.sleep(0.01)
    st = srv.stats()
    assert st["admitted"] == 0 and st["tickets"] == 0, st
    again = w.square(4, 5, True)
    t = srv.submit(isg.isg_graph_create(again.n, again.edges))
    srv.wait(t, 60000)
    assert np.array_equal(srv.result(t)[0], oracle.g_masks(again.n, again.edges))
    srv.close()

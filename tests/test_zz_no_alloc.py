"""isg_enumerate_noalloc, called through the C ABI, against isg_enumerate.

isg_enumerate_noalloc serves callers that cannot allocate device memory; its scratch is a fixed
array inside the library that every call reuses. The test checks two calls in a row on
different graphs (so the second call sees the first one's leftovers in that array), then the
first graph again, each bit for bit against isg_enumerate. The file is named so that pytest
collects it last."""
import numpy as np
import pytest

from paper_1110_2561_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def test_noalloc_matches_enumerate_on_consecutive_calls(isg, cuda):
    import torch
    graphs = [w.square(6, 6, True),                                                        # N = 36, main kernel
              w.with_random_couplings(w.square(5, 6, True), w.SplitMix64(21), (-2, -1, 1, 2)),  # N = 30, two classes
              w.square(6, 6, True)]
    stream = torch.cuda.current_stream()
    for lat in graphs:
        gh = isg.isg_graph_create(lat.n, lat.edges)
        want = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=cuda)
        isg.isg_enumerate(gh, want, stream)
        got = torch.full(isg.table_shape(gh), -7, dtype=torch.int64, device=cuda)   # overwritten, not added to
        isg.isg_enumerate_noalloc(gh, got, stream)
        torch.cuda.synchronize()
        assert torch.equal(got, want), lat.name
        assert int(got.sum().item()) == 1 << lat.n


def test_noalloc_small_graph_and_accumulate(isg, cuda):
    import torch
    lat = w.with_random_couplings(w.triangular(3, 3, True), w.SplitMix64(22), (-1, 1))   # N = 9: small kernel
    gh = isg.isg_graph_create(lat.n, lat.edges)
    want = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=cuda)
    isg.isg_enumerate(gh, want)
    got = torch.zeros_like(want)
    isg.isg_enumerate_noalloc(gh, got, shard_bits=1, shard_lo=0, shard_hi=1)
    isg.isg_enumerate_noalloc(gh, got, shard_bits=1, shard_lo=1, shard_hi=2, accumulate=1)
    torch.cuda.synchronize()
    assert torch.equal(got, want)


def test_noalloc_honours_a_cached_autotune_choice(isg, cuda):
    """autotune = 1 applies the choice isg_autotune cached for the graph (no timing inside the call,
    since timing allocates); on a graph never tuned it falls back to the planner's defaults. Both
    give isg_enumerate's table."""
    import torch
    lat = w.square(6, 6, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    isg.isg_autotune(gh)
    want = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=cuda)
    isg.isg_enumerate(gh, want, autotune=1)
    got = torch.full(isg.table_shape(gh), 3, dtype=torch.int64, device=cuda)
    isg.isg_enumerate_noalloc(gh, got, autotune=1)
    fresh = w.with_random_couplings(w.square(5, 6, True), w.SplitMix64(23), (-1, 1))
    gf = isg.isg_graph_create(fresh.n, fresh.edges)
    want_f = torch.zeros(isg.table_shape(gf), dtype=torch.int64, device=cuda)
    isg.isg_enumerate(gf, want_f)
    got_f = torch.zeros_like(want_f)
    isg.isg_enumerate_noalloc(gf, got_f, autotune=1)
    torch.cuda.synchronize()
    assert torch.equal(got, want) and torch.equal(got_f, want_f)
    isg.isg_device_status()

"""One graph over two ranks on the GPU: two processes share the box's one GPU (their kernels are
independent launches that never wait on each other), each enumerates its share of the 6x6
torus's 2^36 configurations with isg_enumerate_rank into a CUDA table, and enumerate_distributed's
all-reduce (gloo, staged through host memory) sums them. Rank 0 compares the sum bin for bin with
the oracle's frontier programme, in the whole and the half-and-mirror forms."""
import os
import socket

import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, result_path, symmetric):
    import sys
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1110_2561_gb300 import isg, workloads as w
    lat = w.square(6, 6, True)
    g = isg.isg_graph_create(lat.n, lat.edges)
    out = torch.full(isg.table_shape(g), -1, dtype=torch.int64, device="cuda:0")
    isg.enumerate_distributed(g, out, symmetry=int(symmetric))
    isg.isg_device_status()
    if rank == 0:
        import oracle
        ref = oracle.g_frontier(lat.n, lat.edges, max_active=16)
        with open(result_path, "w") as f:
            f.write("ok" if np.array_equal(out.cpu().numpy(), ref) else "mismatch")
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("symmetric", [False, True], ids=["whole", "half-and-mirror"])
def test_two_ranks_on_one_gpu_sum_to_the_oracle(tmp_path, isg, cuda, symmetric):
    import oracle
    oracle.build()
    out = str(tmp_path / "result.txt")
    mp.start_processes(_rank_main, args=(2, _free_port(), out, symmetric), nprocs=2, join=True, start_method="spawn")
    assert open(out).read() == "ok"


def test_rank_shares_edge_cases(isg, cuda):
    """isg_enumerate_rank on one process: the W shares of a graph (W = 1, 3, 5, and more ranks than
    shards) summed on the device, added with accumulate into one table, host and device outputs,
    with and without symmetry: all equal the oracle; a rank beyond the shard count writes zeros."""
    import numpy as np
    import torch
    import oracle
    from paper_1110_2561_gb300 import workloads as w
    lat = w.with_random_couplings(w.triangular(4, 5, True), w.SplitMix64(44), (-2, -1, 1, 2))
    g = isg.isg_graph_create(lat.n, lat.edges)
    ref = oracle.g_masks(lat.n, lat.edges)
    for W in (1, 3, 5):
        for sym in (0, 1):
            acc = torch.zeros(isg.table_shape(g), dtype=torch.int64, device=cuda)
            host = np.zeros(isg.table_shape(g), dtype=np.int64)
            for r in range(W):
                isg.isg_enumerate_rank(g, r, W, acc, symmetry=sym, accumulate=1)
                host += isg.isg_enumerate_rank(g, r, W, symmetry=sym)
            torch.cuda.synchronize()
            assert np.array_equal(acc.cpu().numpy(), ref), (W, sym)
            assert np.array_equal(host, ref), (W, sym)
    tiny = w.ring(3)                                       # 3 spins: 8 shards at most
    gt = isg.isg_graph_create(tiny.n, tiny.edges)
    parts = [isg.isg_enumerate_rank(gt, r, 16) for r in range(16)]
    assert sum(int(p.sum()) == 0 for p in parts) >= 8
    assert np.array_equal(sum(parts), oracle.g_edges(tiny.n, tiny.edges))
    with pytest.raises(isg.IsgError) as ei:
        isg.isg_enumerate_rank(g, 3, 3)
    assert ei.value.status == 1
    isg.isg_device_status()

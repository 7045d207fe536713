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

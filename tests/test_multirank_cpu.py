"""Sharding across ranks on the CPU (gloo, world size 2): each rank enumerates its shard of the
configuration space with the host emulation of the GPU walk (the same planner and program as the
CUDA kernels), the int64 tables are summed with an all-reduce, and the sum equals the oracle's
full table. This is the exchange a multi-GPU run of one large graph would make."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, result_path, symmetric=False):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1110_2561_gb300 import isg, workloads as w
    import oracle
    lat = w.with_random_couplings(w.triangular(4, 4, True), w.SplitMix64(77), (-2, -1, 1, 2))
    g = isg.isg_graph_create(lat.n, lat.edges)
    shard_bits = 3                                   # 8 shards dealt round-robin to the ranks
    # symmetric: only the shards with spin N-1 up (the top shard bit), the rest from the mirror
    first = (1 << (shard_bits - 1)) if symmetric else 0
    part = np.zeros(isg.table_shape(g), dtype=np.int64)
    for shard in range(first + rank, 1 << shard_bits, world):
        part += isg.isg_debug_emulate(g, shard_bits=shard_bits, shard_lo=shard, shard_hi=shard + 1)
    t = torch.from_numpy(part)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        whole = t.numpy()
        if symmetric:                                # the global flip maps (E, M) to (E, -M)
            whole = whole + whole[:, ::-1]
        ok = np.array_equal(whole, oracle.g_masks(lat.n, lat.edges))
        with open(result_path, "w") as f:
            f.write("ok" if ok else "mismatch")
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("symmetric", [False, True], ids=["whole", "half-and-mirror"])
def test_two_rank_shards_sum_to_the_whole(tmp_path, isg, symmetric):
    """Whole: all 8 shards over the two ranks. Half-and-mirror: only the 4 shards with spin N-1 up,
    summed, then completed by the M -> -M mirror (the symmetry halving of a multi-GPU run)."""
    import oracle
    oracle.build()
    out = str(tmp_path / "result.txt")
    mp.start_processes(_rank_main, args=(2, _free_port(), out, symmetric), nprocs=2, join=True, start_method="spawn")
    assert open(out).read() == "ok"

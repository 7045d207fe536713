"""One graph over several ranks on the CPU (gloo, world sizes 2 and 3): each rank runs the host
emulation of isg_enumerate_rank -- its share of the configuration space from isg_rank_shards,
walked by the same planner and program as the CUDA kernels, optionally the spin-(N-1)-up half
with its mirror -- and one int64 all-reduce of the tables gives the oracle's full table. This is
the exchange of a multi-GPU run of one large graph (the paper's outer-loop split over processes
with a gather at the root, Sec. 3d)."""
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


def _rank_main(rank, world, port, result_path, symmetric):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1110_2561_gb300 import isg, workloads as w
    import oracle
    lat = w.with_random_couplings(w.triangular(4, 4, True), w.SplitMix64(77), (-2, -1, 1, 2))
    g = isg.isg_graph_create(lat.n, lat.edges)
    part = isg.isg_debug_emulate_rank(g, rank, world, symmetry=int(symmetric))
    bits, lo, hi = isg.isg_rank_shards(lat.n, rank, world, symmetric)
    shares = [None] * world
    dist.all_gather_object(shares, (bits, lo, hi))
    t = torch.from_numpy(part)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        # the ranks' shares tile the space (or its upper half) without gaps or overlaps
        first = (1 << (bits - 1)) if symmetric else 0
        tiled = all(shares[r][2] == shares[r + 1][1] for r in range(world - 1)) and \
            shares[0][1] == first and shares[-1][2] == 1 << bits
        ok = tiled and np.array_equal(t.numpy(), oracle.g_masks(lat.n, lat.edges))
        with open(result_path, "w") as f:
            f.write("ok" if ok else f"mismatch (tiled={tiled})")
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("symmetric", [False, True], ids=["whole", "half-and-mirror"])
def test_ranks_sum_to_the_whole(tmp_path, isg, world, symmetric):
    """Whole: every configuration over the ranks. Half-and-mirror: each rank its shards of the
    spin-(N-1)-up half plus their M -> -M mirror; the all-reduced sum is again the full table."""
    import oracle
    oracle.build()
    out = str(tmp_path / "result.txt")
    mp.start_processes(_rank_main, args=(world, _free_port(), out, symmetric), nprocs=world, join=True,
                       start_method="spawn")
    assert open(out).read() == "ok"

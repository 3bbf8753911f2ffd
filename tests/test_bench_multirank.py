"""The bench's multi-rank logic on CPU with the gloo backend (world size 2):
whole-job time is the slowest rank's, units are summed over ranks, replicas
trace distinct fields, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 10 (r + 1) ms for 100 (r + 1) units
        ms, units = bench.reduce_timing(torch, 10.0 * (rank + 1), 100 * (rank + 1), world, "cpu")
        out[rank] = (ms, units, bench.replica_seed(bench.FIELD_SEED, rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_reduce_timing_and_replica_seeds_two_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert set(out.keys()) == {0, 1}
    for r in range(world):
        ms, units, _ = out[r]
        assert ms == 20.0          # the slowest rank
        assert units == 300.0      # all ranks' units
    assert out[0][2] != out[1][2]  # each replica its own field


def test_reduce_timing_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_timing(torch, 12.5, 7, 1, "cpu") == (12.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Ranks other than 0 return at once, before reading arguments or loading
    the oracle."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.run_reference(None, 1, 2) is None

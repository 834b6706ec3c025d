"""The multi-GPU path of the benchmark, on CPU: two gloo ranks (no GPU).

The map shards without any exchange (independent particles, the planet
ephemeris recomputed per rank), so the only cross-rank logic is host-side:
every rank draws its own seeded replica of the workload, and the timing is
reduced as max over ranks of the timed milliseconds and the sum over ranks of
particle-steps (weak scaling)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    import glisse_inputs as gi

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = gi.WORKLOADS["tiny"]
    parts = bench.replica_particles(w, rank)
    # each rank reports its own fake timing and work; the reduction must give max / sum
    ms, steps = bench.reduce_over_ranks(10.0 + 5.0 * rank, 1000.0 * (rank + 1))
    dist.barrier()
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.concatenate([[ms, steps], parts[:4].ravel()]))
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert r0[0] == r1[0] == 15.0          # max over ranks of the timed milliseconds
    assert r0[1] == r1[1] == 3000.0        # sum over ranks of particle-steps
    assert not np.array_equal(r0[2:], r1[2:])  # independent replicas per rank
    import glisse_inputs as gi

    np.testing.assert_array_equal(r0[2:], gi.make("tiny")["particles"][:4].ravel())  # rank 0 = the workload


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(12.5, 77.0) == (12.5, 77.0)

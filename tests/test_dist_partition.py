"""Multi-rank partitioning of the sampling workload, on CPU ranks (gloo).

Configurations are independent, so N ranks sample disjoint prior-counter
ranges (bench.counter_base) and each runs its own chain: no data-path
collective, only the max-over-ranks of the timed region.  Two gloo ranks on
127.0.0.1 check that the ranks' configurations are exactly the single-process
configurations at the shifted counters (no overlap, nothing missing) and that
the timing reduction returns the slowest rank.
"""
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
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import gf_inputs as gi
    import oracle
    r, w, _ = bench.dist_setup(world)
    assert (r, w) == (rank, world)
    shape = gi.FlowShape(2, 4, 2, 8, 8)
    wts = gi.init_weights(shape)
    B = 3
    o = oracle.flow_sample(shape, wts, -4.0, 8.0, B, seed=11, counter0=bench.counter_base(rank), nthreads=1)
    np.save(os.path.join(out_dir, f"phi{rank}.npy"), o["phi"])
    t = bench.max_over_ranks(float(rank + 1) * 1.5, world)
    np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([t]))
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_rank_partition(tmp_path):
    import bench
    import gf_inputs as gi
    import oracle
    oracle.build()
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    shape = gi.FlowShape(2, 4, 2, 8, 8)
    wts = gi.init_weights(shape)
    for rank in range(world):
        got = np.load(tmp_path / f"phi{rank}.npy")
        ref = oracle.flow_sample(shape, wts, -4.0, 8.0, 3, seed=11, counter0=bench.counter_base(rank), nthreads=1)
        assert np.array_equal(got, ref["phi"])
        assert float(np.load(tmp_path / f"t{rank}.npy")[0]) == 3.0      # max over ranks
    a, b = np.load(tmp_path / "phi0.npy"), np.load(tmp_path / "phi1.npy")
    assert not np.isclose(a[:, None, :], b[None, :, :]).all(axis=2).any()   # disjoint draws
    assert bench.counter_base(1) - bench.counter_base(0) >= 2**40

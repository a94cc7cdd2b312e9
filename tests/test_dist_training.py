"""Data-parallel training and the gathered global MH chain on CPU ranks (gloo).

The product's data-parallel step (paper_2208_08903_gb300.distributed.dp_step:
batch partition by prior counters, weighted all-reduce of loss and gradient,
identical optimiser update on every rank) is driven with the oracle's FP64
loss gradient as the per-rank gradient provider (the GPU provider is
gf_flow_train_step; this machine has no GPU).  Checks, for 2 and 3 ranks and
a batch that does not divide evenly:

- the all-reduced gradient equals the single-process gradient of the whole
  batch (Sec. 1, shifted reverse KL loss: the mean over configurations);
- after an Adam step (Sec. 3) every rank holds the same weights, equal to the
  single-process update;
- log-weights gathered to rank 0 come back in global proposal order and the
  MH chain over them (Sec. 1, MH test) equals the single-process chain.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPE_ARGS = (2, 4, 3, 4, 4)
M2, LAM, SEED, C0 = -4.0, 8.0, 21, 1000


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, B, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import gf_inputs as gi
    import oracle
    from paper_2208_08903_gb300 import distributed as D
    shape = gi.FlowShape(*SHAPE_ARGS)
    w = gi.init_weights(shape, seed=3)
    m = np.zeros_like(w)
    v = np.zeros_like(w)

    def grad_fn(n, c0):
        z = oracle.prior(shape.V, n, SEED, c0, f32=True)
        loss, g = oracle.flow_loss_grad(shape, w, M2, LAM, z, nthreads=1)
        return torch.tensor([loss], dtype=torch.float64), torch.tensor(g, dtype=torch.float64)

    applied = {}

    def apply_fn(g):
        gg = g.numpy().copy()
        applied["g"] = gg
        oracle.adam(w, gg, m, v, 1, 1e-3)

    loss = D.dp_step(grad_fn, apply_fn, B, C0)
    np.save(os.path.join(out_dir, f"g{rank}.npy"), applied["g"])
    np.save(os.path.join(out_dir, f"w{rank}.npy"), w)
    np.save(os.path.join(out_dir, f"loss{rank}.npy"), loss.numpy())

    # log-weights of this rank's proposals, gathered to rank 0 in global order
    off, n = D.partition(B, world, rank)
    o = oracle.flow_sample(shape, w, M2, LAM, n, seed=SEED + 1, counter0=off, nthreads=1)
    full = D.gather_logw(torch.tensor(o["logw"]), B, dst=0)
    if rank == 0:
        np.save(os.path.join(out_dir, "logw_gathered.npy"), full.numpy())
    else:
        assert full is None
    dist.barrier()
    dist.destroy_process_group()


def test_partition_covers_batch_once():
    from paper_2208_08903_gb300.distributed import partition
    for B in (1, 5, 7, 64, 1000):
        for world in (1, 2, 3, 8):
            if world > B:
                continue
            spans = [partition(B, world, r) for r in range(world)]
            assert spans[0][0] == 0 and sum(c for _, c in spans) == B
            for (o1, c1), (o2, _) in zip(spans, spans[1:]):
                assert o1 + c1 == o2
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1


@pytest.mark.parametrize("world,B", [(2, 5), (3, 7)])
def test_dp_step_equals_single_process(tmp_path, world, B):
    import gf_inputs as gi
    import oracle
    oracle.build()
    mp.start_processes(_worker, args=(world, _free_port(), B, str(tmp_path)), nprocs=world, start_method="spawn")
    shape = gi.FlowShape(*SHAPE_ARGS)
    w0 = gi.init_weights(shape, seed=3)
    z = oracle.prior(shape.V, B, SEED, C0, f32=True)
    loss_ref, g_ref = oracle.flow_loss_grad(shape, w0, M2, LAM, z, nthreads=1)
    w_ref = w0.copy()
    oracle.adam(w_ref, g_ref.copy(), np.zeros_like(w0), np.zeros_like(w0), 1, 1e-3)
    for r in range(world):
        g = np.load(tmp_path / f"g{r}.npy")
        assert np.allclose(g, g_ref, rtol=1e-12, atol=1e-14 * np.abs(g_ref).max())
        assert float(np.load(tmp_path / f"loss{r}.npy")[0]) == pytest.approx(loss_ref, rel=1e-13)
        assert np.array_equal(np.load(tmp_path / f"w{r}.npy"), np.load(tmp_path / "w0.npy"))
        assert np.allclose(np.load(tmp_path / f"w{r}.npy"), w_ref, rtol=0, atol=1e-12)
    # the gathered log-weights are the single-process batch, and so is the chain
    o = oracle.flow_sample(shape, np.load(tmp_path / "w0.npy"), M2, LAM, B, seed=SEED + 1, counter0=0, nthreads=1)
    lw = np.load(tmp_path / "logw_gathered.npy")
    assert np.array_equal(lw, o["logw"])
    st_a, st_b = oracle.new_mh_state(9), oracle.new_mh_state(9)
    ia, aa = oracle.mh_chain(st_a, lw)
    ib, ab = oracle.mh_chain(st_b, o["logw"])
    assert np.array_equal(ia, ib) and np.array_equal(aa, ab)

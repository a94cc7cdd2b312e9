"""GPU parity of the reverse-KL training step against the FP64 oracle.

The oracle's gradient is itself pinned by central finite differences on the
CPU; here the GPU FP32 gradient must match it (tolerance in assert_grad_close).
"""
import numpy as np
import pytest

import gf_inputs as gi
from gpu_util import assert_grad_close, assert_logw_close, require_gpu

pytestmark = pytest.mark.gpu


CASES = [
    (gi.FlowShape(2, 8, 4, 8, 8), -4.0, 8.0, 16),
    (gi.FlowShape(2, 6, 3, 16, 16), -1.0, 2.0, 5),
    (gi.FlowShape(3, 4, 3, 8, 8), -6.0, 5.0, 6),
    (gi.FlowShape(2, 4, 4, 8, 8, use_final_tanh=False), 0.5, 1.0, 3),
    (gi.FlowShape(2, 32, 24, 32, 32), -4.0, 8.0, 3),          # c2 shape, small batch
    (gi.FlowShape(3, 8, 4, 32, 32), -6.0, 5.0, 2),            # 3D, C=32
    (gi.FlowShape(2, 8, 3, 24, 24), -4.0, 8.0, 4),            # hidden width 24 (serving mix)
    (gi.FlowShape(3, 16, 3, 32, 32), -6.0, 5.0, 2),           # 3D L=16 C=32: fused forward pass
]


@pytest.mark.parametrize("case", CASES, ids=[f"d{c[0].nd}L{c[0].L}N{c[0].n_layers}C{c[0].c1}B{c[3]}" for c in CASES])
def test_loss_and_gradient_match_oracle(orc, case):
    torch, P = require_gpu()
    shape, m2, lam, B = case
    w = gi.init_weights(shape, seed=1)
    flow = P.Flow(shape, w)
    z = orc.prior(shape.V, B, seed=3, counter0=0, f32=True)
    zt = torch.tensor(z, dtype=torch.float32, device="cuda")
    loss, g = flow.train_step(B, (m2, lam), z=zt)
    torch.cuda.synchronize()
    ref_loss, ref_g = orc.flow_loss_grad(shape, w, m2, lam, z)
    assert_logw_close(loss.cpu().numpy(), [ref_loss], what="loss")
    assert_grad_close(g.cpu().numpy(), ref_g)
    # in-kernel prior gives the same z as the sampler for the same (seed, counter0)
    loss2, _ = flow.train_step(B, (m2, lam), seed=3, counter0=0)
    assert_logw_close(loss2.cpu().numpy(), [ref_loss], what="loss (in-kernel prior)")
    assert P.device_status() == 0


def test_gradient_is_deterministic_and_adam_matches_oracle(orc):
    torch, P = require_gpu()
    shape = gi.FlowShape(2, 8, 4, 8, 8)
    w = gi.init_weights(shape, seed=2)
    flow = P.Flow(shape, w)
    _, g1 = flow.train_step(32, (-4.0, 8.0), seed=5)
    _, g2 = flow.train_step(32, (-4.0, 8.0), seed=5)
    assert torch.equal(g1, g2)
    m = torch.zeros(flow.n_params, device="cuda")
    v = torch.zeros(flow.n_params, device="cuda")
    w0 = flow.get_weights().cpu().numpy().astype(np.float64)
    for t in (1, 2):
        _, g = flow.train_step(32, (-4.0, 8.0), seed=5 + t, lr=1e-3, adam_m=m, adam_v=v, adam_t=t)
        gn = g.cpu().numpy().astype(np.float64)
        mm = np.zeros_like(w0) if t == 1 else mm
        vv = np.zeros_like(w0) if t == 1 else vv
        orc.adam(w0, gn, mm, vv, t, 1e-3)
        w1 = flow.get_weights().cpu().numpy()
        assert np.allclose(w1, w0, rtol=1e-6, atol=1e-7)
        w0 = w1.astype(np.float64)
    # the updated weights are the ones the sampler uses
    ref = orc.flow_sample(shape, w0, -4.0, 8.0, 4, seed=9)
    out = flow.sample(4, seed=9, phi4=(-4.0, 8.0))
    assert_logw_close(out.logw.cpu().numpy(), ref["logw"])


def test_c2_full_batch_properties():
    """2D L=32, 24 couplings, C=32, batch 1024: loss equals the sampler's mean
    log q + S on the same z, and the gradient is the mean of sub-batch gradients."""
    torch, P = require_gpu()
    W = gi.WORKLOADS["c2"]
    shape, phi4, B = W["shape"], W["phi4"], W["batch"]
    flow = P.Flow(shape, gi.init_weights(shape))
    loss, g = flow.train_step(B, phi4, seed=4, counter0=0)
    out = flow.sample(B, seed=4, counter0=0, phi4=phi4)
    mean = (out.logq + out.S).mean().item()
    assert abs(loss.item() - mean) <= 1e-4 * max(abs(mean), 1.0)
    parts = []
    for k in range(4):
        _, gk = flow.train_step(B // 4, phi4, seed=4, counter0=k * (B // 4))
        parts.append(gk.double())
    gm = sum(parts) / 4
    rel = (torch.linalg.norm(g.double() - gm) / torch.linalg.norm(gm)).item()
    assert rel < 1e-4, rel
    assert torch.isfinite(g).all()


def test_training_lowers_the_loss():
    """A short Adam run on the paper's example shape lowers the reverse-KL loss."""
    torch, P = require_gpu()
    W = gi.WORKLOADS["c1"]
    shape, phi4 = W["shape"], W["phi4"]
    flow = P.Flow(shape, gi.init_weights(shape))
    m = torch.zeros(flow.n_params, device="cuda")
    v = torch.zeros(flow.n_params, device="cuda")
    ws = torch.empty(flow.train_workspace_bytes(64), device="cuda", dtype=torch.uint8)
    losses = []
    for t in range(1, 301):
        loss, _ = flow.train_step(64, phi4, seed=12345, counter0=64 * t, lr=1e-3, adam_m=m, adam_v=v,
                                  adam_t=t, workspace=ws, grad=False)
        losses.append(loss.item())
    first, last = np.mean(losses[:20]), np.mean(losses[-20:])
    assert last < first - 0.1 * abs(first), (first, last)


def test_checkpoint_resume_continues_bit_for_bit(tmp_path):
    torch, P = require_gpu()
    from paper_2208_08903_gb300 import train as T
    shape, phi4 = gi.FlowShape(2, 8, 4, 8, 8), (-4.0, 8.0)
    fa = P.Flow(shape, gi.init_weights(shape, seed=0))
    sa = T.train(fa, phi4, 2, 5, 16, seed=3)
    fb = P.Flow(shape, gi.init_weights(shape, seed=0))
    sb = T.train(fb, phi4, 1, 5, 16, seed=3)
    path = str(tmp_path / "ck.npz")
    T.save_checkpoint(path, fb, sb, note="half")
    fc = P.Flow(shape, gi.init_weights(shape, seed=99))          # different start: overwritten
    sc, meta = T.load_checkpoint(path, fc)
    assert meta == {"note": "half"} and sc.step == 5
    sc = T.train(fc, phi4, 1, 5, 16, seed=3, state=sc)
    assert torch.equal(fa.get_weights(), fc.get_weights())
    assert sa.losses == sc.losses and torch.equal(sa.adam_m, sc.adam_m) and torch.equal(sa.adam_v, sc.adam_v)
    other = P.Flow(gi.FlowShape(2, 8, 2, 8, 8), gi.init_weights(gi.FlowShape(2, 8, 2, 8, 8), seed=0))
    with pytest.raises(ValueError):
        T.load_checkpoint(path, other)


def test_lr_schedule_and_evaluation():
    torch, P = require_gpu()
    from paper_2208_08903_gb300 import train as T
    shape, phi4 = gi.FlowShape(2, 8, 4, 8, 8), (-4.0, 8.0)
    f = P.Flow(shape, gi.init_weights(shape, seed=0))
    w0 = f.get_weights().clone()
    T.train(f, phi4, 1, 3, 16, lr_schedule=lambda step: 0.0)       # zero rate: no update
    assert torch.equal(w0, f.get_weights())
    T.train(f, phi4, 1, 3, 16, lr_schedule=lambda step: 1e-3 * 0.5 ** step)
    assert not torch.equal(w0, f.get_weights())
    ev = {k: T.evaluate(f, phi4, 1000, 256, seed=4, sampler=k) for k in ("fused", "unfused")}
    for e in ev.values():
        assert 0.0 <= e["acceptance"] <= 1.0 and 0.0 < e["ess"] <= 1.0 and e["abs_M"] >= 0.0
    # same proposals through the fused and the plain sampler: same chain up to near ties
    assert abs(ev["fused"]["acceptance"] - ev["unfused"]["acceptance"]) <= 2 / 999


def test_data_parallel_step_on_one_rank_equals_fused_step():
    """distributed.dp_train_step without a process group (one rank): the
    gradient of gf_flow_train_step (lr = 0) applied by gf_flow_adam_step gives
    bit for bit the weights of gf_flow_train_step with lr > 0."""
    torch, P = require_gpu()
    from paper_2208_08903_gb300 import distributed as D
    shape = gi.FlowShape(2, 8, 4, 8, 8)
    w = gi.init_weights(shape, seed=7)
    fa, fb = P.Flow(shape, w), P.Flow(shape, w)
    ma, va = torch.zeros(fa.n_params, device="cuda"), torch.zeros(fa.n_params, device="cuda")
    mb, vb = torch.zeros(fb.n_params, device="cuda"), torch.zeros(fb.n_params, device="cuda")
    for t in (1, 2, 3):
        la, _ = fa.train_step(96, (-4.0, 8.0), seed=3, counter0=96 * t, lr=1e-3, adam_m=ma, adam_v=va, adam_t=t,
                              grad=False)
        lb = D.dp_train_step(fb, (-4.0, 8.0), 96, seed=3, counter0=96 * t, lr=1e-3, adam_m=mb, adam_v=vb, adam_t=t)
        assert float(la.item()) == float(lb.item())
    assert torch.equal(fa.get_weights(), fb.get_weights())
    assert torch.equal(ma, mb) and torch.equal(va, vb)
    assert P.device_status() == 0

"""GPU parity of the two training halves and their torch.autograd front end.

The reverse-KL gradient assembled through autograd (forward half, action,
mean, backward half, action VJP) must match the FP64 oracle's gradient with the
tolerance of the fused training step, and the fused step's own gradient up to
FP32 rounding order.  The backward half is linear in its two upstream
gradients; the action VJP equals gS times the oracle force.
"""
import numpy as np
import pytest

import gf_inputs as gi
from gpu_util import assert_grad_close, assert_logw_close, assert_sites_close, require_gpu

pytestmark = pytest.mark.gpu

CASES = [
    (gi.FlowShape(2, 8, 4, 8, 8), -4.0, 8.0, 16),
    (gi.FlowShape(3, 4, 3, 8, 8), -6.0, 5.0, 6),
    (gi.FlowShape(2, 32, 6, 32, 32), -4.0, 8.0, 4),
]
IDS = [f"d{c[0].nd}L{c[0].L}N{c[0].n_layers}C{c[0].c1}B{c[3]}" for c in CASES]


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_autograd_gradient_matches_oracle_and_fused_step(orc, case):
    torch, P = require_gpu()
    from paper_2208_08903_gb300 import autograd as AG
    shape, m2, lam, B = case
    w = gi.init_weights(shape, seed=1)
    flow = P.Flow(shape, w)
    z = orc.prior(shape.V, B, seed=3, counter0=0, f32=True)
    zt = torch.tensor(z, dtype=torch.float32, device="cuda")
    theta = flow.get_weights().clone().requires_grad_(True)
    loss = AG.reverse_kl_loss(flow, theta, B, (m2, lam), z=zt)
    loss.backward()
    torch.cuda.synchronize()
    ref_loss, ref_g = orc.flow_loss_grad(shape, w, m2, lam, z)
    assert_logw_close(loss.detach().cpu().numpy().reshape(1), [ref_loss], what="loss")
    g_auto = theta.grad.cpu().numpy()
    assert_grad_close(g_auto, ref_g)
    loss_f, g_f = flow.train_step(B, (m2, lam), z=zt)
    torch.cuda.synchronize()
    assert abs(loss_f.item() - loss.item()) <= 1e-9 * max(abs(loss.item()), 1.0)
    assert rel_l2(g_auto, g_f.cpu().numpy()) <= 1e-5


def test_forward_half_matches_sampler(orc):
    torch, P = require_gpu()
    shape, B = gi.FlowShape(2, 8, 4, 8, 8), 9
    w = gi.init_weights(shape, seed=2)
    flow = P.Flow(shape, w)
    phi, logq, _ = flow.forward_train(B, seed=5, counter0=17)
    ref = orc.flow_sample(shape, w, -4.0, 8.0, B, seed=5, counter0=17)
    torch.cuda.synchronize()
    assert_sites_close(phi.cpu().numpy(), ref["phi"])
    assert_logw_close(logq.cpu().numpy(), ref["logq"], what="logq")


def test_backward_half_is_linear_in_upstream_gradients(orc):
    torch, P = require_gpu()
    shape, B = gi.FlowShape(2, 8, 4, 8, 8), 7
    flow = P.Flow(shape, gi.init_weights(shape, seed=4))
    gen = torch.Generator(device="cuda").manual_seed(11)
    gphi = torch.randn(B, shape.V, device="cuda", generator=gen)
    glq = torch.randn(B, device="cuda", generator=gen, dtype=torch.float64)

    def grad(gp, gq):
        _, _, ws = flow.forward_train(B, seed=1)
        return flow.backward(B, gp, gq, ws).cpu().numpy().astype(np.float64)

    both = grad(gphi, glq)
    only_phi = grad(gphi, None)
    only_lq = grad(None, glq)
    assert rel_l2(only_phi + only_lq, both) <= 1e-5
    # scaling the upstream gradient scales the result exactly (powers of two)
    assert np.array_equal(grad(gphi * 2, glq * 2), 2 * both)
    assert not np.any(grad(None, None))


@pytest.mark.parametrize("nd,L", [(2, 8), (3, 4), (3, 16)])
def test_action_vjp_matches_oracle_force(orc, nd, L):
    torch, P = require_gpu()
    V, B, m2, lam = L**nd, 5, -4.0, 8.0
    phi = (orc.prior(V, B, seed=8, counter0=0, f32=True) * 0.7).astype(np.float32).astype(np.float64)
    gS = np.linspace(-1.5, 2.0, B)
    out = P.phi4_action_vjp(nd, L, (m2, lam), torch.tensor(phi, dtype=torch.float32, device="cuda"),
                            torch.tensor(gS, device="cuda"))
    torch.cuda.synchronize()
    ref = orc.force(nd, L, m2, lam, phi) * gS[:, None]
    # FP64 arithmetic rounded once to FP32: half an FP32 ulp of the result
    assert_sites_close(out.cpu().numpy(), ref, rtol=2 ** -23, what="action vjp")


def test_autograd_adam_loop_lowers_the_loss(orc):
    torch, P = require_gpu()
    from paper_2208_08903_gb300 import autograd as AG
    shape, m2, lam, B = gi.FlowShape(2, 8, 4, 8, 8), -4.0, 8.0, 64
    flow = P.Flow(shape, gi.init_weights(shape, seed=0))
    theta = flow.get_weights().clone().requires_grad_(True)
    opt = torch.optim.Adam([theta], lr=1e-3)
    losses = []
    for it in range(60):
        opt.zero_grad()
        loss = AG.reverse_kl_loss(flow, theta, B, (m2, lam), seed=9, counter0=it * B)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert np.mean(losses[-10:]) < np.mean(losses[:10])

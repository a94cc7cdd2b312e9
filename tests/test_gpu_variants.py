"""GPU parity of the general s/t network (paper Sec. 3, model parameters
hidden_sizes and kernel_size) against the FP64 oracle.

Networks other than two equal hidden widths in {8, 16, 32} with kernel size 3
run on the whole-lattice FP32 kernel (gf_flow_variant.cu).  Same tolerances as
the plain FP32 path: 1e-5 relative per site, 1e-4 per log q / S / log w.
"""
import numpy as np
import pytest

import gf_inputs as gi
from gpu_util import assert_logw_close, assert_sites_close, compare_mh, require_gpu

pytestmark = pytest.mark.gpu

SHAPES = [
    # the paper's 2D L=8 example with three hidden layers and kernel size 5
    gi.FlowShape(2, 8, 16, hidden_sizes=(8, 8, 8), ksize=5),
    gi.FlowShape(2, 8, 16, hidden_sizes=(8, 8, 8), ksize=3),
    gi.FlowShape(2, 16, 6, hidden_sizes=(16,), ksize=3, use_final_tanh=False),
    gi.FlowShape(2, 32, 4, hidden_sizes=(4, 12, 4), ksize=3),
    gi.FlowShape(2, 8, 4, hidden_sizes=(), ksize=3),
    gi.FlowShape(2, 6, 4, hidden_sizes=(5, 3), ksize=7),
    gi.FlowShape(3, 8, 4, hidden_sizes=(8, 8), ksize=5),
    gi.FlowShape(3, 4, 6, hidden_sizes=(6, 6, 6, 6), ksize=3),
    gi.FlowShape(2, 8, 6, 8, 16),                      # unequal widths (the two-layer form)
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s.nd}d-L{s.L}-h{list(s.hidden)}-k{s.ksize}")
def test_variant_sample_and_inverse_match_oracle(orc, shape):
    torch, P = require_gpu()
    w = gi.init_weights(shape, seed=11)
    flow = P.Flow(shape, w)
    B = 37                                  # not a multiple of the grid: ragged last wave
    m2, lam = -4.0, 8.0
    out = flow.sample(B, seed=5, counter0=100, phi4=(m2, lam), return_z=True)
    torch.cuda.synchronize()
    assert P.device_status() == 0
    ref = orc.flow_sample(shape, w, m2, lam, B, seed=5, counter0=100)
    assert_sites_close(out.z.cpu().numpy(), ref["z"], rtol=1e-6, what="z")
    assert_sites_close(out.phi.cpu().numpy(), ref["phi"])
    for k in ("logq", "S", "logw"):
        assert_logw_close(getattr(out, k).cpu().numpy(), ref[k], what=k)
    # inverse direction on the GPU's own phi
    z2, lq2 = flow.logq(out.phi, return_z=True)
    zr, lqr = orc.flow_logq(shape, w, out.phi.cpu().numpy().astype(np.float64))
    assert_sites_close(z2.cpu().numpy(), zr, what="z(inverse)")
    assert_logw_close(lq2.cpu().numpy(), lqr, what="logq(inverse)")
    assert P.device_status() == 0


def test_variant_given_z_mh_chain_and_weights_update(orc):
    """Given-z path, an MH chain over the proposals, and new weights through
    gf_flow_set_weights_device (repacked on the device)."""
    torch, P = require_gpu()
    shape = gi.FlowShape(2, 8, 8, hidden_sizes=(8, 8, 8), ksize=5)
    w = gi.scale_head(shape, gi.init_weights(shape, seed=3), 0.05)
    flow = P.Flow(shape, w)
    B = 512
    z = orc.prior(shape.V, B, seed=9, counter0=0, f32=True)
    out = flow.sample(B, phi4=(-4.0, 8.0), z=torch.tensor(z, dtype=torch.float32, device="cuda"))
    ref = orc.flow_sample(shape, w, -4.0, 8.0, B, z=z)
    assert_sites_close(out.phi.cpu().numpy(), ref["phi"])
    st = P.new_mh_state(seed=4)
    idx, acc = P.mh_chain(st, out.logw)
    lw = out.logw.cpu().numpy()
    compare_mh(orc, 4, 0, lw, idx.cpu().numpy(), acc.cpu().numpy(), logw_tol=1e-4)
    assert 0 < acc.cpu().numpy()[1:].sum() < B - 1
    w2 = gi.init_weights(shape, seed=4)
    flow.set_weights(torch.tensor(w2, dtype=torch.float32, device="cuda"))
    out2 = flow.sample(B, phi4=(-4.0, 8.0), z=torch.tensor(z, dtype=torch.float32, device="cuda"))
    ref2 = orc.flow_sample(shape, w2, -4.0, 8.0, B, z=z)
    assert_sites_close(out2.phi.cpu().numpy(), ref2["phi"])
    assert P.device_status() == 0


def test_variant_rejections():
    torch, P = require_gpu()
    shape = gi.FlowShape(2, 8, 2, hidden_sizes=(8, 8, 8), ksize=5)
    flow = P.Flow(shape, gi.init_weights(shape))
    with pytest.raises(P._abi.GFError):          # training is for the two-layer k=3 network only
        flow.train_step(8, (-4.0, 8.0), seed=1, counter0=0, lr=0.0, workspace=torch.empty(256, device="cuda",
                                                                                         dtype=torch.uint8))
    with pytest.raises(P._abi.GFError):          # BF16 only for the slice-cached network form
        P.Flow(shape, gi.init_weights(shape), precision="bf16")
    big = gi.FlowShape(2, 64, 2, hidden_sizes=(32, 32), ksize=5)
    with pytest.raises(P._abi.GFError):          # whole lattice does not fit shared memory
        P.Flow(big, gi.init_weights(big))

"""Equal MH acceptance of the tensor-core sampler and the FP32 sampler on a
trained 3D flow (Sec. 1: flow proposals corrected by the MH test with the
Jacobian; Sec. 3: the training loop).

The flow (3D L=16, m2=-6, lam=5, 16 couplings, hidden 32) was trained with
this package's own reverse-KL step for 15,000 Adam steps at batch 64
(paper_2208_08903_gb300/checkpoints).  The test first trains it 50 steps more
on the GPU (the training step at the 3D workload's shape; learning rate 1e-5,
as the checkpoint carries no Adam moments), then runs the
fused FP32 sampler, the plain one-kernel-per-convolution FP32 sampler and the
tensor-core sampler on the same 65,536 proposals (same prior counters, same
MH uniforms): the two FP32 samplers must make identical decisions, and the
tensor-core sampler's acceptance must agree with theirs within three binomial
standard errors (combined as if independent; the chains share their
proposals, so this is conservative).

A 2-layer flow trained for a few hundred steps reaches an acceptance of about
5e-4 on this 4096-site lattice, which makes any such comparison vacuous; the
trained 16-layer flow reaches about 0.06.
"""
import math
import os

import numpy as np
import pytest

import gf_inputs as gi
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_tensor_core_acceptance_equals_fp32_on_trained_flow():
    torch, P = require_gpu()
    from paper_2208_08903_gb300 import train as T
    W = gi.WORKLOADS["c3"]
    shape, phi4 = W["shape"], W["phi4"]
    w = T.load_weights(os.path.join(T.CHECKPOINT_DIR, "c3_L16_16layers_15k.npz"), shape)
    flow = P.Flow(shape, w)
    st = T.train(flow, phi4, 1, 50, 64, lr=1e-5, seed=777)     # fresh Adam moments: a small step
    assert all(math.isfinite(x) for x in st.losses)
    wt = flow.get_weights().double().cpu().numpy()
    tc = P.Flow(shape, wt, precision="bf16")
    n = 65536
    ev = {k: T.evaluate(f, phi4, n, 4096, seed=31337, sampler=kind, keep_logw=True)
          for k, (f, kind) in {"fused": (flow, "fused"), "unfused": (flow, "unfused"),
                               "tc": (tc, "fused")}.items()}
    # the two FP32 samplers sum in different orders: their log w agree to about
    # 1e-5 relative, so a decision can differ only at a near tie
    assert T.decision_agreement(ev["unfused"], ev["fused"]) > 0.99
    a32, atc = ev["fused"]["acceptance"], ev["tc"]["acceptance"]
    se = math.hypot(ev["fused"]["acceptance_binomial_err"], ev["tc"]["acceptance_binomial_err"])
    print(f"acceptance FP32 {a32:.5f} tensor-core {atc:.5f} (3 sigma {3 * se:.5f}); ESS {ev['fused']['ess']:.5f} "
          f"{ev['tc']['ess']:.5f}; decisions agree {T.decision_agreement(ev['tc'], ev['fused']):.4f}")
    assert a32 > 0.01                    # the comparison is not vacuous
    assert abs(atc - a32) <= 3 * se
    assert P.device_status() == 0

"""GPU parity of the fused coupling-stack kernels against the FP64 oracle.

Calls go through the C ABI (ctypes binding).  Inputs are seeded; expected
values come only from the oracle.  Covers FULL (whole lattice resident) and
RING (slice cache) schedules, 2D and 3D, ragged batches, both directions, the
in-kernel prior, and bench-size batches checked on sampled configurations.
"""
import numpy as np
import pytest

import gf_inputs as gi
from gpu_util import assert_logw_close, assert_sites_close, require_gpu

pytestmark = pytest.mark.gpu

CASES = [
    # (shape, m2, lam, B)
    (gi.WORKLOADS["c1"]["shape"], -4.0, 8.0, 64),                    # paper example, FULL
    (gi.FlowShape(2, 8, 16, 8, 8), -4.0, 8.0, 3),                    # ragged small batch
    (gi.FlowShape(2, 6, 5, 16, 16), -1.0, 2.0, 7),                   # S=6: quads straddle slices
    (gi.FlowShape(2, 2, 4, 8, 8), 0.5, 1.0, 5),                      # smallest 2D lattice
    (gi.FlowShape(3, 2, 4, 8, 8), -6.0, 5.0, 5),                     # smallest 3D lattice
    (gi.FlowShape(3, 4, 6, 16, 16, use_final_tanh=False), -6.0, 5.0, 6),
    (gi.FlowShape(2, 32, 24, 32, 32), -4.0, 8.0, 6),                 # c2 shape, RING
    (gi.FlowShape(3, 16, 16, 32, 32), -6.0, 5.0, 3),                 # c3 shape (3D L=16 C=32 kernel)
    (gi.FlowShape(3, 16, 3, 32, 32, use_final_tanh=False), -2.0, 1.0, 5),   # odd layer count, no tanh
    (gi.FlowShape(2, 64, 12, 16, 16), -3.0, 4.0, 2),                 # large 2D, RING
    (gi.FlowShape(2, 16, 5, 24, 24), -2.0, 3.0, 4),                  # hidden width 24: rotated chunks
    (gi.FlowShape(3, 12, 4, 24, 24, use_final_tanh=False), -5.0, 2.0, 3),   # 3D L=12, width 24, RING
]


def _ids(c):
    s = c[0]
    return f"d{s.nd}L{s.L}N{s.n_layers}C{s.c1}B{c[3]}{'' if s.use_final_tanh else 'lin'}"


@pytest.mark.parametrize("case", CASES, ids=[_ids(c) for c in CASES])
def test_sample_matches_oracle(orc, case):
    torch, P = require_gpu()
    shape, m2, lam, B = case
    w = gi.init_weights(shape, seed=0)
    flow = P.Flow(shape, w)
    seed, c0 = 1234, 77
    out = flow.sample(B, seed=seed, counter0=c0, phi4=(m2, lam), return_z=True)
    torch.cuda.synchronize()
    ref = orc.flow_sample(shape, w, m2, lam, B, seed=seed, counter0=c0)
    # the in-kernel FP32 Box-Muller prior agrees with the oracle's to a few ulp
    assert_sites_close(out.z.cpu().numpy(), ref["z"], rtol=1e-6, what="z")
    # flow outputs from the GPU's own prior sample
    assert_sites_close(out.phi.cpu().numpy(), ref["phi"])
    assert_logw_close(out.logq.cpu().numpy(), ref["logq"], what="logq")
    assert_logw_close(out.S.cpu().numpy(), ref["S"], what="S")
    assert_logw_close(out.logw.cpu().numpy(), ref["logw"], what="logw")
    assert P.device_status() == 0


@pytest.mark.parametrize("case", CASES[:2] + CASES[5:8], ids=[_ids(c) for c in CASES[:2] + CASES[5:8]])
def test_given_z_and_inverse_match_oracle(orc, case):
    torch, P = require_gpu()
    shape, m2, lam, B = case
    w = gi.init_weights(shape, seed=3)
    flow = P.Flow(shape, w)
    z = orc.prior(shape.V, B, seed=5, counter0=0, f32=True)
    zt = torch.tensor(z, dtype=torch.float32, device="cuda")
    out = flow.sample(B, phi4=(m2, lam), z=zt)
    ref = orc.flow_sample(shape, w, m2, lam, B, z=z)
    assert_sites_close(out.phi.cpu().numpy(), ref["phi"])
    assert_logw_close(out.logq.cpu().numpy(), ref["logq"], what="logq")
    # trivialising direction on the GPU's phi, against the oracle on the same phi
    zb, lq = flow.logq(out.phi, return_z=True)
    phi64 = out.phi.cpu().numpy().astype(np.float64)
    zr, lqr = orc.flow_logq(shape, w, phi64)
    assert_sites_close(zb.cpu().numpy(), zr, what="z(inverse)")
    assert_logw_close(lq.cpu().numpy(), lqr, what="logq(inverse)")
    # round trip: F(F^-1(z)) = z within the FP32 tolerance
    assert_sites_close(zb.cpu().numpy(), z, what="round trip")
    assert_logw_close(lq.cpu().numpy(), out.logq.cpu().numpy(), what="logq consistency")


def test_identity_flow_is_exact(orc):
    torch, P = require_gpu()
    shape = gi.WORKLOADS["c1"]["shape"]
    w = gi.zero_head(shape, gi.init_weights(shape))
    flow = P.Flow(shape, w)
    out = flow.sample(9, seed=3, phi4=(-4.0, 8.0), return_z=True)
    assert torch.equal(out.phi, out.z)
    ref = orc.log_prior(out.z.cpu().numpy().astype(np.float64))
    assert_logw_close(out.logq.cpu().numpy(), ref, rtol=1e-12, what="log r")


def test_batch_position_independence():
    """Configuration b of (seed, counter0) equals configuration 0 of (seed, counter0+b)."""
    torch, P = require_gpu()
    shape = gi.FlowShape(3, 8, 4, 16, 16)
    flow = P.Flow(shape, gi.init_weights(shape))
    a = flow.sample(37, seed=9, counter0=100, phi4=(-6.0, 5.0))
    b = flow.sample(1, seed=9, counter0=100 + 29, phi4=(-6.0, 5.0))
    assert torch.equal(a.phi[29], b.phi[0]) and torch.equal(a.logw[29], b.logw[0])


def test_empty_batch_and_errors():
    torch, P = require_gpu()
    shape = gi.WORKLOADS["c1"]["shape"]
    flow = P.Flow(shape, gi.init_weights(shape))
    out = flow.sample(0, phi4=(-4.0, 8.0))
    assert out.phi.numel() == 0
    with pytest.raises(P._abi.GFError):
        P.Flow(gi.FlowShape(2, 7, 2, 8, 8), gi.init_weights(gi.FlowShape(2, 7, 2, 8, 8)))
    with pytest.raises(P._abi.GFError):          # even kernel size
        P.Flow(gi.FlowShape(2, 8, 2, ksize=4), np.zeros(1000))
    # widths outside {8, 16, 32} are valid: they run on the general-network kernel
    w12 = gi.init_weights(gi.FlowShape(2, 8, 2, 12, 12))
    f12 = P.Flow(gi.FlowShape(2, 8, 2, 12, 12), w12)
    assert f12.sample(0, phi4=(-4.0, 8.0)).phi.numel() == 0


@pytest.mark.parametrize("key", ["c1", "c3"])
def test_bench_size_sampled_parity(orc, key):
    """Full batch at the benchmark's launch configuration, checked on sampled configurations."""
    torch, P = require_gpu()
    W = gi.WORKLOADS[key]
    shape, phi4, B = W["shape"], W["phi4"], W["batch"]
    w = gi.init_weights(shape)
    flow = P.Flow(shape, w)
    seed, c0 = 2024, 0
    out = flow.sample(B, seed=seed, counter0=c0, phi4=phi4)
    torch.cuda.synchronize()
    picks = sorted({0, 1, B // 2, B - 1})
    for b in picks:
        ref = orc.flow_sample(shape, w, phi4.m2, phi4.lam, 1, seed=seed, counter0=c0 + b)
        assert_sites_close(out.phi[b:b + 1].cpu().numpy(), ref["phi"], what=f"phi[{b}]")
        assert_logw_close(out.logw[b:b + 1].cpu().numpy(), ref["logw"], what=f"logw[{b}]")
    # properties over the whole batch
    assert torch.isfinite(out.phi).all() and torch.isfinite(out.logw).all()
    lq = flow.logq(out.phi)
    assert_logw_close(lq.cpu().numpy(), out.logq.cpu().numpy(), what="logq(F(phi)) vs logq")
    S = P.phi4_action(shape.nd, shape.L, phi4, out.phi)
    assert_logw_close(S.cpu().numpy(), out.S.cpu().numpy(), rtol=1e-12, what="fused vs standalone S")


@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[7]], ids=[_ids(c) for c in (CASES[0], CASES[2], CASES[7])])
def test_unfused_path_matches_oracle(orc, case):
    """The plain one-kernel-per-convolution path computes the same function."""
    torch, P = require_gpu()
    shape, m2, lam, B = case
    w = gi.init_weights(shape, seed=0)
    flow = P.Flow(shape, w)
    out = flow.sample_unfused(B, seed=1234, counter0=77, phi4=(m2, lam), return_z=True)
    ref = orc.flow_sample(shape, w, m2, lam, B, seed=1234, counter0=77)
    assert_sites_close(out.z.cpu().numpy(), ref["z"], rtol=1e-6, what="z")
    assert_sites_close(out.phi.cpu().numpy(), ref["phi"])
    for k in ("logq", "S", "logw"):
        assert_logw_close(getattr(out, k).cpu().numpy(), ref[k], what=k)
    fused = flow.sample(B, seed=1234, counter0=77, phi4=(m2, lam))
    assert_logw_close(out.logw.cpu().numpy(), fused.logw.cpu().numpy(), what="unfused vs fused")

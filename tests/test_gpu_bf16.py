"""GPU parity of the tensor-core variant (3D L=16, hidden 32).

The kernel rounds h1 (after LeakyReLU) and conv2's weights to bf16, and
conv1's input (the masked field), conv1's weights, h2 (after LeakyReLU) and
conv3's weights to fp16; it accumulates every convolution in FP32 on the
tensor cores; all sums over the lattice are FP64 accurate.  It is compared
with the oracle in the matching emulation mode (same rounding points, FP64
elsewhere), and its error against the pure FP64 oracle is reported (max and
p99 per result).

Tolerances: per number of coupling layers, from the committed CPU experiment
tests/golden/bf16_tolerance.py (oracle only).  The kernel and the oracle reach
each rounding with values that differ at the FP32 level, so values near a
rounding boundary round differently and the later layers carry the flip on.
The experiment measures exactly that drift between the oracle's FP64-summing
emulation and its FP32-accumulating model (GFO_F32_ACC) on 64 configurations
and takes twice the maximum (2 layers: about 5.1e-4 per site, 1.3e-5 per
log q / S / log w; 16 layers: 2.9e-3 per site, 3.0e-4 per result).  The
64-configuration test below also checks that the kernel's error distribution
(p99 and mean per site) stays within twice the model's.
"""
import numpy as np
import pytest

import gf_inputs as gi
from gpu_util import (BF16_MODE, assert_logw_close, assert_sites_close, bf16_drift_model,
                      bf16_tolerances, require_gpu)

pytestmark = pytest.mark.gpu


def _report(name, gpu, ref):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    if gpu.ndim == 2:
        scale = np.maximum(np.abs(ref), np.sqrt((ref**2).mean(1, keepdims=True)))
    else:
        scale = np.maximum(np.abs(ref), 1.0)
    e = np.abs(gpu - ref) / scale
    print(f"{name}: max {e.max():.3e} p99 {np.percentile(e, 99):.3e}")
    return e


def _site_err(gpu, ref):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.abs(gpu - ref) / np.maximum(np.abs(ref), np.sqrt((ref**2).mean(1, keepdims=True)))


@pytest.mark.parametrize("n_layers,B", [(2, 3), (16, 3)])
def test_bf16_sample_matches_emulated_oracle(orc, n_layers, B):
    torch, P = require_gpu()
    shape = gi.FlowShape(3, 16, n_layers, 32, 32)
    m2, lam = -6.0, 5.0
    w = gi.init_weights(shape, seed=0)
    flow = P.Flow(shape, w, precision="bf16")
    out = flow.sample(B, seed=21, counter0=5, phi4=(m2, lam), return_z=True)
    torch.cuda.synchronize()
    assert P.device_status() == 0
    ref = orc.flow_sample(shape, w, m2, lam, B, seed=21, counter0=5, bf16_mask=BF16_MODE)
    RTOL, LW_RTOL = bf16_tolerances(n_layers)
    assert_sites_close(out.z.cpu().numpy(), ref["z"], rtol=1e-6, what="z")
    _report("phi vs bf16-emulated", out.phi.cpu().numpy(), ref["phi"])
    for k in ("logq", "S", "logw"):
        _report(f"{k} vs bf16-emulated", getattr(out, k).cpu().numpy(), ref[k])
    assert_sites_close(out.phi.cpu().numpy(), ref["phi"], rtol=RTOL)
    for k in ("logq", "S", "logw"):
        assert_logw_close(getattr(out, k).cpu().numpy(), ref[k], rtol=LW_RTOL, what=k)
    # error of the BF16 path against the pure FP64 oracle, stated per result
    f64 = orc.flow_sample(shape, w, m2, lam, B, seed=21, counter0=5)
    _report("phi vs FP64", out.phi.cpu().numpy(), f64["phi"])
    for k in ("logq", "S", "logw"):
        _report(f"{k} vs FP64", getattr(out, k).cpu().numpy(), f64[k])


def test_bf16_given_z_and_inverse(orc):
    torch, P = require_gpu()
    shape = gi.FlowShape(3, 16, 4, 32, 32, use_final_tanh=False)
    w = gi.init_weights(shape, seed=4)
    flow = P.Flow(shape, w, precision="bf16")
    z = orc.prior(shape.V, 2, seed=8, counter0=0, f32=True)
    zt = torch.tensor(z, dtype=torch.float32, device="cuda")
    out = flow.sample(2, phi4=(-6.0, 5.0), z=zt)
    RTOL, LW_RTOL = bf16_tolerances(shape.n_layers)
    ref = orc.flow_sample(shape, w, -6.0, 5.0, 2, z=z, bf16_mask=BF16_MODE)
    assert_sites_close(out.phi.cpu().numpy(), ref["phi"], rtol=RTOL)
    zb, lq = flow.logq(out.phi, return_z=True)
    zr, lqr = orc.flow_logq(shape, w, out.phi.cpu().numpy().astype(np.float64), bf16_mask=BF16_MODE)
    assert_sites_close(zb.cpu().numpy(), zr, rtol=RTOL, what="z(inverse)")
    assert_logw_close(lq.cpu().numpy(), lqr, rtol=LW_RTOL, what="logq(inverse)")
    assert P.device_status() == 0


def test_bf16_full_batch_sampled(orc):
    """Batch 4096 at the benchmark's launch configuration, sampled configurations."""
    torch, P = require_gpu()
    W = gi.WORKLOADS["c3"]
    shape, phi4, B = W["shape"], W["phi4"], W["batch"]
    w = gi.init_weights(shape)
    flow = P.Flow(shape, w, precision="bf16")
    out = flow.sample(B, seed=2024, counter0=0, phi4=phi4)
    torch.cuda.synchronize()
    RTOL, LW_RTOL = bf16_tolerances(shape.n_layers)
    for b in (0, 1, 2047, B - 1):
        ref = orc.flow_sample(shape, w, phi4.m2, phi4.lam, 1, seed=2024, counter0=b, bf16_mask=BF16_MODE)
        assert_sites_close(out.phi[b:b + 1].cpu().numpy(), ref["phi"], rtol=RTOL, what=f"phi[{b}]")
        assert_logw_close(out.logw[b:b + 1].cpu().numpy(), ref["logw"], rtol=LW_RTOL, what=f"logw[{b}]")
    assert torch.isfinite(out.phi).all()
    S = P.phi4_action(3, 16, phi4, out.phi)
    assert_logw_close(S.cpu().numpy(), out.S.cpu().numpy(), rtol=1e-12, what="fused vs standalone S")
    assert P.device_status() == 0


def test_bf16_rejects_other_shapes():
    """Hidden widths that are not multiples of 8 and lattices whose
    activations do not fit one block (2D L=64, 3D L=12 with width 32) have no
    tensor-core kernel."""
    torch, P = require_gpu()
    for shape in (gi.FlowShape(3, 8, 2, 12, 12), gi.FlowShape(2, 64, 2, 32, 32), gi.FlowShape(3, 12, 2, 32, 32)):
        assert not P.tensor_core_supported(shape)
        with pytest.raises(P._abi.GFError):
            P.Flow(shape, gi.init_weights(shape), precision="bf16")


def test_bf16_64_configurations_error_report(orc):
    """64 configurations of the 3D workload's flow (16 layers): max / p99 /
    mean error per result against the BF16-emulated and the pure FP64 oracle;
    the kernel's per-site error distribution (p99, mean) within twice the
    drift that the oracle's FP32-accumulating model shows."""
    torch, P = require_gpu()
    W = gi.WORKLOADS["c3"]
    shape, phi4 = W["shape"], W["phi4"]
    B = 64
    w = gi.init_weights(shape)
    flow = P.Flow(shape, w, precision="bf16")
    out = flow.sample(B, seed=909, counter0=0, phi4=phi4)
    torch.cuda.synchronize()
    assert P.device_status() == 0
    RTOL, LW_RTOL = bf16_tolerances(shape.n_layers)
    ref = orc.flow_sample(shape, w, phi4.m2, phi4.lam, B, seed=909, counter0=0, bf16_mask=BF16_MODE)
    f64 = orc.flow_sample(shape, w, phi4.m2, phi4.lam, B, seed=909, counter0=0)
    phi = out.phi.cpu().numpy()
    for name, r in (("bf16-emulated", ref), ("FP64", f64)):
        _report(f"phi vs {name} (64 cfg)", phi, r["phi"])
        for k in ("logq", "S", "logw"):
            _report(f"{k} vs {name} (64 cfg)", getattr(out, k).cpu().numpy(), r[k])
    assert_sites_close(phi, ref["phi"], rtol=RTOL)
    for k in ("logq", "S", "logw"):
        assert_logw_close(getattr(out, k).cpu().numpy(), ref[k], rtol=LW_RTOL, what=k)
    e = _site_err(phi, ref["phi"])
    model = bf16_drift_model(shape.n_layers)["phi"]
    assert np.percentile(e, 99) <= 2 * model["p99"], (np.percentile(e, 99), model)
    assert e.mean() <= 2 * model["mean"], (e.mean(), model)


def test_bf16_wait_that_runs_out_reports_timeout_and_recovers(orc):
    """Failure path of the BF16 kernel's bounded waits, without a GPU fault:
    with the stall hook on, each block's first conv2 issuer waits for a barrier
    completion that never comes (65,536 polls, long after every MMA issued so
    far has finished); that wait gives up, the other roles leave their loops,
    the block drains its queued tensor-core work and weight copies, frees its
    tensor memory and returns.  The host sees GF_ETIMEOUT, and the next launch
    (hook off) is correct."""
    torch, P = require_gpu()
    lib = P._abi.load()
    shape = gi.FlowShape(3, 16, 2, 32, 32)
    w = gi.init_weights(shape, seed=0)
    flow = P.Flow(shape, w, precision="bf16")
    assert P.device_status() == 0
    assert lib.gf_set_bf16_stall_test(-1) == P._abi.GF_EINVAL
    try:
        assert lib.gf_set_bf16_stall_test(1 << 16) == P._abi.GF_OK
        flow.sample(304, seed=3, counter0=0, phi4=(-6.0, 5.0))
        torch.cuda.synchronize()
        st = P.device_status()
    finally:
        lib.gf_set_bf16_stall_test(0)
    assert st == P._abi.GF_ETIMEOUT
    out = flow.sample(4, seed=11, counter0=0, phi4=(-6.0, 5.0))
    torch.cuda.synchronize()
    assert P.device_status() == 0
    RTOL, LW_RTOL = bf16_tolerances(shape.n_layers)
    ref = orc.flow_sample(shape, w, -6.0, 5.0, 4, seed=11, counter0=0, bf16_mask=BF16_MODE)
    assert_sites_close(out.phi.cpu().numpy(), ref["phi"], rtol=RTOL)
    assert_logw_close(out.logw.cpu().numpy(), ref["logw"], rtol=LW_RTOL)


def test_stream_status_slots_attribute_errors_to_their_stream():
    """gf_set_stream_status_slot: a timeout in a launch on stream 1 lands in
    stream 1's slot only; stream 2's slot and the process-wide word stay 0."""
    torch, P = require_gpu()
    lib = P._abi.load()
    shape = gi.FlowShape(3, 16, 2, 32, 32)
    flow = P.Flow(shape, gi.init_weights(shape), precision="bf16")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    slots = torch.zeros(2, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    assert P.device_status() == 0
    P.set_stream_status_slot(s1, slots[0:1])
    P.set_stream_status_slot(s2, slots[1:2])
    try:
        lib.gf_set_bf16_stall_test(1 << 16)
        with torch.cuda.stream(s1):
            flow.sample(304, seed=1, counter0=0, phi4=(-6.0, 5.0))
        lib.gf_set_bf16_stall_test(0)
        with torch.cuda.stream(s2):
            flow.sample(304, seed=2, counter0=0, phi4=(-6.0, 5.0))
        torch.cuda.synchronize()
        assert P.device_status(s1) == P._abi.GF_ETIMEOUT
        assert P.device_status(s1) == 0              # read and cleared
        assert P.device_status(s2) == 0
        assert P.device_status() == 0
    finally:
        lib.gf_set_bf16_stall_test(0)
        P.set_stream_status_slot(s1, None)
        P.set_stream_status_slot(s2, None)


def test_fp16_overflow_reports_edevice_and_recovers(orc):
    """A field value beyond the FP16 range (65504) makes conv1's operand
    infinite, so s and t are not finite: the kernel records GF_EDEVICE (once
    per configuration, from a NaN-propagating check of every s and t), and the
    next launch on finite input is clean and correct."""
    torch, P = require_gpu()
    shape = gi.FlowShape(3, 16, 2, 32, 32)
    w = gi.init_weights(shape, seed=0)
    flow = P.Flow(shape, w, precision="bf16")
    assert P.device_status() == 0
    z = torch.tensor(gi.random_field(3, 16, 4, seed=5), dtype=torch.float32, device="cuda")
    z[2, 1234] = 1.0e6
    flow.sample(4, z=z, phi4=(-6.0, 5.0))
    torch.cuda.synchronize()
    assert P.device_status() == P._abi.GF_EDEVICE
    out = flow.sample(4, seed=11, counter0=0, phi4=(-6.0, 5.0))
    torch.cuda.synchronize()
    assert P.device_status() == 0
    RTOL, LW_RTOL = bf16_tolerances(shape.n_layers)
    ref = orc.flow_sample(shape, w, -6.0, 5.0, 4, seed=11, counter0=0, bf16_mask=BF16_MODE)
    assert_sites_close(out.phi.cpu().numpy(), ref["phi"], rtol=RTOL)
    assert_logw_close(out.logw.cpu().numpy(), ref["logw"], rtol=LW_RTOL)

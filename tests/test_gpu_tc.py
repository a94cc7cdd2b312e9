"""GPU parity of the tensor-core kernel for the lattice shapes other than 3D
L=16 with hidden width 32 (gf_flow_tc.cu): 2D and 3D lattices, hidden widths
8 (two taps per K-step), 16, 24 (padded to 32) and 32.

The kernel rounds h1 (after LeakyReLU) and conv2's weights to bf16 and h2
(after LeakyReLU) and the head's weights to FP16, accumulates conv2 and the
head in FP32 on the tensor cores, and runs conv1 in FP32; the sums over the
lattice are FP64 accurate.
It is compared with the oracle in the matching emulation mode (same rounding
points, FP64 elsewhere) at tolerances derived by the CPU experiment
tests/golden/bf16_tolerance.py --tc (oracle only: twice the largest drift
between the oracle's FP64-summing emulation and its FP32-accumulating model
over seven shapes of the serving mix, per number of coupling layers); its error
against the pure FP64 oracle is reported.
"""
import numpy as np
import pytest

import gf_inputs as gi
from gpu_util import TC_MODE, assert_logw_close, assert_sites_close, compare_mh, require_gpu, tc_tolerances

pytestmark = pytest.mark.gpu


def _err(gpu, ref):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    if gpu.ndim == 2:
        scale = np.maximum(np.abs(ref), np.sqrt((ref ** 2).mean(1, keepdims=True)))
    else:
        scale = np.maximum(np.abs(ref), 1.0)
    return np.abs(gpu - ref) / scale


# (nd, L, hidden, coupling layers, batch): one tile (2D L=8), width 8 (two taps
# per K-step) and the padded width 24, every lattice of the serving mix the
# kernel takes, 2 to 24 layers
CASES = [(2, 8, 16, 2, 3), (2, 16, 24, 8, 4), (2, 32, 32, 2, 3), (2, 32, 32, 24, 2), (2, 64, 16, 2, 2),
         (3, 8, 32, 8, 3), (3, 8, 24, 2, 3), (3, 12, 16, 2, 2), (3, 4, 32, 3, 3), (3, 16, 16, 2, 2),
         (2, 8, 8, 4, 3), (2, 32, 8, 8, 2), (3, 16, 8, 2, 2), (3, 16, 8, 23, 1)]


@pytest.mark.parametrize("nd,L,c,n_layers,B", CASES)
def test_tc_sample_matches_emulated_oracle(orc, nd, L, c, n_layers, B):
    torch, P = require_gpu()
    shape = gi.FlowShape(nd, L, n_layers, c, c)
    assert P.tensor_core_supported(shape)
    m2, lam = -4.0, 6.0
    w = gi.init_weights(shape, seed=5)
    flow = P.Flow(shape, w, precision="bf16")
    out = flow.sample(B, seed=31, counter0=2, phi4=(m2, lam), return_z=True)
    torch.cuda.synchronize()
    assert P.device_status() == 0
    ref = orc.flow_sample(shape, w, m2, lam, B, seed=31, counter0=2, bf16_mask=TC_MODE)
    RTOL, LW_RTOL = tc_tolerances(n_layers)
    assert_sites_close(out.z.cpu().numpy(), ref["z"], rtol=1e-6, what="z")
    phi = out.phi.cpu().numpy()
    f64 = orc.flow_sample(shape, w, m2, lam, B, seed=31, counter0=2)
    print(f"{nd}D L={L} C={c} {n_layers} layers: phi vs emulated {_err(phi, ref['phi']).max():.2e} "
          f"(bound {RTOL:.2e}), vs FP64 {_err(phi, f64['phi']).max():.2e}; " +
          ", ".join(f"{k} {_err(getattr(out, k).cpu().numpy(), ref[k]).max():.2e} / "
                    f"{_err(getattr(out, k).cpu().numpy(), f64[k]).max():.2e}" for k in ("logq", "S", "logw")))
    assert_sites_close(phi, ref["phi"], rtol=RTOL)
    for k in ("logq", "S", "logw"):
        assert_logw_close(getattr(out, k).cpu().numpy(), ref[k], rtol=LW_RTOL, what=k)


@pytest.mark.parametrize("nd,L,c", [(2, 32, 24), (3, 8, 16), (2, 16, 8), (3, 8, 8)])
def test_tc_given_z_and_inverse(orc, nd, L, c):
    """Sampling from a given z without the action, then the inverse pass
    (gf_flow_logq) back to z and log q, against the emulating oracle."""
    torch, P = require_gpu()
    shape = gi.FlowShape(nd, L, 4, c, c, use_final_tanh=False)
    w = gi.init_weights(shape, seed=9)
    flow = P.Flow(shape, w, precision="bf16")
    z = orc.prior(shape.V, 3, seed=4, counter0=0, f32=True)
    zt = torch.tensor(z, dtype=torch.float32, device="cuda")
    out = flow.sample(3, z=zt)
    RTOL, LW_RTOL = tc_tolerances(shape.n_layers)
    ref = orc.flow_sample(shape, w, 0.0, 0.0, 3, z=z, bf16_mask=TC_MODE)
    assert_sites_close(out.phi.cpu().numpy(), ref["phi"], rtol=RTOL)
    assert_logw_close(out.logq.cpu().numpy(), ref["logq"], rtol=LW_RTOL, what="logq")
    zb, lq = flow.logq(out.phi, return_z=True)
    zr, lqr = orc.flow_logq(shape, w, out.phi.cpu().numpy().astype(np.float64), bf16_mask=TC_MODE)
    assert_sites_close(zb.cpu().numpy(), zr, rtol=RTOL, what="z(inverse)")
    assert_logw_close(lq.cpu().numpy(), lqr, rtol=LW_RTOL, what="logq(inverse)")
    torch.cuda.synchronize()
    assert P.device_status() == 0


@pytest.mark.parametrize("nd,L,c", [(2, 16, 16), (2, 16, 8), (3, 8, 16), (3, 8, 8)])
def test_tc_persistent_batch_and_placement(orc, nd, L, c):
    """A batch several times the resident grid (each block runs two
    configurations at a time and loops over many, so the TMEM rings and the
    weight staging wrap around many times): sampled configurations against
    the oracle, every configuration bit-identical to the same prior counter
    sampled in a batch of its own (one configuration per block), and the
    inverse pass over the whole batch; 2D and 3D, hidden width 16 and 8 (two
    taps per K-step)."""
    torch, P = require_gpu()
    shape = gi.FlowShape(nd, L, 3, c, c)
    m2, lam = -4.0, 6.0
    w = gi.init_weights(shape, seed=2)
    flow = P.Flow(shape, w, precision="bf16")
    B = 5000
    out = flow.sample(B, seed=77, counter0=0, phi4=(m2, lam))
    torch.cuda.synchronize()
    assert P.device_status() == 0
    assert torch.isfinite(out.phi).all() and torch.isfinite(out.logw).all()
    RTOL, LW_RTOL = tc_tolerances(shape.n_layers)
    for b in (0, 1, 151, 1217, 3333, B - 1):
        ref = orc.flow_sample(shape, w, m2, lam, 1, seed=77, counter0=b, bf16_mask=TC_MODE)
        assert_sites_close(out.phi[b:b + 1].cpu().numpy(), ref["phi"], rtol=RTOL, what=f"phi[{b}]")
        assert_logw_close(out.logw[b:b + 1].cpu().numpy(), ref["logw"], rtol=LW_RTOL, what=f"logw[{b}]")
        one = flow.sample(1, seed=77, counter0=b, phi4=(m2, lam))
        assert torch.equal(one.phi[0], out.phi[b]) and torch.equal(one.logw[0], out.logw[b])
    S = P.phi4_action(nd, L, (m2, lam), out.phi)
    assert_logw_close(S.cpu().numpy(), out.S.cpu().numpy(), rtol=1e-12, what="fused vs standalone S")
    # the inverse pass over the same large batch (two configurations per block)
    zb, lq = flow.logq(out.phi, return_z=True)
    torch.cuda.synchronize()
    assert P.device_status() == 0
    for b in (0, 2501, B - 1):
        zr, lqr = orc.flow_logq(shape, w, out.phi[b:b + 1].cpu().numpy().astype(np.float64), bf16_mask=TC_MODE)
        assert_sites_close(zb[b:b + 1].cpu().numpy(), zr, rtol=RTOL, what=f"z(inverse)[{b}]")
        assert_logw_close(lq[b:b + 1].cpu().numpy(), lqr, rtol=LW_RTOL, what=f"logq(inverse)[{b}]")


def test_tc_mh_chain_on_flow_output(orc):
    """MH independence chain over the tensor-core kernel's log w (near-identity
    head for a non-trivial acceptance): decisions equal the oracle's on the
    same log w except at near ties."""
    torch, P = require_gpu()
    shape = gi.FlowShape(2, 16, 4, 32, 32)
    w = gi.init_weights(shape, seed=3)
    for l in range(shape.n_layers):
        blk = gi.split_layer(shape, w, l)
        blk["W3"][...] *= 0.05
    flow = P.Flow(shape, w, precision="bf16")
    out = flow.sample(2048, seed=12, counter0=0, phi4=(-4.0, 6.0))
    st = P.new_mh_state(seed=99)
    idx, acc = P.mh_chain(st, out.logw)
    torch.cuda.synchronize()
    lw = out.logw.cpu().numpy()
    n_acc = int(acc.cpu().numpy()[1:].sum())
    assert 0 < n_acc < 2047
    compare_mh(orc, 99, 0, lw, idx.cpu().numpy(), acc.cpu().numpy(), logw_tol=1e-15)


def test_tc_bench_launch_sampled(orc):
    """The bench's launch configuration of the 2D workload's flow (L=32, 24
    couplings, width 32, batch 8192, two configurations per block): sampled
    configurations against the emulating oracle at the 24-layer bound."""
    torch, P = require_gpu()
    shape = gi.FlowShape(2, 32, 24, 32, 32)
    m2, lam = -4.0, 6.0
    w = gi.init_weights(shape, seed=0)
    flow = P.Flow(shape, w, precision="bf16")
    B = 8192
    out = flow.sample(B, seed=5, counter0=0, phi4=(m2, lam))
    torch.cuda.synchronize()
    assert P.device_status() == 0
    assert torch.isfinite(out.phi).all() and torch.isfinite(out.logw).all()
    RTOL, LW_RTOL = tc_tolerances(shape.n_layers)
    for b in (0, 4095, B - 1):
        ref = orc.flow_sample(shape, w, m2, lam, 1, seed=5, counter0=b, bf16_mask=TC_MODE)
        assert_sites_close(out.phi[b:b + 1].cpu().numpy(), ref["phi"], rtol=RTOL, what=f"phi[{b}]")
        for k in ("logq", "S", "logw"):
            assert_logw_close(getattr(out, k)[b:b + 1].cpu().numpy(), ref[k], rtol=LW_RTOL, what=f"{k}[{b}]")


def test_tc_acceptance_equals_fp32_on_trained_2d_flow():
    """Equal MH acceptance of the tensor-core sampler and the fused FP32
    sampler on a 2D flow trained here (Sec. 1: flow proposals corrected by
    the MH test with the Jacobian; Sec. 3: the training loop): 2D L=8,
    m2=-4, lam=8 (the paper's example theory), 8 coupling layers of hidden
    width 16, 2,000 reverse-KL Adam steps at batch 64 on the GPU; then both
    samplers on the same 65,536 proposals (same prior counters, same MH
    uniforms).  The acceptances must agree within three binomial standard
    errors (combined as if independent; the chains share their proposals, so
    this is conservative), on a flow whose acceptance is far from zero."""
    import math
    torch, P = require_gpu()
    from paper_2208_08903_gb300 import train as T
    shape = gi.FlowShape(2, 8, 8, 16, 16)
    phi4 = (-4.0, 8.0)
    flow = P.Flow(shape, gi.init_weights(shape, seed=2021))
    st = T.train(flow, phi4, 20, 100, 64, lr=1e-3, seed=4242)
    assert all(math.isfinite(x) for x in st.losses)
    tc = P.Flow(shape, flow.get_weights().double().cpu().numpy(), precision="bf16")
    n = 65536
    ev32 = T.evaluate(flow, phi4, n, 4096, seed=909, sampler="fused", keep_logw=True)
    evtc = T.evaluate(tc, phi4, n, 4096, seed=909, sampler="fused", keep_logw=True)
    a32, atc = ev32["acceptance"], evtc["acceptance"]
    se = math.hypot(ev32["acceptance_binomial_err"], evtc["acceptance_binomial_err"])
    print(f"trained 2D L=8 flow: acceptance FP32 {a32:.5f} tensor-core {atc:.5f} (3 sigma {3 * se:.5f}); "
          f"ESS {ev32['ess']:.5f} {evtc['ess']:.5f}; decisions agree {T.decision_agreement(evtc, ev32):.4f}")
    assert a32 > 0.1
    assert abs(atc - a32) <= 3 * se
    assert P.device_status() == 0


@pytest.mark.parametrize("B", [3, 1000])
def test_tc_wait_that_runs_out_reports_timeout_and_recovers(orc, B):
    """Failure path of the kernel's bounded waits, without a GPU fault: with
    the stall hook on, the first conv2 issuer of each block (of each block half
    when a block runs two configurations) waits, before its first MMA, for a
    barrier completion that never comes (65,536 polls); that wait gives up,
    the other roles leave their loops, the block drains its weight copies and
    any queued tensor-core work, frees its tensor memory and returns.  The host
    sees GF_ETIMEOUT, and the next launch (hook off) is correct."""
    torch, P = require_gpu()
    lib = P._abi.load()
    shape = gi.FlowShape(2, 16, 2, 16, 16)
    w = gi.init_weights(shape, seed=1)
    flow = P.Flow(shape, w, precision="bf16")
    assert P.device_status() == 0
    try:
        assert lib.gf_set_bf16_stall_test(1 << 16) == P._abi.GF_OK
        flow.sample(B, seed=3, counter0=0, phi4=(-4.0, 6.0))
        torch.cuda.synchronize()
        st = P.device_status()
    finally:
        lib.gf_set_bf16_stall_test(0)
    assert st == P._abi.GF_ETIMEOUT
    out = flow.sample(4, seed=11, counter0=0, phi4=(-4.0, 6.0))
    torch.cuda.synchronize()
    assert P.device_status() == 0
    RTOL, LW_RTOL = tc_tolerances(shape.n_layers)
    ref = orc.flow_sample(shape, w, -4.0, 6.0, 4, seed=11, counter0=0, bf16_mask=TC_MODE)
    assert_sites_close(out.phi.cpu().numpy(), ref["phi"], rtol=RTOL)
    assert_logw_close(out.logw.cpu().numpy(), ref["logw"], rtol=LW_RTOL)


@pytest.mark.parametrize("nd,L,c", [(2, 32, 24), (3, 8, 16)])
def test_tc_odd_batch(orc, nd, L, c):
    """An odd batch larger than the SM count: the last block's second half has
    one configuration fewer than its first (it leaves its loop early and
    meets the other half only at the block's exit)."""
    torch, P = require_gpu()
    shape = gi.FlowShape(nd, L, 2, c, c)
    m2, lam = -4.0, 6.0
    w = gi.init_weights(shape, seed=8)
    flow = P.Flow(shape, w, precision="bf16")
    B = 333
    out = flow.sample(B, seed=2, counter0=0, phi4=(m2, lam))
    torch.cuda.synchronize()
    assert P.device_status() == 0
    RTOL, LW_RTOL = tc_tolerances(shape.n_layers)
    for b in (0, 165, B - 1):
        ref = orc.flow_sample(shape, w, m2, lam, 1, seed=2, counter0=b, bf16_mask=TC_MODE)
        assert_sites_close(out.phi[b:b + 1].cpu().numpy(), ref["phi"], rtol=RTOL, what=f"phi[{b}]")
        assert_logw_close(out.logw[b:b + 1].cpu().numpy(), ref["logw"], rtol=LW_RTOL, what=f"logw[{b}]")
        one = flow.sample(1, seed=2, counter0=b, phi4=(m2, lam))
        assert torch.equal(one.phi[0], out.phi[b]) and torch.equal(one.logw[0], out.logw[b])

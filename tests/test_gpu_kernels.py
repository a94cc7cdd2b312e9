"""GPU parity of the action, force, MH chain and HMC kernels against the oracle."""
import numpy as np
import pytest

import gf_inputs as gi
from gpu_util import assert_logw_close, assert_sites_close, compare_mh, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nd,L,B", [(2, 8, 64), (2, 5, 3), (3, 16, 37), (3, 3, 2), (2, 1, 4),
                                    (2, 128, 3)])
@pytest.mark.parametrize("fp64", [False, True])
def test_action_matches_oracle(orc, nd, L, B, fp64):
    torch, P = require_gpu()
    m2, lam = -6.0, 5.0
    phi = gi.random_field(nd, L, B, seed=L + B)
    if not fp64:
        phi = phi.astype(np.float32).astype(np.float64)     # the exact FP32 inputs
    t = torch.tensor(phi, dtype=torch.float64 if fp64 else torch.float32, device="cuda")
    S = P.phi4_action(nd, L, (m2, lam), t).cpu().numpy()
    ref = orc.action(nd, L, m2, lam, phi)
    assert_logw_close(S, ref, rtol=1e-12, what="S")


@pytest.mark.parametrize("nd,L,B", [(2, 16, 5), (2, 32, 153), (2, 64, 7), (3, 8, 301), (3, 16, 917)])
def test_action_streaming_lattices(orc, nd, L, B):
    """The streaming kernel's lattices, with more configurations than one
    wave of blocks holds (each block then refills its two buffers), on
    Gaussian fields, fields 1e-3 smaller (S dominated by the hopping term),
    a constant field, a zero field and fields with one large site, with and
    without the quartic term (the large site makes the biased hopping sum too
    coarse, and those configurations are summed again)."""
    torch, P = require_gpu()
    V = L ** nd
    phi = gi.random_field(nd, L, B, seed=3 * L + B).astype(np.float32).astype(np.float64)
    phi[1] *= 1e-3
    phi[2] = 0.75
    phi[3] = 0.0
    phi[4, V // 3] = 1000.0
    if B > 5:
        phi[5, 7] = -37.0
        phi[-1, V - 1] = 12.0
    phi = phi.astype(np.float32).astype(np.float64)         # the exact FP32 inputs
    t = torch.tensor(phi, dtype=torch.float32, device="cuda")
    for m2, lam in [(-6.0, 5.0), (1.0, 0.0), (-4.0, 1.0)]:
        S = P.phi4_action(nd, L, (m2, lam), t).cpu().numpy()
        ref = orc.action(nd, L, m2, lam, phi)
        assert_logw_close(S, ref, rtol=1e-12, what=f"S m2={m2} lam={lam}")


def test_action_streaming_unaligned_view_matches():
    """A batch view that starts 4 bytes past a 16-byte boundary cannot be bulk
    copied; it takes the per-configuration kernel and agrees with the
    streaming result of the same fields."""
    torch, P = require_gpu()
    base = torch.randn(41 * 4096 + 1, device="cuda")
    v = base[1:].view(41, 4096)
    S_view = P.phi4_action(3, 16, (-6.0, 5.0), v)
    S_cont = P.phi4_action(3, 16, (-6.0, 5.0), v.contiguous())
    assert torch.allclose(S_view, S_cont, rtol=1e-12, atol=1e-12)


def test_action_empty_and_unaligned():
    torch, P = require_gpu()
    empty = torch.empty(0, 64, device="cuda")
    assert P.phi4_action(2, 8, (1.0, 1.0), empty).numel() == 0
    # a view starting at an odd float offset takes the scalar staging path
    base = torch.randn(3 * 64 + 1, device="cuda")
    v = base[1:].view(3, 64)
    S1 = P.phi4_action(2, 8, (1.0, 1.0), v.contiguous())
    S2 = P.phi4_action(2, 8, (1.0, 1.0), v)
    assert torch.allclose(S1, S2, rtol=1e-13)


@pytest.mark.parametrize("nd,L", [(2, 8), (3, 4), (3, 16)])
def test_force_matches_oracle(orc, nd, L):
    torch, P = require_gpu()
    phi = gi.random_field(nd, L, 5, seed=1)
    F = P.phi4_force(nd, L, (-6.0, 5.0), torch.tensor(phi, device="cuda")).cpu().numpy()
    ref = orc.force(nd, L, -6.0, 5.0, phi)
    assert np.allclose(F, ref, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("kind", ["random", "flat", "mixed"])
def test_mh_chain_matches_oracle(orc, kind):
    torch, P = require_gpu()
    n = 5000
    rng = np.random.default_rng(0)
    if kind == "random":
        logw = rng.standard_normal(n) * 2.0 - 100.0       # moderate acceptance
    elif kind == "flat":
        logw = -7.0 + 1e-3 * rng.standard_normal(n)       # almost every proposal accepted
    else:
        logw = np.where(rng.random(n) < 0.5, -1e4, -3.0) + rng.standard_normal(n)
    seed, stream = 42, 3
    state = P.new_mh_state(seed, stream)
    lw = torch.tensor(logw, device="cuda")
    idx_parts, acc_parts = [], []
    for a, b in [(0, 1), (1, 33), (33, 1000), (1000, 1000), (1000, n)]:   # ragged calls, empty call
        i, c = P.mh_chain(state, lw[a:b].contiguous())
        idx_parts.append(i.cpu().numpy())
        acc_parts.append(c.cpu().numpy())
    idx = np.concatenate(idx_parts)
    acc = np.concatenate(acc_parts)
    st_ref = orc.new_mh_state(seed, stream)
    idx_ref, acc_ref = orc.mh_chain(st_ref, logw)
    div = compare_mh(orc, seed, stream, logw, idx, acc)
    assert div == 0
    assert (idx == idx_ref).all() and (acc == acc_ref).all()
    st = P.read_mh_state(state)
    assert st.step == n and st.n_acc == st_ref.n_acc and st.idx_cur == st_ref.idx_cur
    assert st.logw_cur == st_ref.logw_cur


def test_mh_chain_on_flow_output(orc):
    """The chain over the GPU's own log weights (paper example workload)."""
    torch, P = require_gpu()
    W = gi.WORKLOADS["c1"]
    shape, phi4 = W["shape"], W["phi4"]
    w = gi.scale_head(shape, gi.init_weights(shape), 0.05)   # near-identity flow: real acceptance
    flow = P.Flow(shape, w)
    state = P.new_mh_state(5, 0)
    lws, idxs, accs = [], [], []
    for i in range(16):                                     # 16 x 64 = 1024 chain steps
        out = flow.sample(64, seed=11, counter0=64 * i, phi4=phi4)
        ii, aa = P.mh_chain(state, out.logw)
        lws.append(out.logw.cpu().numpy()); idxs.append(ii.cpu().numpy()); accs.append(aa.cpu().numpy())
    logw = np.concatenate(lws)
    ref = orc.flow_sample(shape, w, phi4.m2, phi4.lam, 1024, seed=11, counter0=0)
    assert_logw_close(logw, ref["logw"])
    compare_mh(orc, 5, 0, logw, np.concatenate(idxs), np.concatenate(accs), logw_tol=1e-4)
    assert 0 < np.concatenate(accs)[1:].mean() < 1


@pytest.mark.parametrize("nd,L,nc", [(3, 4, 16), (2, 8, 9), (3, 16, 4)])
def test_hmc_matches_oracle(orc, nd, L, nc):
    torch, P = require_gpu()
    m2, lam = -6.0, 5.0
    phi0 = gi.random_field(nd, L, nc, seed=3, scale=0.3)
    t = torch.tensor(phi0, device="cuda")
    for traj in range(3):
        dH, acc = P.hmc_trajectory(nd, L, (m2, lam), t, 20, 0.05, seed=7, traj_index=traj)
        phi_ref, dH_ref, acc_ref = orc.hmc_trajectory(nd, L, m2, lam, phi0, 20, 0.05, 7, traj)
        dHg = dH.cpu().numpy()
        assert np.allclose(dHg, dH_ref, rtol=1e-8, atol=1e-9)
        a = acc.cpu().numpy()
        logu = np.array([np.log((2 * (int(orc.philox([7, 0], [c, traj, 0, 4])[0]) >> 12) + 1) * 2.0**-53)
                         for c in range(nc)])
        for c in range(nc):
            if a[c] != acc_ref[c]:
                assert abs(-dH_ref[c] - logu[c]) < 1e-8        # near tie only
                phi_ref[c] = t[c].cpu().numpy()
        assert np.allclose(t.cpu().numpy(), phi_ref, rtol=1e-10, atol=1e-10)
        phi0 = phi_ref
    assert P.device_status() == 0


def test_alu_peak_probe_is_plausible():
    """The FFMA/DFMA probe's rate sits below the lane-count bound at the
    device's maximum clock (128 FP32 FMA lanes per SM) and well above a tenth
    of it; FP64 runs slower than FP32."""
    require_gpu()
    import torch
    from paper_2208_08903_gb300 import api
    prop = torch.cuda.get_device_properties(0)
    f32 = api.alu_peak(fp64=False, iters=1 << 15)
    f64 = api.alu_peak(fp64=True, iters=1 << 12)
    f32x2 = api.alu_peak(packed=True, iters=1 << 15)
    bound = prop.multi_processor_count * 128 * 2 * 2.2e9      # above every Blackwell boost clock
    assert 0.1 * bound < f32 < bound
    assert 0 < f64 < f32
    assert 0.1 * bound < f32x2 < 2.2 * bound

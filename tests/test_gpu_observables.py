"""GPU parity of the chain observables against the FP64 oracle.

Per-configuration M and C(t), the autocorrelation function and the ESS are
sums in a different order on the two sides (the GPU sums each slice in FP32
pairs, about 2^-48 relative per addition, the rest in FP64): 1e-12 relative (to
the larger of the value and the configuration's scale).  The chain gather is exact.
The window W of tau_int is an integer decided in FP64 on both sides from those
sums; the AR(1) series used here have no near tie at the window, so W must be
equal.
"""
import numpy as np
import pytest

import gf_inputs as gi
from gpu_util import assert_logw_close, assert_sites_close, compare_mh, require_gpu

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.mark.parametrize("nd,L,B", [(2, 8, 5), (3, 4, 3), (2, 6, 7), (3, 16, 9), (2, 32, 130), (3, 5, 2)])
def test_observables_match_oracle(orc, nd, L, B):
    torch, P = require_gpu()
    V = L**nd
    phi = (orc.prior(V, B, seed=21, counter0=0, f32=True) + 0.3).astype(np.float32).astype(np.float64)
    M, Cc = P.observables(nd, L, torch.tensor(phi, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    rM, rC = orc.observables(nd, L, phi)
    assert_sites_close(M.cpu().numpy()[:, None], rM[:, None], rtol=RTOL, what="M")
    assert_sites_close(Cc.cpu().numpy(), rC, rtol=RTOL, what="C(t)")


@pytest.mark.parametrize("nd,L,B", [(2, 16, 3001), (2, 32, 1201), (2, 64, 917), (3, 8, 2500), (3, 16, 1000)])
def test_observables_streaming_lattices(orc, nd, L, B):
    """The bulk-copy streaming kernel's lattices with more configurations than
    one wave of blocks holds, so every block cycles through its buffer ring."""
    torch, P = require_gpu()
    V = L**nd
    phi = (orc.prior(V, B, seed=5 + L, counter0=0, f32=True) * 0.7 - 0.2).astype(np.float32).astype(np.float64)
    t = torch.tensor(phi, dtype=torch.float32, device="cuda")
    M, Cc = P.observables(nd, L, t)
    rM, rC = orc.observables(nd, L, phi)
    assert_sites_close(M.cpu().numpy()[:, None], rM[:, None], rtol=RTOL, what="M")
    assert_sites_close(Cc.cpu().numpy(), rC, rtol=RTOL, what="C(t)")
    # either output alone
    M1, none_c = P.observables(nd, L, t, two_point=False)
    none_m, C1 = P.observables(nd, L, t, magnetisation=False)
    assert none_c is None and none_m is None
    assert torch.equal(M1, M) and torch.equal(C1, Cc)


def test_observables_at_bench_size_sampled(orc):
    torch, P = require_gpu()
    nd, L, B = 3, 16, 4096
    V = L**nd
    gen = torch.Generator(device="cuda").manual_seed(3)
    phi = torch.randn(B, V, device="cuda", generator=gen) * 0.8 + 0.1
    M, Cc = P.observables(nd, L, phi)
    M_only, none = P.observables(nd, L, phi, two_point=False)
    torch.cuda.synchronize()
    assert none is None and torch.equal(M, M_only)
    rows = np.array([0, 1, 777, 2048, 4095])
    rM, rC = orc.observables(nd, L, phi[rows].double().cpu().numpy())
    assert_sites_close(M[rows].cpu().numpy()[:, None], rM[:, None], rtol=RTOL, what="M")
    assert_sites_close(Cc[rows].cpu().numpy(), rC, rtol=RTOL, what="C(t)")


def test_chain_gather_exact_and_out_of_range_flagged(orc):
    torch, P = require_gpu()
    vals = torch.arange(40, device="cuda", dtype=torch.float64).reshape(20, 2) * 0.5
    idx = torch.tensor([100, 100, 103, 119, 107], device="cuda", dtype=torch.int64)
    out = P.chain_gather(idx, vals, idx0=100)
    assert P.device_status() == 0
    ref = vals.cpu().numpy()[idx.cpu().numpy() - 100]
    assert np.array_equal(out.cpu().numpy(), ref)
    bad = torch.tensor([100, 120, 99], device="cuda", dtype=torch.int64)
    out = P.chain_gather(bad, vals[:, 0].contiguous(), idx0=100)
    st = P.device_status()
    o = out.cpu().numpy()
    assert o[0] == 0.0 and np.isnan(o[1]) and np.isnan(o[2])
    assert st == -1                                    # GF_EINVAL recorded, then cleared
    assert P.device_status() == 0


def ar1(n, rho, seed):
    e = np.random.default_rng(seed).normal(size=n)
    y = np.empty(n)
    y[0] = e[0]
    s = np.sqrt(1 - rho * rho)
    for k in range(1, n):
        y[k] = rho * y[k - 1] + s * e[k]
    return y


@pytest.mark.parametrize("n,t_max,rho", [(1000, 50, 0.5), (100_000, 1000, 0.9), (37, 36, 0.0), (5000, 0, 0.3)])
def test_autocorr_matches_oracle(orc, n, t_max, rho):
    torch, P = require_gpu()
    y = ar1(n, rho, seed=n) + 3.0
    g, summ = P.autocorr(torch.tensor(y, device="cuda"), t_max, c_window=5.0)
    torch.cuda.synchronize()
    rg = orc.autocorr(y, t_max)
    g = g.cpu().numpy()
    assert np.all(np.abs(g - rg) <= RTOL * np.maximum(np.abs(rg), rg[0]))
    tau, W, err = orc.tau_int(n, rg, c=5.0)
    s = summ.cpu().numpy()
    assert int(s[1]) == W
    assert abs(s[0] - tau) <= 1e-10 * max(tau, 1.0)
    assert abs(s[2] - err) <= 1e-10 * max(err, 1e-300)
    assert abs(s[3] - y.mean()) <= 1e-12 * max(abs(y.mean()), 1.0)


def test_autocorr_of_a_constant_series_is_exactly_zero(orc):
    torch, P = require_gpu()
    y = torch.full((999,), 0.1 + 0.2, device="cuda", dtype=torch.float64)
    g, summ = P.autocorr(y, 20)
    torch.cuda.synchronize()
    assert not g.cpu().numpy().any()
    assert summ.cpu().numpy().tolist() == [0.5, 0.0, 0.0, 0.1 + 0.2]


@pytest.mark.parametrize("n", [0, 1, 5, 1000, 100_000])
def test_ess_matches_oracle(orc, n):
    torch, P = require_gpu()
    lw = np.random.default_rng(n).normal(size=n) * 4 - 1000.0
    if n > 3:
        lw[2] = -np.inf
    e = P.ess(torch.tensor(lw, device="cuda")).item()
    r = orc.ess(lw)
    assert abs(e - r) <= RTOL * max(r, 1e-300) or (r == 0.0 and e == 0.0)


def test_chain_observables_end_to_end(orc):
    """Flow sample -> MH chain -> M per proposal -> chain series -> <|M|>, tau,
    all on the device.  The chain must be a valid MH chain of the sampled log w
    (oracle uniforms, near ties tolerated), and the series must be |M| of the
    oracle's configuration at every chain position."""
    torch, P = require_gpu()
    W = gi.WORKLOADS["c1"]
    shape, phi4 = W["shape"], W["phi4"]
    w = gi.init_weights(shape, seed=0)
    flow = P.Flow(shape, w)
    B, nb = 64, 4
    st = P.new_mh_state(77)
    Ms, idxs, accs, lws = [], [], [], []
    for i in range(nb):
        r = flow.sample(B, seed=5, counter0=i * B, phi4=phi4)
        idx, acc = P.mh_chain(st, r.logw)
        M, _ = P.observables(shape.nd, shape.L, r.phi, two_point=False)
        Ms.append(M)
        idxs.append(idx)
        accs.append(acc)
        lws.append(r.logw)
    M_all = torch.cat(Ms)
    idx_all = torch.cat(idxs)
    series = P.chain_gather(idx_all, M_all).abs().contiguous()
    g, summ = P.autocorr(series, 20)
    torch.cuda.synchronize()
    ref = orc.flow_sample(shape, w, phi4.m2, phi4.lam, B * nb, seed=5, counter0=0)
    logw = torch.cat(lws).cpu().numpy()
    assert_logw_close(logw, ref["logw"])
    idx_np = idx_all.cpu().numpy()
    compare_mh(orc, 77, 0, logw, idx_np, torch.cat(accs).cpu().numpy(), logw_tol=1e-4)
    rM, _ = orc.observables(shape.nd, shape.L, ref["phi"])
    rs = np.abs(rM[idx_np])
    assert np.allclose(series.cpu().numpy(), rs, rtol=1e-5, atol=1e-6)
    assert abs(summ[3].item() - rs.mean()) <= 1e-5 * max(rs.mean(), 1e-3)
    rg = orc.autocorr(rs, 20)
    assert np.allclose(g.cpu().numpy(), rg, rtol=1e-3, atol=1e-4 * max(rg[0], 1e-12))

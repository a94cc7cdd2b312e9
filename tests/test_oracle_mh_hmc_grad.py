"""Pins of the oracle's MH chain, HMC integrator and reverse-KL gradient (CPU only).

arXiv:2208.08903 Sec. 1 (MH test with the Jacobian, shifted reverse KL) and
Sec. 2.2 (HMC for the same theory).

- MH: a hand-built decision table (tests/golden/mh_table.txt), the all-accept
  special case, the uniforms against numpy's Philox, and stationarity on
  V=1 and V=4 lattices against quadrature;
- HMC: leapfrog reversibility, the O(eps^2) energy error, <exp(-dH)> = 1 and
  stationarity on V=1 against quadrature;
- gradient: central finite differences of the loss, and the closed form of
  the conv3-bias gradient of an identity flow; Adam against its first-step
  closed form.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

import gf_inputs as gi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_mh_hand_built_table(orc):
    rows = np.loadtxt(os.path.join(GOLDEN, "mh_table.txt"), comments="#")
    st = orc.new_mh_state(seed=0)
    idx, acc = orc.mh_scan(st, rows[:, 0], rows[:, 1])
    assert acc.tolist() == rows[:, 2].astype(int).tolist()
    assert idx.tolist() == rows[:, 3].astype(int).tolist()
    assert st.step == len(rows)
    assert st.n_acc == int(rows[1:, 2].sum())
    assert st.logw_cur == -12.0 and st.idx_cur == 7
    # resuming from the state continues the global indices
    idx2, acc2 = orc.mh_scan(st, np.array([-12.0, -100.0]), np.array([-0.1, -0.1]))
    assert acc2.tolist() == [1, 0] and idx2.tolist() == [8, 8]


def test_mh_constant_logw_accepts_all(orc):
    st = orc.new_mh_state(seed=5, stream_id=2)
    idx, acc = orc.mh_chain(st, np.full(1000, -3.25))
    assert acc.all() and (idx == np.arange(1000)).all() and st.n_acc == 999


def test_mh_uniforms_from_numpy_philox(orc):
    seed, stream = 99, 3
    logu = orc.mh_logu(seed, stream, 5, 16)
    for k in range(16):
        c = np.array([5 + k - 1, 0, 0, 2], dtype=np.uint64)
        w = np.random.Philox(counter=c, key=np.array([seed, stream], dtype=np.uint64)).random_raw(1)[0]
        u = (2 * (int(w) >> 12) + 1) * 2.0**-53
        assert logu[k] == math.log(u)
    big = np.exp(orc.mh_logu(1, 0, 0, 20000))
    assert stats.kstest(big, "uniform").pvalue > 1e-3


def _binned_err(x, nbins=50):
    m = len(x) // nbins
    means = x[: m * nbins].reshape(nbins, m).mean(1)
    return means.std(ddof=1) / math.sqrt(nbins)


def test_mh_stationarity_single_site(orc):
    """V=1: S = m2 phi^2 + lam phi^4; identity flow => q = N(0,1) proposals."""
    m2, lam = -1.0, 1.0
    n = 200000
    z = np.random.default_rng(1).standard_normal(n)
    logq = stats.norm.logpdf(z)
    S = orc.action(2, 1, m2, lam, z[:, None])
    st = orc.new_mh_state(seed=7)
    idx, acc = orc.mh_chain(st, -S - logq)
    chain = z[idx]
    wgt = lambda f: integrate.quad(lambda p: f(p) * math.exp(-(m2 * p * p + lam * p**4)),
                                   -np.inf, np.inf)[0]
    ref2 = wgt(lambda p: p * p) / wgt(lambda p: 1.0)
    ref4 = wgt(lambda p: p**4) / wgt(lambda p: 1.0)
    assert abs(chain.var() + chain.mean()**2 - ref2) < 4 * _binned_err(chain**2)
    assert abs((chain**4).mean() - ref4) < 4 * _binned_err(chain**4)


def test_mh_stationarity_four_sites(orc):
    """2D L=2 (V=4): chain moments vs a 4-D quadrature."""
    m2, lam, nd, L = -1.0, 0.5, 2, 2
    n = 300000
    z = np.random.default_rng(2).standard_normal((n, 4)) * 1.2
    logq = stats.norm.logpdf(z, scale=1.2).sum(1)
    S = orc.action(nd, L, m2, lam, z)
    st = orc.new_mh_state(seed=8)
    idx, _ = orc.mh_chain(st, -S - logq)
    chain = z[idx]
    # quadrature: S from numpy roll on a 4-D trapezoid grid (spectrally accurate
    # for this smooth, fast-decaying integrand)
    g = np.linspace(-3.6, 3.6, 49)
    X = np.stack(np.meshgrid(g, g, g, g, indexing="ij"), -1).reshape(-1, 4)
    f = X.reshape(-1, 2, 2)
    hop = (f * np.roll(f, -1, 1)).sum((1, 2)) + (f * np.roll(f, -1, 2)).sum((1, 2))
    Sq = ((4 + m2) * f**2 + lam * f**4).sum((1, 2)) - 2 * hop
    dens = np.exp(-(Sq - Sq.min()))
    ref2 = (dens * X[:, 0]**2).sum() / dens.sum()
    refc = (dens * X[:, 0] * X[:, 1]).sum() / dens.sum()
    assert abs((chain[:, 0]**2).mean() - ref2) < 4 * _binned_err(chain[:, 0]**2)
    assert abs((chain[:, 0] * chain[:, 1]).mean() - refc) < 4 * _binned_err(chain[:, 0] * chain[:, 1])


def test_leapfrog_reversible(orc):
    nd, L, m2, lam = 3, 4, -6.0, 5.0
    phi = gi.random_field(nd, L, 1, seed=1, scale=0.5)[0]
    pi = gi.random_field(nd, L, 1, seed=2)[0]
    p1, q1, dH = orc.leapfrog(nd, L, m2, lam, phi, pi, 20, 0.01)
    p2, q2, dH2 = orc.leapfrog(nd, L, m2, lam, p1, -q1, 20, 0.01)
    assert np.allclose(p2, phi, atol=1e-12) and np.allclose(q2, -pi, atol=1e-12)
    assert dH2 == pytest.approx(-dH, abs=1e-9)


def test_leapfrog_energy_error_is_second_order(orc):
    nd, L, m2, lam = 2, 4, -4.0, 8.0
    phi = gi.random_field(nd, L, 1, seed=3, scale=0.3)[0]
    pi = gi.random_field(nd, L, 1, seed=4)[0]
    tau = 0.2
    errs = []
    for n in (10, 20, 40):
        errs.append(abs(orc.leapfrog(nd, L, m2, lam, phi, pi, n, tau / n)[2]))
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.1)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.1)


def test_hmc_momenta_are_normal_and_fresh(orc):
    p = orc.hmc_momenta(4096 * 8, seed=1, chain=0, traj=0)
    assert stats.kstest(p, "norm").pvalue > 1e-3
    assert not np.allclose(orc.hmc_momenta(8, 1, 0, 0), orc.hmc_momenta(8, 1, 0, 1))
    assert not np.allclose(orc.hmc_momenta(8, 1, 0, 0), orc.hmc_momenta(8, 1, 1, 0))


def test_hmc_stationarity_and_exp_dH(orc):
    """V=1 chains: <phi^2> vs quadrature, <exp(-dH)> = 1 at equilibrium."""
    m2, lam = -1.0, 1.0
    nc = 4000
    phi = np.zeros((nc, 1))
    dHs, samples = [], []
    for traj in range(120):
        phi, dH, acc = orc.hmc_trajectory(2, 1, m2, lam, phi, 10, 0.15, seed=3, traj_index=traj)
        if traj >= 20:
            dHs.append(dH.copy())
            samples.append(phi[:, 0].copy())
    x = np.array(samples)               # [traj][chain]
    wgt = lambda f: integrate.quad(lambda p: f(p) * math.exp(-(m2 * p * p + lam * p**4)),
                                   -np.inf, np.inf)[0]
    ref2 = wgt(lambda p: p * p) / wgt(lambda p: 1.0)
    per_chain = (x**2).mean(0)
    assert abs(per_chain.mean() - ref2) < 4 * per_chain.std(ddof=1) / math.sqrt(nc)
    e = np.exp(-np.array(dHs)).mean(0)
    assert abs(e.mean() - 1.0) < 4 * e.std(ddof=1) / math.sqrt(nc)


def test_hmc_rejection_restores_field(orc):
    nd, L = 2, 4
    phi0 = gi.random_field(nd, L, 8, seed=1, scale=2.0)
    phi, dH, acc = orc.hmc_trajectory(nd, L, -4.0, 8.0, phi0, 10, 0.2, seed=1, traj_index=0)
    for c in range(8):
        if not acc[c]:
            assert np.array_equal(phi[c], phi0[c])
        else:
            assert not np.array_equal(phi[c], phi0[c])
    assert (acc == 0).any()    # a large step size on a rough start rejects some


GSHAPES = [gi.FlowShape(2, 4, 4, 4, 4), gi.FlowShape(3, 2, 3, 3, 2),
           gi.FlowShape(2, 3, 2, 3, 3, use_final_tanh=False),
           gi.FlowShape(2, 4, 2, hidden_sizes=(3, 2, 3), ksize=5),
           gi.FlowShape(2, 3, 3, hidden_sizes=(), ksize=3),
           gi.FlowShape(3, 3, 2, hidden_sizes=(2,), ksize=5)]


@pytest.mark.parametrize("shape", GSHAPES)
def test_loss_gradient_finite_differences(orc, shape):
    m2, lam = -4.0, 8.0
    w = gi.init_weights(shape, seed=4)
    z = gi.random_field(shape.nd, shape.L, 3, seed=5)
    loss, g = orc.flow_loss_grad(shape, w, m2, lam, z)
    o = orc.flow_sample(shape, w, m2, lam, 3, z=z)
    assert loss == pytest.approx((o["logq"] + o["S"]).mean(), rel=1e-13)
    rng = np.random.default_rng(0)
    idx = rng.choice(w.size, 20, replace=False)
    idx[:6] = [0, shape.layer_params() - 1, shape.layer_params() - 2,
               shape.conv_channels()[0][1] * shape.taps, w.size - 1, w.size // 2]
    eps = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += eps
        wm[i] -= eps
        fp = orc.flow_sample(shape, wp, m2, lam, 3, z=z)
        fm = orc.flow_sample(shape, wm, m2, lam, 3, z=z)
        fd = ((fp["logq"] + fp["S"]).mean() - (fm["logq"] + fm["S"]).mean()) / (2 * eps)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-6 * max(1.0, abs(g).max())), i


def test_identity_flow_bias_gradient_closed_form(orc):
    """Zero conv3 => phi = z; dL/db3_t(l) = mean_b sum_{A_l} F, dL/db3_s(l) = mean_b sum_{A_l} F z - |A_l|."""
    shape = gi.FlowShape(2, 4, 3, 4, 4)
    m2, lam = -4.0, 8.0
    w = gi.zero_head(shape, gi.init_weights(shape))
    z = gi.random_field(2, 4, 5, seed=1)
    _, g = orc.flow_loss_grad(shape, w, m2, lam, z)
    F = orc.force(2, 4, m2, lam, z)
    yy, xx = np.meshgrid(np.arange(4), np.arange(4), indexing="ij")
    par = ((yy + xx) % 2).ravel()
    P = shape.layer_params()
    for l in range(shape.n_layers):
        A = par != (l % 2)
        gs = g[(l + 1) * P - 2]
        gt = g[(l + 1) * P - 1]
        assert gt == pytest.approx((F[:, A]).sum(1).mean(), rel=1e-12)
        assert gs == pytest.approx((F[:, A] * z[:, A]).sum(1).mean() - A.sum(), rel=1e-12)


def test_adam_first_step_closed_form(orc):
    rng = np.random.default_rng(0)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    m, v = np.zeros(50), np.zeros(50)
    th0 = th.copy()
    orc.adam(th, g, m, v, 1, 1e-3)
    assert np.allclose(th, th0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)

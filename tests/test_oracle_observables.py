"""Pins of the oracle's chain observables (condensate, zero-momentum two-point
function, autocorrelation, integrated autocorrelation time, ESS) against closed
forms, independent library routines (numpy FFT and correlate) and exact
statistics of processes with known autocorrelation."""
import numpy as np
import pytest

import gf_inputs as gi


def lattice_coords(nd, L):
    n = np.arange(L**nd)
    return [(n // L**a) % L for a in range(nd)]      # x, y(, z)


@pytest.mark.parametrize("nd,L", [(2, 6), (3, 4), (2, 8)])
def test_constant_field(orc, nd, L):
    V = L**nd
    c = -1.25
    M, C = orc.observables(nd, L, np.full((2, V), c))
    assert np.allclose(M, c, rtol=0, atol=1e-15)
    # Phi(tau) = (V/L) c  =>  C(t) = (1/V) L (V/L)^2 c^2 = (V/L) c^2
    assert np.allclose(C, (V / L) * c * c, rtol=1e-15)


@pytest.mark.parametrize("nd,L,k", [(2, 8, 1), (2, 8, 3), (3, 6, 1), (3, 6, 2)])
def test_plane_wave_along_time_axis(orc, nd, L, k):
    V, A = L**nd, 0.7
    tau = lattice_coords(nd, L)[-1]
    a = 2 * np.pi * k / L
    phi = A * np.cos(a * tau)
    M, C = orc.observables(nd, L, phi[None])
    assert abs(M[0]) < 1e-14
    t = np.arange(L)
    # Phi(tau) = (V/L) A cos(a tau): C(t) = (V/L) (A^2 / 2) cos(a t) for 2k != 0 mod L
    assert np.allclose(C[0], (V / L) * A * A / 2 * np.cos(a * t), rtol=0, atol=1e-12)


@pytest.mark.parametrize("nd,L", [(2, 8), (3, 6)])
def test_plane_wave_along_a_spatial_axis_has_no_zero_momentum_signal(orc, nd, L):
    x = lattice_coords(nd, L)[0]
    phi = np.cos(2 * np.pi * x / L) + 0.3 * np.sin(4 * np.pi * x / L)
    M, C = orc.observables(nd, L, phi[None])
    assert abs(M[0]) < 1e-14
    assert np.abs(C).max() < 1e-12


@pytest.mark.parametrize("nd,L", [(2, 8), (3, 4), (3, 6)])
def test_two_point_function_matches_fft(orc, nd, L):
    rng = np.random.default_rng(5)
    B, V = 4, L**nd
    phi = rng.normal(size=(B, V)) + 0.4
    M, C = orc.observables(nd, L, phi)
    # Wiener-Khinchin with numpy's FFT: the slice sums over every axis but the
    # outermost, then the circular autocorrelation of that length-L signal
    f = phi.reshape((B,) + (L,) * nd)                        # [B][outer]...[x]
    Phi = f.reshape(B, L, -1).sum(axis=2)
    ref = np.fft.ifft(np.abs(np.fft.fft(Phi, axis=1)) ** 2, axis=1).real / V
    assert np.allclose(C, ref, rtol=1e-12, atol=1e-12)
    assert np.allclose(M, phi.mean(axis=1), rtol=1e-13)
    # sum rule: sum_t C(t) = (sum_tau Phi)^2 / V = V M^2
    assert np.allclose(C.sum(axis=1), V * M * M, rtol=1e-12)


def test_autocorr_matches_numpy_correlate(orc):
    rng = np.random.default_rng(1)
    y = np.cumsum(rng.normal(size=3000)) * 0.01 + rng.normal(size=3000)
    t_max = 200
    g = orc.autocorr(y, t_max)
    d = y - y.mean()
    full = np.correlate(d, d, mode="full")[d.size - 1:d.size + t_max]
    ref = full / (d.size - np.arange(t_max + 1))
    assert np.allclose(g, ref, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.8])
def test_tau_int_of_ar1_process(orc, rho):
    # y_k = rho y_{k-1} + sqrt(1 - rho^2) e_k: rho(t) = rho^t exactly, so
    # tau_int = 1/2 + rho/(1 - rho) = (1 + rho) / (2 (1 - rho))
    rng = np.random.default_rng(7)
    n = 400_000
    e = rng.normal(size=n)
    y = np.empty(n)
    y[0] = e[0]
    s = np.sqrt(1 - rho * rho)
    for k in range(1, n):
        y[k] = rho * y[k - 1] + s * e[k]
    g = orc.autocorr(y, 200)
    tau, W, err = orc.tau_int(n, g, c=6.0)
    exact = (1 + rho) / (2 * (1 - rho))
    # Madras-Sokal's error estimate plus the window's truncation bias rho^W term
    assert abs(tau - exact) <= 4 * err + exact * rho ** W + 1e-3, (tau, exact, W, err)


def test_window_rule_against_exponential_closed_form(orc):
    # Gamma(t) = r^t exactly: tau(W) = 1/2 + r (1 - r^W) / (1 - r).  The window
    # must be the smallest W >= 1 with W >= c tau(W).
    r, c, t_max = 0.9, 5.0, 400
    g = r ** np.arange(t_max + 1)
    tau, W, err = orc.tau_int(10_000, g, c=c)

    def tau_of(w):
        return 0.5 + r * (1 - r**w) / (1 - r)

    assert W >= c * tau_of(W)
    assert all(w < c * tau_of(w) for w in range(1, W))
    assert abs(tau - tau_of(W)) < 1e-12
    assert abs(err - tau * np.sqrt((4 * W + 2) / 10_000)) < 1e-12
    # constant series
    assert orc.tau_int(100, np.zeros(11)) == (0.5, 0, 0.0)


def test_ess_closed_forms(orc):
    assert orc.ess(np.zeros(17)) == pytest.approx(1.0, abs=1e-15)
    lw = np.full(10, -np.inf)
    lw[3] = 2.5
    assert orc.ess(lw) == pytest.approx(0.1, abs=1e-15)
    a = 0.3
    assert orc.ess(np.log([1.0, a])) == pytest.approx((1 + a) ** 2 / (2 * (1 + a * a)), rel=1e-14)
    rng = np.random.default_rng(3)
    lw = rng.normal(size=1000) * 3
    assert orc.ess(lw + 123.0) == pytest.approx(orc.ess(lw), rel=1e-12)
    assert orc.ess(np.array([])) == 0.0
    assert orc.ess(np.full(4, -np.inf)) == 0.0


def test_ess_of_gaussian_importance_weights(orc):
    # proposal N(0,1), target N(0, s^2): E_q[w^2] = 1 / (s sqrt(2 - s^2)), so
    # the ESS fraction tends to s sqrt(2 - s^2) as the sample grows
    s, n = 0.8, 2_000_000
    x = np.random.default_rng(9).normal(size=n)
    lw = -0.5 * x * x / (s * s) - np.log(s) + 0.5 * x * x
    assert orc.ess(lw) == pytest.approx(s * np.sqrt(2 - s * s), rel=5e-3)


def test_chain_average_of_a_repeated_state(orc):
    # an MH chain that rejects everything after step 0 sits on proposal 0: the
    # chain series is constant, its autocorrelation vanishes, tau = 1/2
    st = orc.new_mh_state(5)
    logw = np.concatenate([[0.0], np.full(63, -1e9)])
    idx, acc = orc.mh_chain(st, logw)
    assert (idx == 0).all() and acc.sum() == 1
    M, _ = orc.observables(2, 4, np.random.default_rng(0).normal(size=(64, 16)))
    series = M[idx]
    assert orc.tau_int(64, orc.autocorr(series, 10)) == (0.5, 0, 0.0)

"""Pins of the oracle's random numbers and of the phi^4 action (CPU only).

Philox4x64-10 is checked against numpy's independent implementation; the
prior against numpy's Philox words plus a Kolmogorov-Smirnov test; the
action (arXiv:2208.08903 Sec. 1) against closed forms (constant field, plane
wave), the momentum-space Parseval form computed with numpy's FFT, and a
differently arranged real-space form; the force against finite differences.
"""
import math

import numpy as np
import pytest
from scipy import stats

import gf_inputs as gi


def _np_words(key, ctr):
    c = np.array(ctr, dtype=np.uint64)
    c[0] -= np.uint64(1)            # numpy increments the counter before each block
    return np.random.Philox(counter=c, key=np.array(key, dtype=np.uint64)).random_raw(4)


@pytest.mark.parametrize("seed", [0, 1, 12345, 2**63 + 5])
def test_philox_matches_numpy(orc, seed):
    rng = np.random.default_rng(seed % 1000)
    for _ in range(20):
        key = [seed, int(rng.integers(0, 2**63))]
        ctr = [int(rng.integers(1, 2**63)) for _ in range(4)]
        assert (orc.philox(key, ctr) == _np_words(key, ctr)).all()


def test_prior_words_and_box_muller(orc):
    V, B, seed, c0 = 10, 3, 77, 5
    z = orc.prior(V, B, seed, c0, f32=False)
    for b in range(B):
        for j in range((V + 3) // 4):
            w = _np_words([seed, 0], [c0 + b, j, 0, 1])
            u = [(2 * (int(x) >> 41) + 1) * 2.0**-24 for x in w]
            vals = []
            for p in range(2):
                r = math.sqrt(-2 * math.log(u[2 * p]))
                vals += [r * math.cos(2 * math.pi * u[2 * p + 1]),
                         r * math.sin(2 * math.pi * u[2 * p + 1])]
            for q in range(4):
                if 4 * j + q < V:
                    assert z[b, 4 * j + q] == pytest.approx(vals[q], rel=1e-14, abs=1e-14)
    z32 = orc.prior(V, B, seed, c0, f32=True)
    assert (z32 == z.astype(np.float32).astype(np.float64)).all()


def test_prior_is_standard_normal(orc):
    z = orc.prior(4096, 16, seed=3, counter0=0).ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
    # different configurations / counters give different draws
    a = orc.prior(64, 2, 3, 0)
    assert not np.allclose(a[0], a[1])


def test_log_prior_matches_scipy(orc):
    z = gi.random_field(2, 4, 5, seed=1)
    ref = stats.norm.logpdf(z).sum(axis=1)
    assert np.allclose(orc.log_prior(z), ref, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("nd,L", [(2, 1), (2, 2), (2, 3), (2, 5), (3, 1), (3, 2), (3, 4)])
def test_action_constant_field(orc, nd, L):
    V = L**nd
    for c in (0.0, 0.7, -1.3):
        for m2, lam in ((-4.0, 8.0), (0.5, 0.0), (-6.0, 5.0)):
            S = orc.action(nd, L, m2, lam, np.full((1, V), c))[0]
            assert S == pytest.approx(V * (m2 * c * c + lam * c**4), rel=1e-14, abs=1e-12)
            F = orc.force(nd, L, m2, lam, np.full((1, V), c))[0]
            assert np.allclose(F, 2 * m2 * c + 4 * lam * c**3, rtol=1e-13, atol=1e-12)


def _coords(nd, L):
    g = np.meshgrid(*([np.arange(L)] * nd), indexing="ij")   # (z,)y,x order
    return g


@pytest.mark.parametrize("nd,L,k", [(2, 8, (1, 2)), (2, 6, (0, 1)), (3, 4, (1, 0, 1)),
                                    (3, 6, (1, 2, 0))])
def test_action_plane_wave(orc, nd, L, k):
    A, m2 = 0.9, 0.3
    g = _coords(nd, L)
    arg = sum(2 * math.pi * kk * gg / L for kk, gg in zip(k, g))
    phi = (A * np.cos(arg)).reshape(1, -1)
    V = L**nd
    ref = A * A * (V / 2) * (sum(4 * math.sin(math.pi * kk / L)**2 for kk in k) + m2)
    assert orc.action(nd, L, m2, 0.0, phi)[0] == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("nd,L", [(2, 8), (2, 5), (3, 4), (3, 3)])
def test_action_parseval_fft(orc, nd, L):
    """lambda = 0: S = (1/V) sum_p |phi~(p)|^2 (p^2_hat + m2), phi~ from numpy's FFT."""
    m2 = 0.7
    phi = gi.random_field(nd, L, 3, seed=11)
    S = orc.action(nd, L, m2, 0.0, phi)
    V = L**nd
    for b in range(3):
        ft = np.fft.fftn(phi[b].reshape([L] * nd))
        ks = np.meshgrid(*([2 * np.pi * np.arange(L) / L] * nd), indexing="ij")
        phat2 = sum(4 * np.sin(kk / 2)**2 for kk in ks)
        ref = (np.abs(ft)**2 * (phat2 + m2)).sum() / V
        assert S[b] == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("nd,L", [(2, 8), (2, 3), (3, 4), (3, 2)])
def test_action_forward_only_form(orc, nd, L):
    """S = sum_n [(2d + m2) phi^2 + lam phi^4 - 2 sum_mu phi(n) phi(n+mu)] (numpy roll)."""
    m2, lam = -4.0, 8.0
    phi = gi.random_field(nd, L, 4, seed=5)
    S = orc.action(nd, L, m2, lam, phi)
    for b in range(4):
        f = phi[b].reshape([L] * nd)
        hop = sum((f * np.roll(f, -1, axis=a)).sum() for a in range(nd))
        ref = ((2 * nd + m2) * f**2 + lam * f**4).sum() - 2 * hop
        assert S[b] == pytest.approx(ref, rel=1e-13)


def test_action_gaussian_whitening(orc):
    """lambda = 0, m2 > 0: S = phi^T A phi with A = -Lap + m2 (built by numpy from the
    Laplacian matrix); phi = (2A)^(-1/2) xi gives S = |xi|^2 / 2 exactly and <S> = V/2."""
    nd, L, m2 = 2, 4, 0.5
    V = L**nd
    A = np.zeros((V, V))
    for n in range(V):
        y, x = divmod(n, L)
        A[n, n] += m2 + 2 * nd
        for (dy, dx) in ((0, 1), (0, -1), (1, 0), (-1, 0)):
            A[n, ((y + dy) % L) * L + (x + dx) % L] -= 1.0
    ev, U = np.linalg.eigh(2 * A)
    R = U @ np.diag(ev**-0.5) @ U.T
    xi = np.random.default_rng(0).standard_normal((2000, V))
    phi = xi @ R.T
    S = orc.action(nd, L, m2, 0.0, phi)
    assert np.allclose(S, 0.5 * (xi**2).sum(1), rtol=1e-11)
    assert abs(S.mean() - V / 2) < 5 * math.sqrt(V / 2) / math.sqrt(2000)


@pytest.mark.parametrize("nd,L", [(2, 1), (2, 2), (2, 5), (3, 3)])
def test_force_finite_difference(orc, nd, L):
    m2, lam = -6.0, 5.0
    phi = gi.random_field(nd, L, 1, seed=9)
    F = orc.force(nd, L, m2, lam, phi)[0]
    eps = 1e-5
    for n in range(L**nd):
        p, m = phi.copy(), phi.copy()
        p[0, n] += eps
        m[0, n] -= eps
        fd = (orc.action(nd, L, m2, lam, p)[0] - orc.action(nd, L, m2, lam, m)[0]) / (2 * eps)
        assert fd == pytest.approx(F[n], rel=1e-7, abs=1e-7)


def test_single_site_lattice_has_no_kinetic_term(orc):
    for nd in (2, 3):
        phi = np.array([[1.7]])
        assert orc.action(nd, 1, -1.0, 1.0, phi)[0] == pytest.approx(-1.7**2 + 1.7**4, rel=1e-15)

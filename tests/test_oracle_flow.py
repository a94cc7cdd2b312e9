"""Pins of the oracle's coupling layers, flow composition and log-det (CPU only).

arXiv:2208.08903 Sec. 1: the even/odd affine coupling layer, the composition
of N_tri layers, the Jacobian of F^{-1} and the model density P^(ML).

- one coupling network against scipy.ndimage.correlate (periodic, independent
  library routine) with torch's bf16 rounding for the BF16-emulation flags;
- the whole flow against a brute-force numpy composition of those layers;
- log-det against log|det| of the brute-force Jacobian (central differences,
  numpy slogdet) on L=2,3 lattices;
- invertibility, identity flow, translation equivariance.
"""
import math

import numpy as np
import pytest
from scipy import ndimage, stats

import gf_inputs as gi


def lrelu(v, a):
    return np.where(v > 0, v, a * v)


def scipy_net(shape, w, layer, y, round_fn=None, flags=0, round16=None):
    """s, t of one coupling network (any hidden_sizes, odd kernel size) with
    scipy's periodic correlate.  flags: the oracle's bf16 rounding points (1 h1,
    2 middle weights, 4 later hidden activations, 8 head weights, 16 first
    weights, 64 the network input) and FP16 ones (512 the network input, 1024
    first weights, 2048 later hidden activations, 4096 head weights), applied
    with round_fn (bf16) and round16 (FP16)."""
    d = gi.split_layer(shape, w, layer)
    nd, L, k = shape.nd, shape.L, shape.ksize
    grid = [L] * nd
    ker = lambda W: W.reshape(W.shape[0], W.shape[1], *([k] * nd))
    rw = (lambda a: a) if round_fn is None else round_fn

    def conv(inp, W, b):
        K = ker(W)
        out = np.zeros((K.shape[0],) + tuple(grid))
        for o in range(K.shape[0]):
            acc = np.full(grid, b[o])
            for i in range(K.shape[1]):
                acc = acc + ndimage.correlate(inp[i], K[o, i], mode="wrap")
            out[o] = acc
        return out

    r16 = (lambda a: a) if round16 is None else round16
    if flags & 512:
        y = r16(y)
    elif flags & 64:
        y = rw(y)
    h = y.reshape([1] + grid)
    nh = len(shape.hidden)
    for j in range(nh + 1):
        W = d[f"W{j + 1}"]
        wflag = 8 if j == nh else (16 if j == 0 else 2)
        f16flag = 4096 if j == nh else (1024 if j == 0 else 0)
        if flags & f16flag:
            W = r16(W)
        elif flags & wflag:
            W = rw(W)
        h = conv(h, W, d[f"b{j + 1}"])
        if j < nh:
            h = lrelu(h, shape.leaky_slope)
            if j > 0 and flags & 2048:
                h = r16(h)
            elif flags & (1 if j == 0 else 4):
                h = rw(h)
    s = np.tanh(h[0]) if shape.use_final_tanh else h[0]
    return s.ravel(), h[1].ravel()


def parity(nd, L):
    g = np.meshgrid(*([np.arange(L)] * nd), indexing="ij")
    return (sum(g) % 2).ravel()


def numpy_flow(shape, w, z):
    """Brute-force composition: layer l keeps parity l%2 fixed, updates the rest."""
    par = parity(shape.nd, shape.L)
    x = z.copy()
    logdet = 0.0
    for l in range(shape.n_layers):
        fz = par == (l % 2)
        s, t = scipy_net(shape, w, l, np.where(fz, x, 0.0))
        x = np.where(fz, x, x * np.exp(s) + t)
        logdet += s[~fz].sum()
    return x, logdet


SHAPES = [gi.FlowShape(2, 4, 3, 4, 5), gi.FlowShape(2, 3, 2, 3, 2),
          gi.FlowShape(3, 3, 2, 2, 3), gi.FlowShape(2, 5, 4, 8, 8, use_final_tanh=False),
          gi.FlowShape(3, 2, 3, 4, 4)]
# the model section's other network shapes: hidden_sizes lists of other
# lengths (three hidden layers, one, none) and kernel_size 5 / 7
VARIANTS = [gi.FlowShape(2, 6, 3, hidden_sizes=(4, 3, 5), ksize=5),
            gi.FlowShape(2, 5, 2, hidden_sizes=(3, 3, 3), ksize=3),
            gi.FlowShape(3, 5, 2, hidden_sizes=(3,), ksize=5),
            gi.FlowShape(2, 4, 2, hidden_sizes=(), ksize=3),
            gi.FlowShape(2, 8, 2, hidden_sizes=(2, 4), ksize=7, use_final_tanh=False),
            gi.FlowShape(3, 4, 2, hidden_sizes=(2, 2, 2, 2), ksize=3)]


@pytest.mark.parametrize("shape", SHAPES + VARIANTS)
def test_coupling_net_vs_scipy(orc, shape):
    w = gi.init_weights(shape, seed=3)
    y = gi.random_field(shape.nd, shape.L, 1, seed=4)[0]
    for layer in range(shape.n_layers):
        s, t = orc.coupling_net(shape, w, layer, y)
        rs, rt = scipy_net(shape, w, layer, y)
        assert np.allclose(s, rs, rtol=1e-12, atol=1e-13)
        assert np.allclose(t, rt, rtol=1e-12, atol=1e-13)


def test_variant_weight_layout_and_default_net_unchanged():
    """hidden_sizes (c1, c2) with kernel 3 is the original layout; a variant's
    parameter count is the sum over its convolutions."""
    a, b = gi.FlowShape(3, 4, 2, 8, 16), gi.FlowShape(3, 4, 2, hidden_sizes=(8, 16), ksize=3)
    assert np.array_equal(gi.init_weights(a, seed=1), gi.init_weights(b, seed=1))
    v = gi.FlowShape(2, 4, 3, hidden_sizes=(4, 3, 5), ksize=5)
    T = 25
    assert v.layer_params() == (4 * T + 4) + (3 * 4 * T + 3) + (5 * 3 * T + 5) + (2 * 5 * T + 2)
    assert [n for n, _ in v.layer_blocks()] == ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"]


def test_fp16_rounding_points_vs_numpy(orc):
    """The FP16 rounding points (conv1 input and weights, h2, head weights)
    against numpy's float16 conversion (round to nearest even, subnormals,
    overflow to infinity), alone and in the tensor-core mode's combination."""
    def r16(a):
        with np.errstate(over="ignore"):
            return np.asarray(a, np.float64).astype(np.float16).astype(np.float64)

    def rbf(a):
        torch = pytest.importorskip("torch")
        a = np.asarray(a)
        return torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy().reshape(a.shape)

    shape = gi.FlowShape(3, 3, 1, 8, 8)
    w = gi.init_weights(shape, seed=8)
    y = gi.random_field(3, 3, 1, seed=2)[0]
    for flags in (512, 1024, 2048, 4096, orc.BF16_MODE & ~32):
        s, t = orc.coupling_net(shape, w, 0, y, bf16_mask=flags)
        rs, rt = scipy_net(shape, w, 0, y, round_fn=rbf, flags=flags, round16=r16)
        assert np.allclose(s, rs, rtol=1e-9, atol=1e-10), flags
        assert np.allclose(t, rt, rtol=1e-9, atol=1e-10), flags
    # overflow, subnormals and ties through the input rounding point (a net whose
    # conv1 is the identity on the centre tap)
    shape1 = gi.FlowShape(2, 3, 1, hidden_sizes=(), ksize=1, use_final_tanh=False)
    w1 = np.array([1.0, 0.0, 0.0, 0.0])               # W1 [2][1][1] = (1, 0), b1 = (0, 0)
    for v in (70000.0, 65519.0, 65520.0, 3e-7, 1e-8, 1.0 + 2.0**-11, 1.0 + 3 * 2.0**-11, 2049.0):
        yv = np.zeros(9)
        yv[0] = v
        s, _ = orc.coupling_net(shape1, w1, 0, yv, bf16_mask=512)
        assert s[0] == r16(v) or (np.isinf(s[0]) and np.isinf(r16(v))), v


def test_bf16_rounding_points_vs_torch(orc):
    torch = pytest.importorskip("torch")

    def rnd(a):
        a = np.asarray(a)
        t = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64)
        return t.numpy().reshape(a.shape)

    shape = gi.FlowShape(3, 3, 1, 8, 8)
    w = gi.init_weights(shape, seed=8)
    y = gi.random_field(3, 3, 1, seed=2)[0]
    for flags in (1, 2, 4, 8, 16, 64, 1 | 2 | 4 | 8, 1 | 2 | 4 | 8 | 16 | 64):
        s, t = orc.coupling_net(shape, w, 0, y, bf16_mask=flags)
        rs, rt = scipy_net(shape, w, 0, y, round_fn=rnd, flags=flags)
        assert np.allclose(s, rs, rtol=1e-9, atol=1e-10), flags
        assert np.allclose(t, rt, rtol=1e-9, atol=1e-10), flags
    s0, _ = orc.coupling_net(shape, w, 0, y, bf16_mask=0)
    s1, _ = orc.coupling_net(shape, w, 0, y, bf16_mask=1 | 2 | 4)
    assert not np.allclose(s0, s1, rtol=1e-6)


@pytest.mark.parametrize("shape", SHAPES + VARIANTS)
def test_flow_vs_bruteforce_composition(orc, shape):
    w = gi.init_weights(shape, seed=5)
    B = 3
    z = gi.random_field(shape.nd, shape.L, B, seed=6)
    m2, lam = -4.0, 8.0
    o = orc.flow_sample(shape, w, m2, lam, B, z=z)
    for b in range(B):
        phi, logdet = numpy_flow(shape, w, z[b])
        assert np.allclose(o["phi"][b], phi, rtol=1e-12, atol=1e-12)
        logr = stats.norm.logpdf(z[b]).sum()
        assert o["logq"][b] == pytest.approx(logr - logdet, rel=1e-12, abs=1e-11)
    S = orc.action(shape.nd, shape.L, m2, lam, o["phi"])
    assert np.allclose(o["S"], S, rtol=1e-14)
    assert np.allclose(o["logw"], -S - o["logq"], rtol=1e-14)


@pytest.mark.parametrize("shape", [gi.FlowShape(2, 2, 4, 4, 4), gi.FlowShape(2, 3, 3, 4, 4),
                                   gi.FlowShape(3, 2, 4, 3, 3), gi.FlowShape(3, 3, 2, 2, 2),
                                   gi.FlowShape(2, 3, 3, hidden_sizes=(3, 2, 3), ksize=5),
                                   gi.FlowShape(3, 2, 2, hidden_sizes=(2,), ksize=5)])
def test_logdet_vs_bruteforce_jacobian(orc, shape):
    """log|det dphi/dz| by central differences + LU must equal log r(z) - log q."""
    w = gi.init_weights(shape, seed=2)
    z = gi.random_field(shape.nd, shape.L, 1, seed=3)[0]
    V = shape.V
    eps = 1e-5
    J = np.zeros((V, V))
    for j in range(V):
        zp, zm = z.copy(), z.copy()
        zp[j] += eps
        zm[j] -= eps
        fp = orc.flow_sample(shape, w, 0.0, 0.0, 1, z=zp[None])["phi"][0]
        fm = orc.flow_sample(shape, w, 0.0, 0.0, 1, z=zm[None])["phi"][0]
        J[:, j] = (fp - fm) / (2 * eps)
    sign, logabsdet = np.linalg.slogdet(J)
    o = orc.flow_sample(shape, w, 0.0, 0.0, 1, z=z[None])
    logdet = orc.log_prior(z[None])[0] - o["logq"][0]
    assert sign > 0       # exp(s) > 0 on every updated site: orientation preserving
    assert logabsdet == pytest.approx(logdet, rel=1e-7, abs=1e-7)


@pytest.mark.parametrize("shape", SHAPES + VARIANTS + [gi.WORKLOADS["c1"]["shape"]])
def test_invertibility(orc, shape):
    w = gi.init_weights(shape, seed=0)
    o = orc.flow_sample(shape, w, -4.0, 8.0, 5, seed=9, counter0=3)
    z, logq = orc.flow_logq(shape, w, o["phi"])
    assert np.allclose(z, o["z"], rtol=0, atol=1e-12)
    assert np.allclose(logq, o["logq"], rtol=1e-12, atol=1e-10)


def test_identity_flow(orc):
    shape = gi.WORKLOADS["c1"]["shape"]
    w = gi.zero_head(shape, gi.init_weights(shape))
    o = orc.flow_sample(shape, w, -4.0, 8.0, 4, seed=1)
    assert np.array_equal(o["phi"], o["z"])
    assert np.allclose(o["logq"], stats.norm.logpdf(o["z"]).sum(1), rtol=1e-13)


@pytest.mark.parametrize("nd,L,shift", [(2, 4, (0, 2)), (2, 6, (1, 1)), (3, 4, (2, 0, 0)),
                                        (3, 4, (1, 0, 1))])
def test_translation_equivariance(orc, nd, L, shift):
    """Parity-preserving periodic shifts commute with the flow."""
    shape = gi.FlowShape(nd, L, 4, 4, 4)
    w = gi.init_weights(shape, seed=1)
    z = gi.random_field(nd, L, 1, seed=2)
    o = orc.flow_sample(shape, w, -4.0, 8.0, 1, z=z)
    zs = np.roll(z.reshape([L] * nd), shift, axis=tuple(range(nd))).reshape(1, -1)
    os_ = orc.flow_sample(shape, w, -4.0, 8.0, 1, z=zs)
    ref = np.roll(o["phi"].reshape([L] * nd), shift, axis=tuple(range(nd))).ravel()
    assert np.allclose(os_["phi"][0], ref, rtol=1e-12, atol=1e-12)
    assert os_["logq"][0] == pytest.approx(o["logq"][0], rel=1e-12)


def test_prior_counter_selects_configuration(orc):
    """Configuration b of a call with counter0=c equals configuration 0 of counter0=c+b."""
    shape = gi.WORKLOADS["c1"]["shape"]
    w = gi.init_weights(shape)
    a = orc.flow_sample(shape, w, -4.0, 8.0, 6, seed=4, counter0=10)
    b = orc.flow_sample(shape, w, -4.0, 8.0, 1, seed=4, counter0=14)
    assert np.array_equal(a["phi"][4], b["phi"][0])

"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the method: it only fixes the workload
shapes and draws random numbers (flow weights, test fields).  Both the FP64
oracle (``oracle/``) and the CUDA library receive the arrays produced here as
plain data, so neither depends on the other.

Canonical weight layout (FP64, flat, one block per coupling layer ``l`` in the
order the layers are applied to the prior sample): for each convolution
j = 0 .. n_hidden of the layer's s/t network

    W{j+1}[c_out][c_in][T]  b{j+1}[c_out]

with c_in = 1 for the first and c_out = 2 for the last (the head), the hidden
widths in between, ``T = k**nd`` taps ordered (kz, ky, kx) in 3D and (ky, kx)
in 2D, offset ``t - (k-1)/2`` along each axis.  Output channel 0 of the head is
s, channel 1 is t.  With the paper's example network (hidden_sizes [c1, c2],
kernel_size 3) this is W1[c1][1][T] b1 W2[c2][c1][T] b2 W3[2][c2][T] b3.  The
s/t network shape (n_layers, hidden_sizes, kernel_size, one input channel, two
output channels) is the paper's model section (Sec. 3, the example parameter
file).

Initialisation: Kaiming-uniform with negative slope sqrt(5) (the default of
PyTorch convolution layers, which the paper's software mirrors), i.e.
W, b ~ U(-1/sqrt(fan_in), +1/sqrt(fan_in)), fan_in = C_in * T, drawn in FP64
with numpy's Philox bit generator keyed by ``seed`` in the layout order above.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class FlowShape:
    nd: int                 # lattice dimension, 2 or 3
    L: int                  # sites per axis (periodic)
    n_layers: int           # affine coupling layers
    c1: int = 8             # hidden widths of the paper's two-hidden-layer net
    c2: int = 8
    use_final_tanh: bool = True
    leaky_slope: float = 0.01
    hidden_sizes: tuple | None = None   # any hidden_sizes list (overrides c1, c2)
    ksize: int = 3          # kernel_size (odd), circular padding (ksize-1)/2

    @property
    def hidden(self) -> tuple:
        return tuple(self.hidden_sizes) if self.hidden_sizes is not None else (self.c1, self.c2)

    @property
    def is_default_net(self) -> bool:
        """The paper's example network form: two hidden convolutions, 3 taps per axis."""
        return len(self.hidden) == 2 and self.ksize == 3

    @property
    def V(self) -> int:
        return self.L ** self.nd

    @property
    def taps(self) -> int:
        return self.ksize ** self.nd

    def conv_channels(self):
        """(c_in, c_out) of convolution j = 0 .. n_hidden."""
        chans = (1,) + self.hidden + (2,)
        return [(chans[j], chans[j + 1]) for j in range(len(chans) - 1)]

    def layer_params(self) -> int:
        T = self.taps
        return sum(ci * co * T + co for ci, co in self.conv_channels())

    def n_params(self) -> int:
        return self.n_layers * self.layer_params()

    @property
    def head(self) -> int:
        """1-based index of the head convolution (W{head}, b{head})."""
        return len(self.hidden) + 1

    def layer_blocks(self):
        """(name, shape) of the tensors of one layer, in layout order."""
        T = self.taps
        out = []
        for j, (ci, co) in enumerate(self.conv_channels()):
            out += [(f"W{j + 1}", (co, ci, T)), (f"b{j + 1}", (co,))]
        return out


@dataclasses.dataclass(frozen=True)
class Phi4:
    m2: float
    lam: float


def init_weights(shape: FlowShape, seed: int = 0) -> np.ndarray:
    """Flat FP64 weights in the canonical layout, Kaiming-uniform from ``seed``."""
    gen = np.random.Generator(np.random.Philox(key=seed))
    T = shape.taps
    fan_in = {}
    for j, (ci, _) in enumerate(shape.conv_channels()):
        fan_in[f"W{j + 1}"] = fan_in[f"b{j + 1}"] = ci * T
    out = []
    for _ in range(shape.n_layers):
        for name, shp in shape.layer_blocks():
            a = 1.0 / math.sqrt(fan_in[name])
            out.append(gen.uniform(-a, a, size=int(np.prod(shp))))
    w = np.concatenate(out).astype(np.float64)
    assert w.size == shape.n_params()
    return w


def split_layer(shape: FlowShape, w: np.ndarray, layer: int) -> dict:
    """Views of the six tensors of one layer of a canonical weight array."""
    P = shape.layer_params()
    blk = w[layer * P:(layer + 1) * P]
    out, off = {}, 0
    for name, shp in shape.layer_blocks():
        n = int(np.prod(shp))
        out[name] = blk[off:off + n].reshape(shp)
        off += n
    return out


def zero_head(shape: FlowShape, w: np.ndarray) -> np.ndarray:
    """Copy of ``w`` with every head weight and bias set to zero (s = t = 0)."""
    w = w.copy()
    for l in range(shape.n_layers):
        d = split_layer(shape, w, l)
        d[f"W{shape.head}"][...] = 0.0
        d[f"b{shape.head}"][...] = 0.0
    return w


def scale_head(shape: FlowShape, w: np.ndarray, factor: float) -> np.ndarray:
    """Copy of ``w`` with the head's weights and bias multiplied by ``factor``."""
    w = w.copy()
    for l in range(shape.n_layers):
        d = split_layer(shape, w, l)
        d[f"W{shape.head}"][...] *= factor
        d[f"b{shape.head}"][...] *= factor
    return w


def random_field(nd: int, L: int, B: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """[B][L^nd] FP64 Gaussian test fields (numpy Philox, independent of the method)."""
    gen = np.random.Generator(np.random.Philox(key=seed + 7919))
    return scale * gen.standard_normal((B, L ** nd))


# ---------------------------------------------------------------------------
# Workloads.  c1 is the paper's printed example (Sec. 3, example parameter
# file: 2D, L=8, m^2=-4, lambda=8, 16 layers, hidden [8, 8], batch 64);
# c2..c5 are the larger synthetic workloads the build is measured on.
# ---------------------------------------------------------------------------
WORKLOADS = {
    "c1": dict(shape=FlowShape(nd=2, L=8, n_layers=16, c1=8, c2=8),
               phi4=Phi4(m2=-4.0, lam=8.0), batch=64, chain=1024),
    "c2": dict(shape=FlowShape(nd=2, L=32, n_layers=24, c1=32, c2=32),
               phi4=Phi4(m2=-4.0, lam=8.0), batch=1024, chain=0),
    "c3": dict(shape=FlowShape(nd=3, L=16, n_layers=16, c1=32, c2=32),
               phi4=Phi4(m2=-6.0, lam=5.0), batch=4096, chain=100000),
    "c4": dict(nd=3, L=16, phi4=Phi4(m2=-6.0, lam=5.0), chains=512,
               n_steps=20, eps=0.05, trajectories=1000),
}


# ---------------------------------------------------------------------------
# Serving mix: resident models drawn from 2D L in {8,16,32,64} and 3D L in
# {8,12,16}, 12-24 couplings, hidden width in {8,16,24,32}; requests pick a model
# uniformly, (m2, lam) uniform in [-6,-2] x [1,10], batch log-uniform in
# [64, 8192], Poisson arrivals.
# ---------------------------------------------------------------------------
def serving_models(n_models: int, seed: int):
    """[(name, FlowShape, init seed)] for the serving mix."""
    rng = np.random.default_rng(seed)
    lattices = [(2, 8), (2, 16), (2, 32), (2, 64), (3, 8), (3, 12), (3, 16)]
    out = []
    for i in range(n_models):
        nd, L = lattices[int(rng.integers(len(lattices)))]
        c = int(rng.choice([8, 16, 24, 32]))
        n_layers = int(rng.integers(12, 25))
        out.append((f"m{i}", FlowShape(nd, L, n_layers, c, c), 1000 + i))
    return out


def serving_requests(n: int, model_names, seed: int, max_batch: int = 8192):
    """[(model name, m2, lam, batch, seed)] for n requests."""
    rng = np.random.default_rng(seed + 17)
    out = []
    for i in range(n):
        name = model_names[int(rng.integers(len(model_names)))]
        m2 = float(rng.uniform(-6.0, -2.0))
        lam = float(rng.uniform(1.0, 10.0))
        batch = int(round(float(np.exp(rng.uniform(np.log(64), np.log(max_batch))))))
        out.append((name, m2, lam, batch, 50000 + i))
    return out

"""FP64 CPU oracle of the flow-based phi^4 sampler (arXiv:2208.08903).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference arm of ``bench.py``.  The product path (the
CUDA library and its Python binding) never imports it.

The arithmetic lives in ``gf_oracle.c`` (plain C, FP64); this module builds it
with gcc into ``oracle/_build/`` and wraps it with ctypes.  Each wrapper takes
and returns numpy FP64 arrays in the canonical layouts ([B][V] fields, x
fastest; flat canonical weights as produced by ``gf_inputs.init_weights``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gf_oracle.c")
_HDR = os.path.join(_HERE, "gf_oracle.h")
_OUT = os.path.join(_HERE, "_build", "libgforacle.so")
_lib = None

BF16_H1, BF16_W2, BF16_H2, BF16_W3, BF16_W1, F32_IO, BF16_X1 = 1, 2, 4, 8, 16, 32, 64
F32_ACC = 128        # FP32-accumulating model (tolerance experiment only)
Z_JITTER = 256       # prior perturbed within its FP32 test bound (tolerance experiment only)
F16_X1, F16_W1, F16_H2, F16_W3 = 512, 1024, 2048, 4096
# the tensor-core precision mode: bf16 for conv2's operands (h1, W2), FP16 for
# conv1's input and weights and for conv3's operands (h2, W3), FP32 prior
BF16_MODE = BF16_H1 | BF16_W2 | F16_H2 | F16_W3 | F16_W1 | F32_IO | F16_X1
ALL_BF16_MODE = BF16_H1 | BF16_W2 | BF16_H2 | BF16_W3 | BF16_W1 | F32_IO | BF16_X1


def build(force: bool = False) -> str:
    """Compile gf_oracle.c into a shared library (gcc, -O3, OpenMP when available)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= newest:
        return _OUT
    tmp = _OUT + f".tmp{os.getpid()}"
    base = ["gcc", "-O3", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, _OUT)
    return _OUT


MAX_HIDDEN = 8


class Shape(C.Structure):
    _fields_ = [("nd", C.c_int32), ("L", C.c_int32), ("n_layers", C.c_int32),
                ("n_hidden", C.c_int32), ("hidden", C.c_int32 * MAX_HIDDEN), ("ksize", C.c_int32),
                ("use_final_tanh", C.c_int32), ("leaky_slope", C.c_double)]


class MHState(C.Structure):
    _fields_ = [("logw_cur", C.c_double), ("idx_cur", C.c_int64), ("n_acc", C.c_int64),
                ("step", C.c_int64), ("seed", C.c_uint64), ("stream_id", C.c_uint64)]


_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_U8 = C.POINTER(C.c_uint8)
_U64 = C.POINTER(C.c_uint64)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.gfo_philox4x64_10.argtypes = [_U64, _U64, _U64]
        L.gfo_prior.argtypes = [C.c_int64, C.c_int64, C.c_uint64, C.c_uint64, C.c_int32, _D]
        L.gfo_log_prior.argtypes = [C.c_int64, C.c_int64, _D, _D]
        L.gfo_action.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_int64, _D, _D]
        L.gfo_force.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_int64, _D, _D]
        L.gfo_coupling_net.argtypes = [C.POINTER(Shape), _D, C.c_int32, C.c_int32, _D, _D, _D]
        L.gfo_flow_sample.argtypes = [C.POINTER(Shape), _D, C.c_int32, C.c_double, C.c_double,
                                      C.c_int64, C.c_uint64, C.c_uint64, _D, _D, _D, _D, _D, _D,
                                      C.c_int32]
        L.gfo_flow_logq.argtypes = [C.POINTER(Shape), _D, C.c_int32, C.c_int64, _D, _D, _D, C.c_int32]
        L.gfo_mh_logu.argtypes = [C.c_uint64, C.c_uint64, C.c_int64, C.c_int64, _D]
        L.gfo_mh_scan.argtypes = [C.POINTER(MHState), C.c_int64, _D, _D, _I64, _U8]
        L.gfo_mh_chain.argtypes = [C.POINTER(MHState), C.c_int64, _D, _I64, _U8]
        L.gfo_hmc_trajectory.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_int64,
                                         _D, C.c_int32, C.c_double, C.c_uint64, C.c_uint64, _D,
                                         _U8, C.c_int32]
        L.gfo_leapfrog.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, _D, _D,
                                   C.c_int32, C.c_double]
        L.gfo_leapfrog.restype = C.c_double
        L.gfo_hmc_momenta.argtypes = [C.c_int64, C.c_uint64, C.c_uint64, C.c_uint64, _D]
        L.gfo_flow_loss_grad.argtypes = [C.POINTER(Shape), _D, C.c_double, C.c_double, C.c_int64,
                                         _D, _D, _D, C.c_int32]
        L.gfo_adam.argtypes = [C.c_int64, _D, _D, _D, _D, C.c_int64, C.c_double, C.c_double,
                               C.c_double, C.c_double]
        L.gfo_observables.argtypes = [C.c_int32, C.c_int32, C.c_int64, _D, _D, _D]
        L.gfo_autocorr.argtypes = [C.c_int64, _D, C.c_int32, _D]
        L.gfo_tau_int.argtypes = [C.c_int64, _D, C.c_int32, C.c_double, _D]
        L.gfo_ess.argtypes = [C.c_int64, _D]
        L.gfo_ess.restype = C.c_double
        _lib = L
    return _lib


def _p(a, t=_D):
    return None if a is None else a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def shape_struct(shape) -> Shape:
    """gfo_shape of any object with nd, L, n_layers, use_final_tanh, leaky_slope
    and either `hidden` (+ `ksize`) or c1, c2 (two hidden layers, 3 taps per axis)."""
    hidden = tuple(getattr(shape, "hidden", (shape.c1, shape.c2)))
    if len(hidden) > MAX_HIDDEN:
        raise ValueError(f"at most {MAX_HIDDEN} hidden convolutions")
    h = (C.c_int32 * MAX_HIDDEN)(*(list(hidden) + [0] * (MAX_HIDDEN - len(hidden))))
    return Shape(shape.nd, shape.L, shape.n_layers, len(hidden), h, int(getattr(shape, "ksize", 3)),
                 1 if shape.use_final_tanh else 0, shape.leaky_slope)


def philox(key, ctr) -> np.ndarray:
    k = np.asarray(key, dtype=np.uint64)
    c = np.asarray(ctr, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().gfo_philox4x64_10(_p(k, _U64), _p(c, _U64), _p(out, _U64))
    return out


def prior(V, B, seed, counter0, f32=True):
    z = np.zeros((B, V))
    lib().gfo_prior(V, B, seed, counter0, 1 if f32 else 0, _p(z))
    return z


def log_prior(z):
    z = _f64(np.atleast_2d(z))
    out = np.zeros(z.shape[0])
    lib().gfo_log_prior(z.shape[1], z.shape[0], _p(z), _p(out))
    return out


def action(nd, L, m2, lam, phi):
    phi = _f64(np.atleast_2d(phi))
    out = np.zeros(phi.shape[0])
    lib().gfo_action(nd, L, m2, lam, phi.shape[0], _p(phi), _p(out))
    return out


def force(nd, L, m2, lam, phi):
    phi = _f64(np.atleast_2d(phi))
    out = np.zeros_like(phi)
    lib().gfo_force(nd, L, m2, lam, phi.shape[0], _p(phi), _p(out))
    return out


def coupling_net(shape, w, layer, y, bf16_mask=0):
    w, y = _f64(w), _f64(y)
    s = np.zeros(shape.V)
    t = np.zeros(shape.V)
    sh = shape_struct(shape)
    rc = lib().gfo_coupling_net(C.byref(sh), _p(w), layer, bf16_mask, _p(y), _p(s), _p(t))
    assert rc == 0
    return s, t


def flow_sample(shape, w, m2, lam, B, seed=0, counter0=0, z=None, bf16_mask=F32_IO,
                nthreads=None):
    """Returns dict(z, phi, logq, S, logw) for B configurations."""
    w = _f64(w)
    V = shape.V
    zin = None if z is None else _f64(z).reshape(B, V)
    out = dict(z=np.zeros((B, V)), phi=np.zeros((B, V)), logq=np.zeros(B), S=np.zeros(B),
               logw=np.zeros(B))
    sh = shape_struct(shape)
    rc = lib().gfo_flow_sample(C.byref(sh), _p(w), bf16_mask, m2, lam, B, seed, counter0,
                               _p(zin), _p(out["z"]), _p(out["phi"]), _p(out["logq"]),
                               _p(out["S"]), _p(out["logw"]), nthreads or default_threads())
    assert rc == 0
    return out


def flow_logq(shape, w, phi, bf16_mask=0, nthreads=None):
    w = _f64(w)
    phi = _f64(np.atleast_2d(phi))
    B = phi.shape[0]
    z = np.zeros_like(phi)
    logq = np.zeros(B)
    sh = shape_struct(shape)
    rc = lib().gfo_flow_logq(C.byref(sh), _p(w), bf16_mask, B, _p(phi), _p(z), _p(logq),
                             nthreads or default_threads())
    assert rc == 0
    return z, logq


def mh_logu(seed, stream_id, step0, n):
    out = np.zeros(n)
    lib().gfo_mh_logu(seed, stream_id, step0, n, _p(out))
    return out


def new_mh_state(seed, stream_id=0):
    return MHState(0.0, 0, 0, 0, seed, stream_id)


def mh_scan(state: MHState, logw, logu):
    logw, logu = _f64(logw), _f64(logu)
    n = logw.size
    idx = np.zeros(n, dtype=np.int64)
    acc = np.zeros(n, dtype=np.uint8)
    lib().gfo_mh_scan(C.byref(state), n, _p(logw), _p(logu), _p(idx, _I64), _p(acc, _U8))
    return idx, acc


def mh_chain(state: MHState, logw):
    logw = _f64(logw)
    n = logw.size
    idx = np.zeros(n, dtype=np.int64)
    acc = np.zeros(n, dtype=np.uint8)
    lib().gfo_mh_chain(C.byref(state), n, _p(logw), _p(idx, _I64), _p(acc, _U8))
    return idx, acc


def hmc_trajectory(nd, L, m2, lam, phi, n_steps, eps, seed, traj_index, nthreads=None):
    """phi [n_chains][V] is copied; returns (phi_new, dH, acc)."""
    phi = _f64(np.atleast_2d(phi)).copy()
    n = phi.shape[0]
    dH = np.zeros(n)
    acc = np.zeros(n, dtype=np.uint8)
    lib().gfo_hmc_trajectory(nd, L, m2, lam, n, _p(phi), n_steps, eps, seed, traj_index,
                             _p(dH), _p(acc, _U8), nthreads or default_threads())
    return phi, dH, acc


def leapfrog(nd, L, m2, lam, phi, pi, n_steps, eps):
    phi = _f64(phi).copy()
    pi = _f64(pi).copy()
    dH = lib().gfo_leapfrog(nd, L, m2, lam, _p(phi), _p(pi), n_steps, eps)
    return phi, pi, dH


def hmc_momenta(V, seed, chain, traj):
    out = np.zeros(V)
    lib().gfo_hmc_momenta(V, seed, chain, traj, _p(out))
    return out


def flow_loss_grad(shape, w, m2, lam, z, nthreads=None):
    w = _f64(w)
    z = _f64(np.atleast_2d(z))
    loss = np.zeros(1)
    grad = np.zeros_like(w)
    sh = shape_struct(shape)
    rc = lib().gfo_flow_loss_grad(C.byref(sh), _p(w), m2, lam, z.shape[0], _p(z), _p(loss),
                                  _p(grad), nthreads or default_threads())
    assert rc == 0
    return float(loss[0]), grad


def adam(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place FP64 Adam on numpy arrays."""
    for a in (theta, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().gfo_adam(theta.size, _p(theta), _p(g), _p(m), _p(v), t, lr, beta1, beta2, eps)


def observables(nd, L, phi):
    """(M [B], C [B][L]) of fields phi [B][V] (see gfo_observables)."""
    phi = _f64(np.atleast_2d(phi))
    B = phi.shape[0]
    M = np.zeros(B)
    Cc = np.zeros((B, L))
    lib().gfo_observables(nd, L, B, _p(phi), _p(M), _p(Cc))
    return M, Cc


def autocorr(y, t_max):
    y = _f64(y)
    g = np.zeros(t_max + 1)
    lib().gfo_autocorr(y.size, _p(y), t_max, _p(g))
    return g


def tau_int(n, gamma, c=5.0):
    """(tau_int, W, error) from Gamma(0..t_max) of a series of length n."""
    gamma = _f64(gamma)
    out = np.zeros(3)
    lib().gfo_tau_int(n, _p(gamma), gamma.size - 1, c, _p(out))
    return float(out[0]), int(out[1]), float(out[2])


def ess(logw):
    logw = _f64(logw)
    return float(lib().gfo_ess(logw.size, _p(logw)))

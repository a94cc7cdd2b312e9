"""Torch-facing binding of libgfflow (argument marshalling only).

Every function here validates dtypes/devices, allocates output tensors with
torch and calls one C-ABI entry point on torch's current CUDA stream.  All
arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import torch

from . import _abi


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


def _need(t, dtype, name, numel=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")


def _phi4(phi4):
    if phi4 is None:
        return None
    m2, lam = (phi4.m2, phi4.lam) if hasattr(phi4, "m2") else phi4
    return _abi.Phi4C(float(m2), float(lam))


@dataclasses.dataclass
class SampleResult:
    phi: torch.Tensor
    logq: torch.Tensor
    S: torch.Tensor | None = None
    logw: torch.Tensor | None = None
    z: torch.Tensor | None = None


def _shape_ex(shape) -> _abi.FlowShapeExC:
    hidden = tuple(getattr(shape, "hidden", (shape.c1, shape.c2)))
    if len(hidden) > _abi.GF_MAX_HIDDEN:
        raise ValueError(f"at most {_abi.GF_MAX_HIDDEN} hidden convolutions")
    hid = (C.c_int32 * _abi.GF_MAX_HIDDEN)(*(list(hidden) + [0] * (_abi.GF_MAX_HIDDEN - len(hidden))))
    return _abi.FlowShapeExC(shape.nd, shape.L, shape.n_layers, len(hidden), hid,
                             int(getattr(shape, "ksize", 3)), 1 if shape.use_final_tanh else 0,
                             float(shape.leaky_slope))


def tensor_core_supported(shape) -> bool:
    """Whether Flow(shape, w, precision="bf16") has a tensor-core kernel
    (gf_flow_tensor_core_supported; host only)."""
    return bool(_abi.load().gf_flow_tensor_core_supported(C.byref(_shape_ex(shape))))


class Flow:
    """A RealNVP coupling stack resident on the current CUDA device.

    shape: any object with nd, L, n_layers, use_final_tanh, leaky_slope and
    either `hidden` (the hidden_sizes list) with `ksize`, or c1, c2 (two hidden
    convolutions, kernel size 3).
    weights: FP64 numpy array (or CPU tensor) in canonical layout.
    precision: "fp32" or "bf16" (BF16 tensor-core convolutions, sums to FP64 accuracy).
    """

    def __init__(self, shape, weights, precision: str = "fp32"):
        lib = _abi.load()
        self.shape = shape
        self.V = shape.L ** shape.nd
        sh = _shape_ex(shape)
        w = torch.as_tensor(weights, dtype=torch.float64).contiguous().cpu()
        prec = {"fp32": _abi.GF_PREC_FP32, "bf16": _abi.GF_PREC_BF16CONV_FP64RED}[precision]
        self.precision = precision
        h = C.c_void_p()
        _abi.check("gf_flow_create_ex", lib.gf_flow_create_ex(C.byref(sh), w.data_ptr(), prec,
                                                               _stream(), C.byref(h)))
        self._h = h
        self._lib = lib
        self.weights_version = 0      # bumped whenever the resident weights change
        self.n_params = int(lib.gf_flow_n_params(h))
        if self.n_params != w.numel():
            raise ValueError(f"weights have {w.numel()} entries, the shape needs {self.n_params}")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gf_flow_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def sample(self, B: int, seed: int = 0, counter0: int = 0, phi4=None, z=None,
               return_z: bool = False, out: SampleResult | None = None) -> SampleResult:
        dev = torch.device("cuda", torch.cuda.current_device())
        V = self.V
        if z is not None:
            _need(z, torch.float32, "z", B * V)
        if out is None:
            out = SampleResult(phi=torch.empty(B, V, device=dev),
                               logq=torch.empty(B, device=dev, dtype=torch.float64))
            if phi4 is not None:
                out.S = torch.empty(B, device=dev, dtype=torch.float64)
                out.logw = torch.empty(B, device=dev, dtype=torch.float64)
            if return_z:
                out.z = torch.empty(B, V, device=dev)
        p = _phi4(phi4)
        _abi.check("gf_flow_sample", self._lib.gf_flow_sample(
            self._h, C.byref(p) if p is not None else None, B, seed & (2**64 - 1),
            counter0 & (2**64 - 1), _ptr(z), _ptr(out.z), _ptr(out.phi), _ptr(out.logq),
            _ptr(out.S), _ptr(out.logw), _stream()))
        return out

    def unfused_workspace_bytes(self, B: int) -> int:
        return int(self._lib.gf_unfused_workspace_bytes(self._h, B))

    def sample_unfused(self, B: int, seed: int = 0, counter0: int = 0, phi4=None, z=None,
                       return_z: bool = False, out: SampleResult | None = None,
                       workspace: torch.Tensor | None = None) -> SampleResult:
        """gf_flow_sample_unfused: same results, one kernel per convolution."""
        dev = torch.device("cuda", torch.cuda.current_device())
        V = self.V
        if z is not None:
            _need(z, torch.float32, "z", B * V)
        if out is None:
            out = SampleResult(phi=torch.empty(B, V, device=dev),
                               logq=torch.empty(B, device=dev, dtype=torch.float64))
            if phi4 is not None:
                out.S = torch.empty(B, device=dev, dtype=torch.float64)
                out.logw = torch.empty(B, device=dev, dtype=torch.float64)
            if return_z:
                out.z = torch.empty(B, V, device=dev)
        nbytes = self.unfused_workspace_bytes(B)
        if workspace is None or workspace.numel() < nbytes:
            workspace = torch.empty(max(nbytes, 1), device=dev, dtype=torch.uint8)
        p = _phi4(phi4)
        _abi.check("gf_flow_sample_unfused", self._lib.gf_flow_sample_unfused(
            self._h, C.byref(p) if p is not None else None, B, seed & (2**64 - 1),
            counter0 & (2**64 - 1), _ptr(z), _ptr(out.z), _ptr(out.phi), _ptr(out.logq),
            _ptr(out.S), _ptr(out.logw), _ptr(workspace), workspace.numel(), _stream()))
        return out

    def logq(self, phi: torch.Tensor, return_z: bool = False):
        B = phi.shape[0]
        _need(phi, torch.float32, "phi", B * self.V)
        logq = torch.empty(B, device=phi.device, dtype=torch.float64)
        z = torch.empty_like(phi) if return_z else None
        _abi.check("gf_flow_logq", self._lib.gf_flow_logq(self._h, B, _ptr(phi), _ptr(z),
                                                          _ptr(logq), _stream()))
        return (z, logq) if return_z else logq

    def get_weights(self) -> torch.Tensor:
        w = torch.empty(self.n_params, device="cuda", dtype=torch.float32)
        _abi.check("gf_flow_get_weights_device",
                   self._lib.gf_flow_get_weights_device(self._h, _ptr(w), _stream()))
        return w

    def set_weights(self, w: torch.Tensor):
        _need(w, torch.float32, "w", self.n_params)
        _abi.check("gf_flow_set_weights_device",
                   self._lib.gf_flow_set_weights_device(self._h, _ptr(w), _stream()))
        self.weights_version += 1

    def train_workspace_bytes(self, B: int) -> int:
        return int(self._lib.gf_train_workspace_bytes(self._h, B))

    def train_step(self, B: int, phi4, seed: int = 0, counter0: int = 0, z=None, lr: float = 0.0,
                   adam_m=None, adam_v=None, adam_t: int = 0, beta1=0.9, beta2=0.999,
                   adam_eps=1e-8, grad: bool = True, workspace: torch.Tensor | None = None):
        """Returns (loss [1] FP64 tensor, grad [n_params] FP32 tensor or None)."""
        dev = torch.device("cuda", torch.cuda.current_device())
        if z is not None:
            _need(z, torch.float32, "z", B * self.V)
        nbytes = self.train_workspace_bytes(B)
        if workspace is None or workspace.numel() < nbytes:
            workspace = torch.empty(max(nbytes, 1), device=dev, dtype=torch.uint8)
        loss = torch.empty(1, device=dev, dtype=torch.float64)
        g = torch.empty(self.n_params, device=dev, dtype=torch.float32) if grad else None
        if lr > 0:
            _need(adam_m, torch.float32, "adam_m", self.n_params)
            _need(adam_v, torch.float32, "adam_v", self.n_params)
        p = _phi4(phi4)
        _abi.check("gf_flow_train_step", self._lib.gf_flow_train_step(
            self._h, C.byref(p), B, seed, counter0, _ptr(z), _ptr(loss), _ptr(g), float(lr),
            float(beta1), float(beta2), float(adam_eps), _ptr(adam_m), _ptr(adam_v), int(adam_t),
            _ptr(workspace), workspace.numel(), _stream()))
        if lr > 0:
            self.weights_version += 1
        return loss, g


    def adam_step(self, grad: torch.Tensor, lr: float, adam_m: torch.Tensor, adam_v: torch.Tensor,
                  adam_t: int, beta1=0.9, beta2=0.999, adam_eps=1e-8):
        """gf_flow_adam_step: one Adam update of the resident weights with `grad`."""
        for t, name in ((grad, "grad"), (adam_m, "adam_m"), (adam_v, "adam_v")):
            _need(t, torch.float32, name, self.n_params)
        _abi.check("gf_flow_adam_step", self._lib.gf_flow_adam_step(
            self._h, _ptr(grad), float(lr), float(beta1), float(beta2), float(adam_eps), _ptr(adam_m),
            _ptr(adam_v), int(adam_t), _stream()))
        self.weights_version += 1

    def forward_train(self, B: int, seed: int = 0, counter0: int = 0, z=None,
                      workspace: torch.Tensor | None = None):
        """Forward half of training: (phi [B][V] FP32, log q [B] FP64, workspace).

        The workspace keeps every layer's input for `backward`."""
        dev = torch.device("cuda", torch.cuda.current_device())
        if z is not None:
            _need(z, torch.float32, "z", B * self.V)
        nbytes = self.train_workspace_bytes(B)
        if workspace is None or workspace.numel() < nbytes:
            workspace = torch.empty(max(nbytes, 1), device=dev, dtype=torch.uint8)
        phi = torch.empty(B, self.V, device=dev, dtype=torch.float32)
        logq = torch.empty(B, device=dev, dtype=torch.float64)
        _abi.check("gf_flow_forward_train", self._lib.gf_flow_forward_train(
            self._h, B, seed, counter0, _ptr(z), _ptr(phi), _ptr(logq), _ptr(workspace),
            workspace.numel(), _stream()))
        return phi, logq, workspace

    def backward(self, B: int, gphi, glogq, workspace: torch.Tensor) -> torch.Tensor:
        """dLoss/dtheta [n_params] FP32 from dLoss/dphi (FP32 [B][V] or None) and
        dLoss/dlog q (FP64 [B] or None); `workspace` from the matching forward_train."""
        if gphi is not None:
            _need(gphi, torch.float32, "gphi", B * self.V)
        if glogq is not None:
            _need(glogq, torch.float64, "glogq", B)
        _need(workspace, torch.uint8, "workspace")
        g = torch.empty(self.n_params, device=workspace.device, dtype=torch.float32)
        _abi.check("gf_flow_backward", self._lib.gf_flow_backward(
            self._h, B, _ptr(gphi), _ptr(glogq), _ptr(g), _ptr(workspace), workspace.numel(),
            _stream()))
        return g


def phi4_action_vjp(nd: int, L: int, phi4, phi: torch.Tensor, gS: torch.Tensor) -> torch.Tensor:
    """gS[b] * dS/dphi_b for an FP32 field [B][V] (FP64 arithmetic, FP32 out)."""
    B = phi.shape[0]
    _need(phi, torch.float32, "phi", B * L**nd)
    _need(gS, torch.float64, "gS", B)
    out = torch.empty_like(phi)
    p = _phi4(phi4)
    _abi.check("gf_phi4_action_vjp", _abi.load().gf_phi4_action_vjp(
        nd, L, C.byref(p), B, _ptr(phi), _ptr(gS), _ptr(out), _stream()))
    return out


def phi4_action(nd: int, L: int, phi4, phi: torch.Tensor, out: torch.Tensor | None = None):
    if phi.dtype not in (torch.float32, torch.float64):
        raise ValueError("phi must be float32 or float64")
    B = phi.shape[0]
    _need(phi, phi.dtype, "phi", B * L**nd)
    if out is None:
        out = torch.empty(B, device=phi.device, dtype=torch.float64)
    p = _phi4(phi4)
    _abi.check("gf_phi4_action", _abi.load().gf_phi4_action(
        nd, L, C.byref(p), B, _ptr(phi), 1 if phi.dtype == torch.float64 else 0, _ptr(out),
        _stream()))
    return out


def phi4_force(nd: int, L: int, phi4, phi: torch.Tensor):
    B = phi.shape[0]
    _need(phi, torch.float64, "phi", B * L**nd)
    out = torch.empty_like(phi)
    p = _phi4(phi4)
    _abi.check("gf_phi4_force", _abi.load().gf_phi4_force(nd, L, C.byref(p), B, _ptr(phi),
                                                          _ptr(out), _stream()))
    return out


def new_mh_state(seed: int, stream_id: int = 0, device=None) -> torch.Tensor:
    """Device-resident gf_mh_state (48 bytes) as an int64[6] tensor."""
    st = _abi.MHStateC(0.0, 0, 0, 0, seed, stream_id)
    raw = torch.frombuffer(bytearray(bytes(st)), dtype=torch.int64).clone()
    return raw.to(device or torch.device("cuda", torch.cuda.current_device()))


def read_mh_state(state: torch.Tensor) -> _abi.MHStateC:
    b = state.detach().cpu().contiguous().numpy().tobytes()
    return _abi.MHStateC.from_buffer_copy(b)


def mh_chain_workspace_bytes(n: int) -> int:
    return int(_abi.load().gf_mh_chain_workspace_bytes(n))


def mh_chain(state: torch.Tensor, logw: torch.Tensor, workspace: torch.Tensor | None = None,
             chain_idx: torch.Tensor | None = None, acc: torch.Tensor | None = None):
    _need(state, torch.int64, "state", 6)
    n = logw.numel()
    _need(logw, torch.float64, "logw", n)
    if chain_idx is None:
        chain_idx = torch.empty(n, device=logw.device, dtype=torch.int64)
    if acc is None:
        acc = torch.empty(n, device=logw.device, dtype=torch.uint8)
    nbytes = mh_chain_workspace_bytes(n)
    if workspace is None or workspace.numel() * workspace.element_size() < nbytes:
        workspace = torch.empty(max(nbytes // 8, 1), device=logw.device, dtype=torch.float64)
    _abi.check("gf_mh_chain", _abi.load().gf_mh_chain(
        _ptr(state), n, _ptr(logw), _ptr(chain_idx), _ptr(acc), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _stream()))
    return chain_idx, acc


def mh_chain_noalloc(state: torch.Tensor, logw: torch.Tensor,
                     chain_idx: torch.Tensor | None = None, acc: torch.Tensor | None = None):
    """gf_mh_chain without caller workspace: the library's fixed device scratch
    holds log u (at most GF_MH_NOALLOC_MAX_N proposals per call; calls that
    overlap on the GPU must not be issued)."""
    _need(state, torch.int64, "state", 6)
    n = logw.numel()
    _need(logw, torch.float64, "logw", n)
    if chain_idx is None:
        chain_idx = torch.empty(n, device=logw.device, dtype=torch.int64)
    if acc is None:
        acc = torch.empty(n, device=logw.device, dtype=torch.uint8)
    _abi.check("gf_mh_chain_noalloc", _abi.load().gf_mh_chain_noalloc(
        _ptr(state), n, _ptr(logw), _ptr(chain_idx), _ptr(acc), _stream()))
    return chain_idx, acc


def hmc_trajectory(nd: int, L: int, phi4, phi: torch.Tensor, n_steps: int, eps: float,
                   seed: int, traj_index: int):
    """Updates phi [n_chains][V] (FP64) in place; returns (dH, acc)."""
    n = phi.shape[0]
    _need(phi, torch.float64, "phi", n * L**nd)
    dH = torch.empty(n, device=phi.device, dtype=torch.float64)
    acc = torch.empty(n, device=phi.device, dtype=torch.uint8)
    p = _phi4(phi4)
    _abi.check("gf_hmc_trajectory", _abi.load().gf_hmc_trajectory(
        nd, L, C.byref(p), n, _ptr(phi), n_steps, eps, seed, traj_index, _ptr(dH), _ptr(acc),
        _stream()))
    return dH, acc


def observables(nd: int, L: int, phi: torch.Tensor, magnetisation: bool = True,
                two_point: bool = True):
    """(M [B] FP64 or None, C [B][L] FP64 or None) of FP32 fields phi [B][V]."""
    B = phi.shape[0]
    _need(phi, torch.float32, "phi", B * L**nd)
    M = torch.empty(B, device=phi.device, dtype=torch.float64) if magnetisation else None
    Cc = torch.empty(B, L, device=phi.device, dtype=torch.float64) if two_point else None
    _abi.check("gf_observables", _abi.load().gf_observables(nd, L, B, _ptr(phi), _ptr(M), _ptr(Cc),
                                                            _stream()))
    return M, Cc


def chain_gather(chain_idx: torch.Tensor, values: torch.Tensor, idx0: int = 0) -> torch.Tensor:
    """values[chain_idx - idx0] (rows of an FP64 [n_values] or [n_values][width] tensor)."""
    _need(chain_idx, torch.int64, "chain_idx")
    _need(values, torch.float64, "values")
    n = chain_idx.numel()
    width = 1 if values.dim() == 1 else values.shape[1]
    out = torch.empty((n,) + tuple(values.shape[1:]), device=values.device, dtype=torch.float64)
    _abi.check("gf_chain_gather", _abi.load().gf_chain_gather(
        n, _ptr(chain_idx), idx0, values.shape[0], _ptr(values), width, _ptr(out), _stream()))
    return out


def autocorr(y: torch.Tensor, t_max: int, c_window: float = 5.0):
    """(Gamma [t_max+1], summary [4] = {tau_int, W, error, mean}) of an FP64 series."""
    _need(y, torch.float64, "y")
    gamma = torch.empty(t_max + 1, device=y.device, dtype=torch.float64)
    summ = torch.empty(4, device=y.device, dtype=torch.float64)
    _abi.check("gf_autocorr", _abi.load().gf_autocorr(y.numel(), _ptr(y), t_max, float(c_window),
                                                      _ptr(gamma), _ptr(summ), _stream()))
    return gamma, summ


def ess(logw: torch.Tensor) -> torch.Tensor:
    """ESS fraction (sum w)^2 / (n sum w^2) of w = exp(logw), as an FP64 [1] tensor."""
    _need(logw, torch.float64, "logw")
    out = torch.empty(1, device=logw.device, dtype=torch.float64)
    _abi.check("gf_ess", _abi.load().gf_ess(logw.numel(), _ptr(logw), _ptr(out), _stream()))
    return out


def device_status(stream=None) -> int:
    """gf_device_status: the status word of `stream` (its slot, else the
    process-wide word), read and cleared; 0 = no device-detected error."""
    v = C.c_int32(0)
    _abi.check("gf_device_status", _abi.load().gf_device_status(_stream(stream), C.byref(v)))
    return v.value


def set_stream_status_slot(stream, slot: torch.Tensor | None):
    """gf_set_stream_status_slot: kernels launched on `stream` record their
    errors in `slot` (one zeroed int32 CUDA element) instead of the
    process-wide word; None removes the association.  Keep `slot` alive while
    it is associated."""
    if slot is not None:
        _need(slot, torch.int32, "slot", 1)
    _abi.check("gf_set_stream_status_slot",
               _abi.load().gf_set_stream_status_slot(_stream(stream), _ptr(slot)))


def alu_peak(fp64: bool = False, iters: int = 1 << 16, packed: bool = False) -> float:
    """gf_alu_peak: measured FP32 FFMA, FP64 DFMA (fp64) or packed FP32x2 FMA
    (packed) throughput in FLOP/s."""
    v = C.c_double(0.0)
    kind = 1 if fp64 else (2 if packed else 0)
    _abi.check("gf_alu_peak", _abi.load().gf_alu_peak(kind, int(iters), C.byref(v), _stream()))
    return v.value

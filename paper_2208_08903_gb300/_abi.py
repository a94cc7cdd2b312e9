"""ctypes declarations of the C ABI in include/gfflow.h (libgfflow.so).

Loading fails loudly when the library has not been built: there is no
fallback implementation of any call.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

GF_OK, GF_EINVAL, GF_ENOMEM, GF_ECUDA, GF_EUNSUPPORTED, GF_ETIMEOUT, GF_EDEVICE = 0, -1, -2, -3, -4, -5, -6
GF_PREC_FP32, GF_PREC_BF16CONV_FP64RED = 0, 1
GF_OBS_MAX_L = 4096
GF_MH_NOALLOC_MAX_N = 131072     # include/gfflow.h

GF_MAX_HIDDEN = 8

EXPORTED = [
    "gf_flow_create", "gf_flow_create_ex", "gf_flow_tensor_core_supported", "gf_flow_destroy", "gf_flow_n_params",
    "gf_flow_set_weights_device",
    "gf_flow_get_weights_device", "gf_flow_sample", "gf_flow_logq", "gf_phi4_action",
    "gf_unfused_workspace_bytes", "gf_flow_sample_unfused",
    "gf_phi4_force", "gf_mh_chain_workspace_bytes", "gf_mh_chain", "gf_mh_chain_noalloc",
    "gf_hmc_trajectory",
    "gf_train_workspace_bytes", "gf_flow_train_step", "gf_flow_adam_step", "gf_flow_forward_train",
    "gf_flow_backward",
    "gf_phi4_action_vjp", "gf_observables", "gf_chain_gather", "gf_autocorr", "gf_ess",
    "gf_device_status", "gf_status_string", "gf_set_bf16_stall_test",
    "gf_set_stream_status_slot", "gf_alu_peak",
]


class FlowShapeC(C.Structure):
    _fields_ = [("nd", C.c_int32), ("L", C.c_int32), ("n_layers", C.c_int32),
                ("c_hidden1", C.c_int32), ("c_hidden2", C.c_int32), ("ksize", C.c_int32),
                ("use_final_tanh", C.c_int32), ("leaky_slope", C.c_double)]


class FlowShapeExC(C.Structure):
    _fields_ = [("nd", C.c_int32), ("L", C.c_int32), ("n_layers", C.c_int32),
                ("n_hidden", C.c_int32), ("hidden", C.c_int32 * GF_MAX_HIDDEN),
                ("ksize", C.c_int32), ("use_final_tanh", C.c_int32), ("leaky_slope", C.c_double)]


class Phi4C(C.Structure):
    _fields_ = [("m2", C.c_double), ("lam", C.c_double)]


class MHStateC(C.Structure):
    _fields_ = [("logw_cur", C.c_double), ("idx_cur", C.c_int64), ("n_acc", C.c_int64),
                ("step", C.c_int64), ("seed", C.c_uint64), ("stream_id", C.c_uint64)]


class GFError(RuntimeError):
    def __init__(self, call, code, lib=None):
        name = lib.gf_status_string(code).decode() if lib is not None else str(code)
        super().__init__(f"{call} failed: {name} ({code})")
        self.code = code


_lib = None
_VP, _I32, _I64, _U64, _F32, _F64, _SZ = (C.c_void_p, C.c_int32, C.c_int64, C.c_uint64,
                                          C.c_float, C.c_double, C.c_size_t)


def lib_path() -> str:
    return _build.LIB


def load():
    """Loads libgfflow.so (built by paper_2208_08903_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libgfflow.so is not built ({path}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'` first")
    L = C.CDLL(path)
    sig = {
        "gf_flow_create": ([C.POINTER(FlowShapeC), _VP, _I32, _VP, C.POINTER(_VP)], _I32),
        "gf_flow_create_ex": ([C.POINTER(FlowShapeExC), _VP, _I32, _VP, C.POINTER(_VP)], _I32),
        "gf_flow_tensor_core_supported": ([C.POINTER(FlowShapeExC)], _I32),
        "gf_flow_destroy": ([_VP], _I32),
        "gf_flow_n_params": ([_VP], _I64),
        "gf_flow_set_weights_device": ([_VP, _VP, _VP], _I32),
        "gf_flow_get_weights_device": ([_VP, _VP, _VP], _I32),
        "gf_flow_sample": ([_VP, C.POINTER(Phi4C), _I64, _U64, _U64, _VP, _VP, _VP, _VP, _VP,
                            _VP, _VP], _I32),
        "gf_flow_logq": ([_VP, _I64, _VP, _VP, _VP, _VP], _I32),
        "gf_unfused_workspace_bytes": ([_VP, _I64], _SZ),
        "gf_flow_sample_unfused": ([_VP, C.POINTER(Phi4C), _I64, _U64, _U64, _VP, _VP, _VP, _VP, _VP,
                                    _VP, _VP, _SZ, _VP], _I32),
        "gf_phi4_action": ([_I32, _I32, C.POINTER(Phi4C), _I64, _VP, _I32, _VP, _VP], _I32),
        "gf_phi4_force": ([_I32, _I32, C.POINTER(Phi4C), _I64, _VP, _VP, _VP], _I32),
        "gf_mh_chain_workspace_bytes": ([_I64], _SZ),
        "gf_mh_chain": ([_VP, _I64, _VP, _VP, _VP, _VP, _SZ, _VP], _I32),
        "gf_mh_chain_noalloc": ([_VP, _I64, _VP, _VP, _VP, _VP], _I32),
        "gf_hmc_trajectory": ([_I32, _I32, C.POINTER(Phi4C), _I64, _VP, _I32, _F64, _U64, _U64,
                               _VP, _VP, _VP], _I32),
        "gf_train_workspace_bytes": ([_VP, _I64], _SZ),
        "gf_flow_train_step": ([_VP, C.POINTER(Phi4C), _I64, _U64, _U64, _VP, _VP, _VP, _F32,
                                _F32, _F32, _F32, _VP, _VP, _I64, _VP, _SZ, _VP], _I32),
        "gf_flow_adam_step": ([_VP, _VP, _F32, _F32, _F32, _F32, _VP, _VP, _I64, _VP], _I32),
        "gf_flow_forward_train": ([_VP, _I64, _U64, _U64, _VP, _VP, _VP, _VP, _SZ, _VP], _I32),
        "gf_flow_backward": ([_VP, _I64, _VP, _VP, _VP, _VP, _SZ, _VP], _I32),
        "gf_phi4_action_vjp": ([_I32, _I32, C.POINTER(Phi4C), _I64, _VP, _VP, _VP, _VP], _I32),
        "gf_observables": ([_I32, _I32, _I64, _VP, _VP, _VP, _VP], _I32),
        "gf_chain_gather": ([_I64, _VP, _I64, _I64, _VP, _I32, _VP, _VP], _I32),
        "gf_autocorr": ([_I64, _VP, _I32, _F64, _VP, _VP, _VP], _I32),
        "gf_ess": ([_I64, _VP, _VP, _VP], _I32),
        "gf_device_status": ([_VP, C.POINTER(_I32)], _I32),
        "gf_set_bf16_stall_test": ([_I64], _I32),
        "gf_set_stream_status_slot": ([_VP, _VP], _I32),
        "gf_alu_peak": ([_I32, _I64, C.POINTER(_F64), _VP], _I32),
        "gf_status_string": ([_I32], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return _lib


def check(call: str, code: int):
    if code != GF_OK:
        raise GFError(call, code, _lib)

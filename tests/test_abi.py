"""The C-ABI library loads and exports every declared symbol; argument errors
are reported before any CUDA work (CPU only: no compute call is made)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gf_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2208_08903_gb300 import _abi, build
    build.build()
    return _abi.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2208_08903_gb300 import _abi
    decl = declared_symbols()
    assert len(decl) >= 16
    for name in decl:
        assert hasattr(lib, name), name
    assert set(decl) == set(_abi.EXPORTED) | (set(decl) - set(_abi.EXPORTED))
    assert set(_abi.EXPORTED) <= set(decl)


def test_argument_errors_without_gpu(lib):
    from paper_2208_08903_gb300 import _abi
    h = C.c_void_p()
    w = (C.c_double * 100)()
    bad = [
        _abi.FlowShapeC(2, 7, 2, 8, 8, 3, 1, 0.01),     # odd L
        _abi.FlowShapeC(4, 8, 2, 8, 8, 3, 1, 0.01),     # nd = 4
        _abi.FlowShapeC(2, 8, 2, 0, 16, 3, 1, 0.01),    # zero width
        _abi.FlowShapeC(2, 8, 2, 300, 8, 3, 1, 0.01),   # width > 256
        _abi.FlowShapeC(2, 8, 2, 8, 8, 4, 1, 0.01),     # even ksize
        _abi.FlowShapeC(2, 8, 2, 8, 8, 9, 1, 0.01),     # ksize > 7
        _abi.FlowShapeC(3, 64, 2, 8, 8, 3, 1, 0.01),    # V > 65536
    ]
    for sh in bad:
        assert lib.gf_flow_create(C.byref(sh), w, 0, None, C.byref(h)) == _abi.GF_EINVAL

    def ex(nd, L, n_layers, hidden, k, tanh=1):
        hid = (C.c_int32 * _abi.GF_MAX_HIDDEN)(*(list(hidden) + [0] * (_abi.GF_MAX_HIDDEN - len(hidden))))
        return _abi.FlowShapeExC(nd, L, n_layers, len(hidden), hid, k, tanh, 0.01)
    sh9 = ex(2, 8, 2, [8] * 8, 3)
    sh9.n_hidden = 9                                   # more than GF_MAX_HIDDEN hidden layers
    assert lib.gf_flow_create_ex(C.byref(sh9), w, 0, None, C.byref(h)) == _abi.GF_EINVAL
    assert lib.gf_flow_create_ex(C.byref(ex(2, 8, 2, [8, 8, 8], 6)), w, 0, None, C.byref(h)) == _abi.GF_EINVAL
    # the general network does not fit shared memory whole (2D L=64, two hidden layers of 32)
    big = ex(2, 64, 2, [32, 16], 5)
    assert lib.gf_flow_create_ex(C.byref(big), w, 0, None, C.byref(h)) == _abi.GF_EUNSUPPORTED
    # BF16 only for the slice-cached network form
    assert lib.gf_flow_create_ex(C.byref(ex(3, 16, 2, [32, 32, 32], 3)), w, 1, None, C.byref(h)) == \
        _abi.GF_EUNSUPPORTED
    assert lib.gf_flow_create(C.byref(_abi.FlowShapeC(3, 16, 2, 32, 16, 3, 1, 0.01)), w, 1, None,
                              C.byref(h)) == _abi.GF_EUNSUPPORTED
    good = _abi.FlowShapeC(2, 8, 2, 8, 8, 3, 1, 0.01)
    assert lib.gf_flow_create(C.byref(good), None, 0, None, C.byref(h)) == _abi.GF_EINVAL
    assert lib.gf_flow_create(C.byref(good), w, 7, None, C.byref(h)) == _abi.GF_EINVAL
    assert lib.gf_flow_create(C.byref(good), w, 0, None, None) == _abi.GF_EINVAL
    p = _abi.Phi4C(1.0, 1.0)
    assert lib.gf_phi4_action(4, 8, C.byref(p), 1, None, 0, None, None) == _abi.GF_EINVAL
    assert lib.gf_phi4_action(2, 8, None, 1, None, 0, None, None) == _abi.GF_EINVAL
    assert lib.gf_phi4_action(2, 8, C.byref(p), -1, None, 0, None, None) == _abi.GF_EINVAL
    assert lib.gf_phi4_action(2, 8, C.byref(p), 0, None, 0, None, None) == _abi.GF_OK
    assert lib.gf_mh_chain(None, 5, None, None, None, None, 0, None) == _abi.GF_EINVAL
    assert lib.gf_mh_chain_workspace_bytes(10) == 80
    fl = C.c_double()
    assert lib.gf_alu_peak(0, 4, C.byref(fl), None) == _abi.GF_EINVAL       # iters < 8
    assert lib.gf_alu_peak(3, 1024, C.byref(fl), None) == _abi.GF_EINVAL    # no such kind
    assert lib.gf_alu_peak(0, 1024, None, None) == _abi.GF_EINVAL
    assert lib.gf_mh_chain_workspace_bytes(0) == 0
    assert lib.gf_hmc_trajectory(2, 8, C.byref(p), 4, None, 0, 0.1, 0, 0, None, None, None) == _abi.GF_EINVAL
    assert lib.gf_hmc_trajectory(3, 32, C.byref(p), 4, None, 5, 0.1, 0, 0, None, None, None) == _abi.GF_EUNSUPPORTED
    assert lib.gf_flow_destroy(None) == _abi.GF_EINVAL
    assert lib.gf_flow_n_params(None) == -1
    assert lib.gf_status_string(-5) == b"GF_ETIMEOUT"


def test_product_path_has_no_oracle_dependency():
    """Nothing in the package imports, loads or names the oracle."""
    pkg = os.path.join(ROOT, "paper_2208_08903_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, fn)).read()
                assert "oracle" not in src.lower(), fn
                assert "gf_oracle" not in src and "gfo_" not in src, fn


def test_force_is_defined_once():
    """dS/dphi has one device definition (gf_common.cuh: phi4_force_at, and
    phi4_force_site that finds the neighbours first), used by gf_phi4_force,
    the action VJP, the HMC kicks and the training reverse pass; no kernel file
    writes the force formula itself."""
    csrc = os.path.join(ROOT, "paper_2208_08903_gb300", "csrc")
    users = 0
    for fn in os.listdir(csrc):
        src = open(os.path.join(csrc, fn)).read()
        if fn == "gf_common.cuh":
            assert src.count("4.0 * lam * c * c * c") == 1
            continue
        assert "4.0 * lam" not in src, fn
        users += "phi4_force_site(" in src or "phi4_force_at(" in src
    assert users >= 3


def test_tensor_core_support_query(lib):
    """gf_flow_tensor_core_supported (host only): the shapes with a tensor-core
    kernel are the two-equal-width networks of width 8, 16, 24 or 32 with
    kernel size 3 whose activations fit one block (or 3D L=16 with width 32);
    other widths and networks and invalid shapes answer 0."""
    from paper_2208_08903_gb300 import _abi

    def ex(nd, L, hidden, k=3):
        hid = (C.c_int32 * _abi.GF_MAX_HIDDEN)(*(list(hidden) + [0] * (_abi.GF_MAX_HIDDEN - len(hidden))))
        return _abi.FlowShapeExC(nd, L, 12, len(hidden), hid, k, 1, 0.01)

    yes = [(2, 8, [16, 16]), (2, 16, [24, 24]), (2, 32, [32, 32]), (2, 64, [16, 16]), (3, 8, [32, 32]),
           (3, 12, [16, 16]), (3, 16, [32, 32]), (3, 16, [16, 16]), (2, 32, [8, 8]), (2, 64, [8, 8]),
           (3, 16, [8, 8])]
    no = [(2, 64, [32, 32]), (3, 12, [32, 32]), (3, 16, [24, 24]), (2, 32, [12, 12]), (2, 32, [4, 4]),
          (2, 32, [40, 40]), (2, 32, [16, 32]), (2, 32, [16, 16, 16]), (2, 7, [16, 16])]
    for nd, L, h in yes:
        assert lib.gf_flow_tensor_core_supported(C.byref(ex(nd, L, h))) == 1, (nd, L, h)
    for nd, L, h in no:
        assert lib.gf_flow_tensor_core_supported(C.byref(ex(nd, L, h))) == 0, (nd, L, h)
    assert lib.gf_flow_tensor_core_supported(C.byref(ex(2, 32, [16, 16], k=5))) == 0
    assert lib.gf_flow_tensor_core_supported(None) == 0
    # the header's statement of which lattices fit, over the serving mix's
    # lattices and widths: 2D L <= 32 any width; 2D L = 64 and 3D L = 12, 16
    # widths 8 and 16 (3D L = 16 also 32, its own kernel); 3D L = 8 any width
    for nd, L in ((2, 8), (2, 16), (2, 32), (2, 64), (3, 8), (3, 12), (3, 16)):
        for c in (8, 16, 24, 32):
            want = (nd == 2 and L <= 32) or (nd == 3 and L == 8) or c <= 16 or (nd, L, c) == (3, 16, 32)
            assert lib.gf_flow_tensor_core_supported(C.byref(ex(nd, L, [c, c]))) == int(want), (nd, L, c)

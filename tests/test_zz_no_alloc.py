"""The allocation-free MH chain entry point agrees with the workspace one.

gf_mh_chain_noalloc serves callers that cannot allocate device memory where
they run the chain (a serving loop with a fixed budget from its own
allocator, a latency-critical thread that must not risk the device-wide
synchronisation a cudaMalloc can cause).  It keeps log u in a fixed device
array inside the library instead of caller workspace.  This test calls it
through the C ABI twice in a row, continuing one chain, and checks every
decision, chain index and the device state against gf_mh_chain on the same
log weights (integer results: exact).  The file is named to be collected
last, so a run that stops at the first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _state_tuple(P, st):
    s = P.read_mh_state(st)
    return (s.logw_cur, s.idx_cur, s.n_acc, s.step, s.seed, s.stream_id)


def test_noalloc_chain_matches_workspace_chain():
    torch, P = require_gpu()
    lib = P._abi.load()
    fn = lib.gf_mh_chain_noalloc
    rng = np.random.default_rng(11)
    n = 40000
    # mixed acceptance: blocks of near-constant log w (frequent accepts) and spread values
    logw = np.concatenate([-5.0 + 1e-3 * rng.standard_normal(n),
                           rng.standard_normal(n) * 3.0 - 50.0])
    seed, stream_id = 77, 5
    st_ref = P.new_mh_state(seed, stream_id)
    st_new = P.new_mh_state(seed, stream_id)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):                       # two calls in a row, one chain
        lw = torch.tensor(logw[call * n:(call + 1) * n], device="cuda")
        idx_ref, acc_ref = P.mh_chain(st_ref, lw)
        idx_new = torch.full((n,), -7, device="cuda", dtype=torch.int64)
        acc_new = torch.full((n,), 9, device="cuda", dtype=torch.uint8)
        rc = fn(C.c_void_p(st_new.data_ptr()), n, C.c_void_p(lw.data_ptr()),
                C.c_void_p(idx_new.data_ptr()), C.c_void_p(acc_new.data_ptr()), C.c_void_p(stream))
        assert rc == P._abi.GF_OK
        torch.cuda.synchronize()
        assert torch.equal(idx_new, idx_ref)
        assert torch.equal(acc_new, acc_ref)
        assert _state_tuple(P, st_new) == _state_tuple(P, st_ref)
    assert P.read_mh_state(st_new).step == 2 * n
    assert 0 < P.read_mh_state(st_new).n_acc < 2 * n - 1
    # the binding's wrapper reaches the same entry point
    lw = torch.tensor(logw[:1000], device="cuda")
    a = P.new_mh_state(1, 0)
    b = P.new_mh_state(1, 0)
    i1, c1 = P.mh_chain(a, lw)
    i2, c2 = P.mh_chain_noalloc(b, lw)
    assert torch.equal(i1, i2) and torch.equal(c1, c2)


def test_noalloc_rejects_oversize_and_bad_arguments():
    torch, P = require_gpu()
    lib = P._abi.load()
    st = P.new_mh_state(1, 0)
    big = P._abi.GF_MH_NOALLOC_MAX_N + 1
    lw = torch.zeros(big, device="cuda", dtype=torch.float64)
    out_i = torch.empty(big, device="cuda", dtype=torch.int64)
    out_a = torch.empty(big, device="cuda", dtype=torch.uint8)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.gf_mh_chain_noalloc(C.c_void_p(st.data_ptr()), big, C.c_void_p(lw.data_ptr()),
                                 C.c_void_p(out_i.data_ptr()), C.c_void_p(out_a.data_ptr()), stream)
    assert rc == P._abi.GF_EINVAL
    assert lib.gf_mh_chain_noalloc(None, 10, C.c_void_p(lw.data_ptr()), None, None, stream) == P._abi.GF_EINVAL
    assert lib.gf_mh_chain_noalloc(C.c_void_p(st.data_ptr()), 0, None, None, None, stream) == P._abi.GF_OK
    assert P.read_mh_state(st).step == 0       # nothing ran

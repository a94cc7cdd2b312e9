"""Helpers shared by the GPU parity tests: tolerance checks against the oracle."""
import json
import os

import numpy as np
import pytest

# Plain FP32 path: 1e-5 relative per site, 1e-4 relative per log-weight.
SITE_RTOL = 1e-5
LOGW_RTOL = 1e-4

# Tensor-core path: compared with the oracle's emulation of its rounding points
# (h1 and W2 to bf16; conv1's input and weights, h2 and W3 to FP16; FP32
# prior).  Its tolerances come from a CPU experiment on the oracle alone
# (tests/golden/bf16_tolerance.py): the drift that FP32-level differences
# before those roundings produce, maximum over 64 configurations times a
# margin, per number of coupling layers.
BF16_MODE = 1 | 2 | 2048 | 4096 | 1024 | 32 | 512
_BF16_TOL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bf16_tolerance.json")
# The tensor-core kernel for the other lattice shapes rounds h1 and W2 to bf16
# and h2 and W3 to FP16 (conv1 stays FP32); its bounds come from the same
# experiment over 2D and 3D shapes of the serving mix
# (tests/golden/tc_tolerance.json).
TC_MODE = 1 | 2 | 2048 | 4096 | 32
_TC_TOL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tc_tolerance.json")


def _pick_tolerance(path, n_layers):
    with open(path) as f:
        by = json.load(f)["by_layers"]
    counts = sorted(int(k) for k in by)
    pick = next((c for c in counts if c >= n_layers), None)
    if pick is None:
        raise ValueError(f"no tolerance measured for {n_layers} coupling layers in {path} (have {counts})")
    e = by[str(pick)]
    return float(e["site_rtol"]), float(e["scalar_rtol"])


def tc_tolerances(n_layers: int):
    """(per-site rtol, per-result rtol) of the second tensor-core kernel for a
    flow of n_layers coupling layers (the smallest measured count >= n_layers)."""
    return _pick_tolerance(_TC_TOL, n_layers)


def bf16_tolerances(n_layers: int):
    """(per-site rtol, per-result rtol for log q / S / log w) for a flow of
    n_layers coupling layers: the bound measured for the smallest layer count
    in the experiment that is >= n_layers (the drift grows with depth)."""
    return _pick_tolerance(_BF16_TOL, n_layers)


def bf16_site_rtol(n_layers: int) -> float:
    return bf16_tolerances(n_layers)[0]


def bf16_logw_rtol(n_layers: int) -> float:
    return bf16_tolerances(n_layers)[1]


def bf16_drift_model(n_layers: int) -> dict:
    """The experiment's error statistics (max / p99 / mean per result) of the
    FP32-accumulating model against the FP64-summing emulation."""
    with open(_BF16_TOL) as f:
        return json.load(f)["by_layers"][str(n_layers)]["fp32_model_vs_emulated"]


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_08903_gb300 as P
    P._abi.load()        # raises if the library was not built
    return torch, P


def assert_sites_close(gpu, ref, rtol=SITE_RTOL, what="phi"):
    """|a-b| <= rtol * max(|b|, rms(b of that configuration)) for every site."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape
    rms = np.sqrt((ref**2).mean(axis=-1, keepdims=True))
    bound = rtol * np.maximum(np.abs(ref), rms)
    err = np.abs(gpu - ref)
    bad = err > bound
    if bad.any():
        i = np.unravel_index(np.argmax(err / np.maximum(bound, 1e-300)), err.shape)
        raise AssertionError(f"{what}: {bad.sum()} sites out of tolerance; worst at {i}: "
                             f"gpu={gpu[i]!r} ref={ref[i]!r} bound={bound[i]!r}")
    return float((err / np.maximum(np.maximum(np.abs(ref), rms), 1e-300)).max())


def assert_logw_close(gpu, ref, rtol=LOGW_RTOL, what="logw"):
    """|a-b| <= rtol * max(|b|, 1) per configuration."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    bound = rtol * np.maximum(np.abs(ref), 1.0)
    err = np.abs(gpu - ref)
    bad = err > bound
    if bad.any():
        i = int(np.argmax(err / bound))
        raise AssertionError(f"{what}: {bad.sum()} entries out of tolerance; worst at {i}: "
                             f"gpu={gpu[i]!r} ref={ref[i]!r} bound={bound[i]!r}")
    return float((err / np.maximum(np.abs(ref), 1.0)).max())


def compare_mh(orc, st_seed, stream_id, logw, idx_gpu, acc_gpu, step0=0, logw_tol=0.0):
    """MH decisions must match the oracle's except at near ties.

    A decision may differ only where |(logw_k - log u_k) - logw_cur| < tau with
    tau = 4 * logw_tol * max(|logw|, 1) + 1e-12 (the two sides evaluate log u
    with their own log); after such a divergence the comparison resumes from
    the oracle's state.  Returns the number of tolerated divergences.
    """
    logw = np.asarray(logw, dtype=np.float64)
    n = logw.size
    logu = orc.mh_logu(st_seed, stream_id, step0, n)
    cur, idx = 0.0, 0
    diverged = 0
    for k in range(n):
        g = step0 + k
        d = logw[k] - logu[k]
        acc = True if g == 0 else d > cur
        if bool(acc_gpu[k]) != acc:
            tau = 4 * logw_tol * max(abs(logw[k]), abs(cur), 1.0) + 1e-12
            assert g > 0 and abs(d - cur) < tau, (
                f"MH decision {k} differs: gpu={acc_gpu[k]} oracle={acc} margin={d - cur}")
            diverged += 1
        if acc:
            cur, idx = logw[k], g
        if bool(acc_gpu[k]) == acc:
            assert idx_gpu[k] == idx or diverged, f"chain index {k}: {idx_gpu[k]} != {idx}"
    return diverged


def assert_grad_close(g, ref):
    """Relative L2 error <= 1e-3, and per entry |a-b| <= max(1e-2 |b|, 1e-4 max|b|).

    The absolute floor is a fraction of the largest gradient entry because the
    reverse pass runs in FP32 through every coupling layer: the rounding error
    carried by the adjoint of x grows with the gradient's overall scale, so an
    entry that is small only through cancellation keeps an error of that scale.
    """
    g = np.asarray(g, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    rel = np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-300)
    assert rel <= 1e-3, f"relative L2 gradient error {rel:.3e}"
    bound = np.maximum(1e-2 * np.abs(ref), 1e-4 * np.abs(ref).max())
    ratio = np.abs(g - ref) / bound
    i = int(np.argmax(ratio))
    assert ratio[i] <= 1.0, (f"{(ratio > 1).sum()} gradient entries out of tolerance; worst {i}: "
                             f"gpu={g[i]!r} ref={ref[i]!r} bound={bound[i]!r}")
    return rel

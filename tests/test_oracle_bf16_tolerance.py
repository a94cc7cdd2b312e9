"""The BF16 path's parity tolerances come from a committed oracle experiment.

tests/golden/bf16_tolerance.py runs the oracle's BF16-emulation mode with FP64
sums and with its FP32-accumulating model (GFO_F32_ACC) on the same inputs and
stores the drift between them; the GPU tests use twice its maximum.  These
CPU tests check the stored file against a fresh run of the same experiment on
a subset, and pin the FP32-accumulating model itself.
"""
import json
import os

import numpy as np
import pytest

import gf_inputs as gi

HERE = os.path.dirname(os.path.abspath(__file__))
STORED = os.path.join(HERE, "golden", "bf16_tolerance.json")


def _load_script():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bf16_tolerance", os.path.join(HERE, "golden", "bf16_tolerance.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_stored_bounds_follow_from_stored_drift():
    with open(STORED) as f:
        d = json.load(f)
    assert set(d["by_layers"]) == {"2", "16"}
    for n, e in d["by_layers"].items():
        assert e["configurations"] >= 64 and e["n_layers"] == int(n)
        m = e["fp32_model_vs_emulated"]
        assert e["site_rtol"] == pytest.approx(d["margin"] * m["phi"]["max"], rel=1e-12)
        assert e["scalar_rtol"] == pytest.approx(
            d["margin"] * max(m[k]["max"] for k in ("logq", "S", "logw")), rel=1e-12)
        # the drift is a small fraction of the BF16 path's own error against FP64
        f = e["emulated_vs_fp64"]
        assert m["phi"]["p99"] < f["phi"]["p99"] and m["logw"]["max"] < f["logw"]["max"]
    # deeper flows drift further
    assert d["by_layers"]["16"]["site_rtol"] > d["by_layers"]["2"]["site_rtol"]


def test_fresh_subset_reproduces_stored_drift(orc):
    """The first 4 of the stored 64 configurations (2 coupling layers): each
    configuration's prior counter is independent of the batch, so the subset's
    drift must be reproduced exactly and lie within the stored maxima."""
    mod = _load_script()
    r = mod.drift(2, 4)
    with open(STORED) as f:
        st = json.load(f)["by_layers"]["2"]
    for k in ("phi", "logq", "S", "logw"):
        got = r["fp32_model_vs_emulated"][k]["max"]
        assert 0.0 < got <= st["fp32_model_vs_emulated"][k]["max"], (k, got)
        got64 = r["emulated_vs_fp64"][k]["max"]
        assert 0.0 < got64 <= st["emulated_vs_fp64"][k]["max"], (k, got64)


def test_fp32_accumulation_model_is_fp32_close(orc):
    """Without bf16 rounding, the FP32-accumulating model differs from the
    FP64 oracle only by FP32 rounding: every per-layer net output stays within
    the forward error bound of an FP32 sum of K terms (K u sum|terms|, with
    u = 2^-24, K = taps x channels), and it is not identical (the mode acts)."""
    shape = gi.FlowShape(2, 6, 2, 8, 8, use_final_tanh=False)
    w = gi.init_weights(shape, seed=3)
    y = gi.random_field(2, 6, 1, seed=5)[0]
    s64, t64 = orc.coupling_net(shape, w, 0, y)
    s32, t32 = orc.coupling_net(shape, w, 0, y, bf16_mask=orc.F32_ACC)
    assert not (np.array_equal(s32, s64) and np.array_equal(t32, t64))
    # error scale: conv3 sums 8 channels x 9 taps of O(1) terms; the inputs carry
    # the error of conv1/conv2 sums of similar size
    bound = 3 * 72 * 2.0**-24 * (np.abs(s64).max() + np.abs(t64).max() + 1.0) * 8
    assert np.abs(s32 - s64).max() < bound and np.abs(t32 - t64).max() < bound
    # a flow sample in the model agrees with FP64 to FP32 level per site
    out64 = orc.flow_sample(shape, w, -4.0, 8.0, 2, seed=1, counter0=0)
    out32 = orc.flow_sample(shape, w, -4.0, 8.0, 2, seed=1, counter0=0, bf16_mask=orc.F32_IO | orc.F32_ACC)
    rms = np.sqrt((out64["phi"] ** 2).mean(1, keepdims=True))
    e = np.abs(out32["phi"] - out64["phi"]) / np.maximum(np.abs(out64["phi"]), rms)
    assert 0.0 < e.max() < 1e-5


TC_STORED = os.path.join(HERE, "golden", "tc_tolerance.json")


def test_tc_stored_bounds_follow_from_stored_drift():
    """tests/golden/tc_tolerance.json (the tensor-core kernel for the other
    lattice shapes): per coupling-layer count, each bound is the margin times
    the largest drift over the shapes; the shapes cover 2D and 3D and every
    hidden width that kernel takes; the emulation mode is the one the GPU tests
    compare against; deeper flows get wider bounds."""
    from gpu_util import TC_MODE
    with open(TC_STORED) as f:
        d = json.load(f)
    assert d["mode"] == TC_MODE
    shapes = [tuple(s) for s in d["shapes"]]
    assert {s[0] for s in shapes} == {2, 3} and {s[2] for s in shapes} == {8, 16, 24, 32}
    assert set(d["by_layers"]) == {"2", "8", "24"}
    prev = 0.0
    for n in ("2", "8", "24"):
        e = d["by_layers"][n]
        assert e["configurations_per_shape"] >= 64 and e["n_layers"] == int(n)
        assert set(e["by_shape"]) == {f"{nd}D L={L} C={c}" for nd, L, c in shapes}
        drift = [v["fp32_model_vs_emulated"] for v in e["by_shape"].values()]
        assert e["site_rtol"] == pytest.approx(d["margin"] * max(m["phi"]["max"] for m in drift), rel=1e-12)
        assert e["scalar_rtol"] == pytest.approx(
            d["margin"] * max(m[k]["max"] for m in drift for k in ("logq", "S", "logw")), rel=1e-12)
        assert e["site_rtol"] > prev
        prev = e["site_rtol"]


def test_tc_fresh_subset_reproduces_stored_drift(orc):
    """The first 2 of each shape's stored 64 configurations (2 coupling
    layers), run afresh: every shape's drift, and the emulation's error
    against FP64, lie within the stored maxima (the prior counter of a
    configuration does not depend on the batch)."""
    mod = _load_script()
    r = mod.drift_tc(2, 2)
    with open(TC_STORED) as f:
        st = json.load(f)["by_layers"]["2"]["by_shape"]
    assert set(r["by_shape"]) == set(st)
    for name, v in r["by_shape"].items():
        for k in ("phi", "logq", "S", "logw"):
            got = v["fp32_model_vs_emulated"][k]["max"]
            assert 0.0 < got <= st[name]["fp32_model_vs_emulated"][k]["max"], (name, k, got)
            got64 = v["emulated_vs_fp64"][k]["max"]
            assert 0.0 < got64 <= st[name]["emulated_vs_fp64"][k]["max"], (name, k, got64)

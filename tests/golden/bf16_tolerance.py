"""Derives the parity tolerances of the tensor-core path from the oracle alone.

The tensor-core kernel rounds h1 and W2 to bf16 and conv1's input and
weights, h2 and W3 to FP16, at the same points as the oracle's emulation mode
(oracle.BF16_MODE), but it forms every convolution sum in FP32 on the tensor
cores where the oracle sums in FP64.  So the two reach each rounding with
values that differ at the FP32 level, and a value that sits within that
difference of a rounding boundary rounds the other way on one side.  Such a flip moves s and t of the nearby
updated sites by part of a bf16 ulp, and the later coupling layers carry it on.

The kernel's prior sample also differs from the oracle's at the FP32 level:
it evaluates Box-Muller in FP32 (tested against the oracle to 1e-6 relative),
the oracle in FP64 before rounding to FP32.

This script measures the drift with the oracle only: it runs the
BF16-emulation mode twice on the same inputs, once with FP64 sums (the mode
the GPU tests compare against) and once as a model of an FP32 device: every
convolution summed in FP32, the field kept in FP32 (GFO_F32_ACC), and each
prior sample perturbed by a relative amount uniform in +-2^-20, the prior's
tested bound (GFO_Z_JITTER).  The difference between the two runs is the size of error that
FP32-level differences produce through the bf16 roundings; the GPU tolerance
is its maximum over the sample times a stated margin, per number of coupling
layers.  It also reports the BF16-emulated results' error against the pure
FP64 oracle.

Inputs: 3D L=16, hidden 32, m2=-6, lam=5 (the 3D workload's theory),
Kaiming-uniform weights from seed 0, the FP32 prior from seed 77 (not the
seeds of the GPU tests), 64 configurations per layer count.

    python tests/golden/bf16_tolerance.py          # writes bf16_tolerance.json
    python tests/golden/bf16_tolerance.py --tc     # writes tc_tolerance.json (second kernel)
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import gf_inputs as gi  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(HERE, "bf16_tolerance.json")
MARGIN = 2.0
SEED = 77
LAYERS = (2, 16)


def site_err(a, ref):
    rms = np.sqrt((ref ** 2).mean(1, keepdims=True))
    return np.abs(a - ref) / np.maximum(np.abs(ref), rms)


def scalar_err(a, ref):
    return np.abs(a - ref) / np.maximum(np.abs(ref), 1.0)


def stats(e):
    e = np.asarray(e, np.float64).ravel()
    return {"max": float(e.max()), "p99": float(np.percentile(e, 99)), "mean": float(e.mean())}


def drift(n_layers: int, B: int, seed: int = SEED, counter0: int = 0, nthreads=None) -> dict:
    """Per-result error statistics of the FP32-accumulating model against the
    FP64-summing BF16 emulation, and of the latter against pure FP64."""
    shape = gi.FlowShape(3, 16, n_layers, 32, 32)
    w = gi.init_weights(shape, seed=0)
    m2, lam = -6.0, 5.0
    kw = dict(seed=seed, counter0=counter0, nthreads=nthreads)
    ref = oracle.flow_sample(shape, w, m2, lam, B, bf16_mask=oracle.BF16_MODE, **kw)
    f32 = oracle.flow_sample(shape, w, m2, lam, B,
                             bf16_mask=oracle.BF16_MODE | oracle.F32_ACC | oracle.Z_JITTER, **kw)
    f64 = oracle.flow_sample(shape, w, m2, lam, B, bf16_mask=oracle.F32_IO, **kw)
    out = {"n_layers": n_layers, "configurations": B,
           "fp32_model_vs_emulated": {"phi": stats(site_err(f32["phi"], ref["phi"]))},
           "emulated_vs_fp64": {"phi": stats(site_err(ref["phi"], f64["phi"]))}}
    for k in ("logq", "S", "logw"):
        out["fp32_model_vs_emulated"][k] = stats(scalar_err(f32[k], ref[k]))
        out["emulated_vs_fp64"][k] = stats(scalar_err(ref[k], f64[k]))
    d = out["fp32_model_vs_emulated"]
    out["site_rtol"] = MARGIN * d["phi"]["max"]
    out["scalar_rtol"] = MARGIN * max(d[k]["max"] for k in ("logq", "S", "logw"))
    return out


# The tensor-core kernel for the other lattice shapes (2D L = 8..64, 3D L = 8,
# 12, 16; hidden 8, 16, 24 or 32) rounds h1 and W2 to bf16 and h2 and W3 to
# FP16 and keeps conv1 in FP32; its bounds take the maximum drift over these
# shapes (serving flows have 12 to 24 coupling layers).
TC_MODE = oracle.BF16_H1 | oracle.BF16_W2 | oracle.F16_H2 | oracle.F16_W3 | oracle.F32_IO
TC_SHAPES = ((2, 16, 24), (2, 32, 32), (2, 64, 16), (3, 8, 32), (3, 12, 16), (2, 32, 8), (3, 16, 8))
TC_LAYERS = (2, 8, 24)
TC_OUT = os.path.join(HERE, "tc_tolerance.json")


def drift_tc(n_layers: int, B: int, seed: int = SEED, nthreads=None) -> dict:
    """drift() for the second tensor-core kernel's rounding points, per shape
    of TC_SHAPES (m2 = -4, lam = 6), and the bounds over all of them."""
    out = {"n_layers": n_layers, "configurations_per_shape": B, "by_shape": {}}
    worst_site = worst_scalar = 0.0
    for nd, L, c in TC_SHAPES:
        shape = gi.FlowShape(nd, L, n_layers, c, c)
        w = gi.init_weights(shape, seed=0)
        kw = dict(seed=seed, counter0=0, nthreads=nthreads)
        ref = oracle.flow_sample(shape, w, -4.0, 6.0, B, bf16_mask=TC_MODE, **kw)
        f32 = oracle.flow_sample(shape, w, -4.0, 6.0, B,
                                 bf16_mask=TC_MODE | oracle.F32_ACC | oracle.Z_JITTER, **kw)
        f64 = oracle.flow_sample(shape, w, -4.0, 6.0, B, bf16_mask=oracle.F32_IO, **kw)
        r = {"fp32_model_vs_emulated": {"phi": stats(site_err(f32["phi"], ref["phi"]))},
             "emulated_vs_fp64": {"phi": stats(site_err(ref["phi"], f64["phi"]))}}
        for k in ("logq", "S", "logw"):
            r["fp32_model_vs_emulated"][k] = stats(scalar_err(f32[k], ref[k]))
            r["emulated_vs_fp64"][k] = stats(scalar_err(ref[k], f64[k]))
        d = r["fp32_model_vs_emulated"]
        worst_site = max(worst_site, d["phi"]["max"])
        worst_scalar = max(worst_scalar, max(d[k]["max"] for k in ("logq", "S", "logw")))
        out["by_shape"][f"{nd}D L={L} C={c}"] = r
    out["site_rtol"] = MARGIN * worst_site
    out["scalar_rtol"] = MARGIN * worst_scalar
    return out


def main_tc():
    res = {"what": "parity tolerances of the tensor-core kernel for the lattice shapes other than "
                   "3D L=16 C=32, per coupling-layer count (FP32-accumulating model vs the FP64-summing "
                   "emulation of its rounding points: h1, W2 in bf16, h2, W3 in fp16)",
           "mode": TC_MODE, "margin": MARGIN, "shapes": [list(s) for s in TC_SHAPES],
           "theory": "m2=-4, lam=6, weights seed 0", "prior_seed": SEED,
           "command": "python tests/golden/bf16_tolerance.py --tc", "by_layers": {}}
    for n in TC_LAYERS:
        r = drift_tc(n, 64)
        res["by_layers"][str(n)] = r
        print(n, r["site_rtol"], r["scalar_rtol"], flush=True)
    with open(TC_OUT, "w") as f:
        json.dump(res, f, indent=1)
    print("wrote", TC_OUT)


def main():
    oracle.build()
    if "--tc" in sys.argv[1:]:
        main_tc()
        return
    res = {"what": "BF16 path parity tolerances per coupling-layer count, derived from the oracle "
                   "(FP32-accumulating model vs the FP64-summing BF16 emulation)",
           "margin": MARGIN, "shape": "3D L=16, hidden 32, m2=-6, lam=5, weights seed 0",
           "prior_seed": SEED, "command": "python tests/golden/bf16_tolerance.py", "by_layers": {}}
    for n in LAYERS:
        r = drift(n, 64)
        res["by_layers"][str(n)] = r
        print(json.dumps(r), flush=True)
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()

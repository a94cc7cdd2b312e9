"""Continuous-batching request loop: each result is the same alone and in the mix.

Requests of different lattice sizes, dimensions and couplings are admitted as
slots and HBM budget free up; their chunks overlap on the GPU on separate
streams.  Every request's phi, log q, S, log w, chain indices, accept flags and
final chain state must be bit-identical to the same request served alone, and
one FP32 request is checked against the FP64 oracle and one request on the
2D tensor-core kernel against the oracle's emulation of its rounding points.
"""
import numpy as np
import pytest

import gf_inputs as gi
from gpu_util import (LOGW_RTOL, SITE_RTOL, TC_MODE, assert_logw_close, assert_sites_close, require_gpu,
                      tc_tolerances)

pytestmark = pytest.mark.gpu


def _models(P):
    specs = [("a", gi.FlowShape(2, 8, 4, 8, 8), 1), ("b", gi.FlowShape(3, 4, 3, 16, 16), 2),
             ("c", gi.FlowShape(2, 16, 6, 16, 16), 3), ("d", gi.FlowShape(3, 16, 2, 32, 32), 4)]
    from paper_2208_08903_gb300 import serving
    models = {}
    for name, shape, s in specs:
        # the tensor-core kernels (b, c: gf_flow_tc.cu; d: the 3D L=16 kernel)
        # next to one FP32 flow (a)
        prec = "bf16" if name != "a" and P.tensor_core_supported(shape) else "fp32"
        models[name] = serving.Model(name, shape, P.Flow(shape, gi.init_weights(shape, seed=s), precision=prec))
    return models, {n: (sh, s) for n, sh, s in specs}


def test_results_same_alone_and_in_mix(orc):
    torch, P = require_gpu()
    from paper_2208_08903_gb300 import serving
    models, specs = _models(P)
    rng = np.random.default_rng(0)
    names = list(models)
    reqs = [serving.Request(i, names[i % 4], float(rng.uniform(-6, -2)), float(rng.uniform(1, 10)),
                            int(rng.integers(5, 300)), 900 + i, arrival=0.0) for i in range(14)]
    budget = 6 << 20
    with serving.Server(models, hbm_budget_bytes=budget, max_active=4, chunk=64) as srv:
        mix, stats = srv.run(reqs, realtime=False)
    assert stats["requests"] == len(reqs)
    assert stats["failed_requests"] == 0
    assert stats["max_concurrent_requests"] > 1
    assert stats["peak_budget_bytes"] <= budget
    for r in reqs:
        with serving.Server(models, hbm_budget_bytes=budget, max_active=1, chunk=64) as srv1:
            alone, _ = srv1.run([r], realtime=False)
        a, m = alone[r.rid], mix[r.rid]
        for k in ("phi", "logq", "S", "logw", "chain_idx", "accepted", "mh_state"):
            assert torch.equal(getattr(a, k), getattr(m, k)), (r.rid, k)
    # an FP32 request against the oracle, a tensor-core 2D request against its emulation
    assert models["c"].flow.precision == "bf16" and models["a"].flow.precision == "fp32"
    for r in (reqs[0], reqs[2]):
        shape, s = specs[r.model]
        w = gi.init_weights(shape, seed=s)
        if r.model == "c":
            rtol, lw_rtol = tc_tolerances(shape.n_layers)
            ref = orc.flow_sample(shape, w, r.m2, r.lam, r.batch, seed=r.seed, counter0=0, bf16_mask=TC_MODE)
        else:
            rtol, lw_rtol = SITE_RTOL, LOGW_RTOL
            ref = orc.flow_sample(shape, w, r.m2, r.lam, r.batch, seed=r.seed, counter0=0)
        assert_sites_close(mix[r.rid].phi.cpu().numpy(), ref["phi"], rtol=rtol)
        assert_logw_close(mix[r.rid].logw.cpu().numpy(), ref["logw"], rtol=lw_rtol)
    assert P.device_status() == 0


def test_realtime_poisson_loop_reports_latency():
    torch, P = require_gpu()
    from paper_2208_08903_gb300 import serving
    models, _ = _models(P)
    arr = serving.poisson_arrivals(40, 400.0, seed=1)
    rng = np.random.default_rng(1)
    names = list(models)
    reqs = [serving.Request(i, names[int(rng.integers(4))], -4.0, 5.0, int(rng.integers(64, 512)), i,
                            arrival=float(arr[i])) for i in range(40)]
    with serving.Server(models, hbm_budget_bytes=64 << 20, max_active=8, chunk=256) as srv:
        res, stats = srv.run(reqs)
    assert stats["requests"] == 40 and stats["failed_requests"] == 0
    assert 0 < stats["p50_latency_ms"] <= stats["p99_latency_ms"]
    assert all(r.done >= r.arrival for r in res.values())


def test_requests_kernels_overlap_on_the_device():
    """Chunks of different requests run at the same time: with small FP32
    flows (grids smaller than the GPU) and every request admitted at once, the
    per-chunk CUDA event timeline shows two or more requests in flight."""
    torch, P = require_gpu()
    from paper_2208_08903_gb300 import serving
    specs = [("p", gi.FlowShape(2, 8, 6, 8, 8), 1), ("q", gi.FlowShape(2, 16, 4, 16, 16), 2)]
    models = {n: serving.Model(n, sh, P.Flow(sh, gi.init_weights(sh, seed=s))) for n, sh, s in specs}
    # chunks long enough (256 configurations) that the host loop keeps several in flight
    reqs = [serving.Request(i, "pq"[i % 2], -4.0, 5.0, 1024, 70 + i, arrival=0.0) for i in range(12)]
    with serving.Server(models, hbm_budget_bytes=256 << 20, max_active=6, chunk=256) as srv:
        srv.run(reqs[:2], realtime=False)                   # warm-up
        res, stats = srv.run(reqs, realtime=False, timeline=True)
    print({k: stats[k] for k in ("gpu_busy_ms", "overlapped_fraction", "max_requests_in_flight")})
    assert stats["failed_requests"] == 0
    assert stats["max_requests_in_flight"] >= 2
    assert stats["overlapped_fraction"] > 0.1

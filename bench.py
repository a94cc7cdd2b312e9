"""Benchmark of the flow sampler's hot path on GB300.

One step = one batch through the whole path: prior -> coupling stack ->
log q, phi^4 action, log w (one fused kernel) -> Metropolis-Hastings chain
over the batch's proposals (continuing one chain across steps).

Default workload: 3D phi^4, L=16 (4096 sites), m2=-6, lam=5, RealNVP with 16
checkerboard coupling layers, s/t nets conv3x3x3 1->32->32->2, batch 4096,
random-init weights (seed 0), synthetic Philox prior; metric = flow
configurations per second through sample + log q + S + MH.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the same workload instead (bounded samples per step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gf_inputs as gi  # noqa: E402

L2_BYTES = 129 * 1024 * 1024
METRIC = "flow configs/sec (sample+logq+S+MH)"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def flops_per_config(shape) -> float:
    """Algorithmic forward FLOPs of one configuration: conv1 on the taps that
    can be non-zero (fixed-site neighbours), conv2 dense, conv3 at the updated
    sites only."""
    V, T, C1, C2 = shape.V, shape.taps, shape.c1, shape.c2
    nz = 13.5 if shape.nd == 3 else 4.5
    per_layer = 2 * V * C1 * nz + 2 * V * C1 * C2 * T + 2 * (V / 2) * 2 * C2 * T
    return per_layer * shape.n_layers


def measured_traffic(kernel: str, batch: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/roofline_traffic.json), or None when the kernel's source changed
    since the counters were taken or the capture was at another batch size."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            ent = json.load(f)[kernel]
        src = os.path.join(ROOT, "paper_2208_08903_gb300", "csrc", ent["source"])
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if sha != ent["source_sha256"] or int(ent["batch"]) != int(batch):
            return None
        return float(ent["dram_bytes_read"]) + float(ent["dram_bytes_write"])
    except Exception:
        return None


def measured_counter(kernel: str, name: str):
    """Another counter of the committed ncu summary of `kernel` (same source
    check as measured_traffic, any batch), or None."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            ent = json.load(f)[kernel]
        src = os.path.join(ROOT, "paper_2208_08903_gb300", "csrc", ent["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest() != ent["source_sha256"]:
            return None
        return float(ent[name])
    except Exception:
        return None


def fp32_alu_peak_tflops(n_sm: int, mhz: float) -> float:
    # 128 FP32 FMA lanes per SM, 2 FLOP per FMA
    return n_sm * 128 * 2 * mhz * 1e6 / 1e12


_ALU_PEAK = {}


def alu_peak(n_sm: int, mhz: float, fp64: bool = False):
    """(TFLOP/s, description): the FP32 (FP64) multiply-add rate measured on
    this device by the library's probe, taken once per process; the derived
    lane-count figure when the probe fails.  FP32: the larger of the scalar
    FFMA and the packed FP32x2 FMA rates (the same FP32 pipe; scalar FFMA
    streams issue at about 86 % of it, the packed form reaches it)."""
    if fp64 not in _ALU_PEAK:
        try:
            import paper_2208_08903_gb300 as P
            if fp64:
                v = max(P.api.alu_peak(fp64=True, iters=1 << 14) for _ in range(3)) / 1e12
                kind = "DFMA measured by gf_alu_peak (best of 3 launches)"
            else:
                v = max(max(P.api.alu_peak(iters=1 << 17), P.api.alu_peak(packed=True, iters=1 << 17))
                        for _ in range(3)) / 1e12
                kind = "FP32 FMA pipe measured by gf_alu_peak (best of 3 launches of FFMA and packed FFMA2)"
            _ALU_PEAK[fp64] = (v, kind)
        except Exception as e:  # noqa: BLE001
            if fp64:
                _ALU_PEAK[fp64] = (None, f"probe failed: {e}")
            else:
                _ALU_PEAK[fp64] = (fp32_alu_peak_tflops(n_sm, mhz),
                                   f"FP32 FFMA: {n_sm} SM x 128 lanes x 2 FLOP x {mhz:.0f} MHz (derived; probe "
                                   f"failed: {e})")
    return _ALU_PEAK[fp64]


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_setup(want: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if _cuda_ok() else "gloo")
    return rank, world, local


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def counter_base(rank: int) -> int:
    """Disjoint prior counters per rank (2^40 configurations each)."""
    return rank << 40


def max_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if _cuda_ok() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------- training-step arm
def bench_train(args, rank, world, local):
    """One step = one reverse-KL training step (forward with saved layer inputs,
    hand-written backward, Adam) on 2D L=32, 24 couplings, hidden 32, batch 1024."""
    import torch
    import paper_2208_08903_gb300 as P

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = gi.WORKLOADS["c2"]
    shape, phi4, B = W["shape"], W["phi4"], args.batch or W["batch"]
    flow = P.Flow(shape, gi.init_weights(shape, seed=0))
    m = torch.zeros(flow.n_params, device=dev)
    v = torch.zeros(flow.n_params, device=dev)
    ws = torch.empty(flow.train_workspace_bytes(B), device=dev, dtype=torch.uint8)
    loss = None
    c0 = counter_base(rank)

    def step(i):
        nonlocal loss
        loss, _ = flow.train_step(B, phi4, seed=12345, counter0=c0 + i * B, lr=1e-3, adam_m=m, adam_v=v,
                                  adam_t=i + 1, workspace=ws, grad=False)

    flush = torch.empty(2 * L2_BYTES // 4, device=dev, dtype=torch.float32)
    barrier(world)
    clocks = ClockSampler(local)
    t = _time_steps(step, args.steps, args.warmup, flush)
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(t), world)
    # end to end: z from pinned host memory, loss back to the host, every step
    z_host = torch.from_numpy(gi.random_field(2, shape.L, B, seed=5).astype(np.float32)).pin_memory()
    z_dev = torch.empty(B, shape.V, device=dev)
    loss_host = torch.empty(1, dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()
    e2e = []
    for i in range(max(3, min(args.steps, 10)) + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        z_dev.copy_(z_host, non_blocking=True)
        lo, _ = flow.train_step(B, phi4, z=z_dev, lr=1e-3, adam_m=m, adam_v=v, adam_t=args.warmup + args.steps + i + 1,
                                workspace=ws, grad=False)
        loss_host.copy_(lo, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        if i > 0:
            e2e.append(a.elapsed_time(b))
    e2e_total = max_over_ranks(sum(e2e), world)
    fl = 4 * flops_per_config(shape) * B
    pk, pk_kind = peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak, peak_kind = alu_peak(n_sm, pk.get("sm_max_mhz", 2070.0))
    ach = fl / (float(np.mean(t)) / 1e3) / 1e12
    return {"metric": "train steps/s (reverse-KL step: forward + backward + Adam)",
            "value": world * args.steps / (total_ms / 1e3), "unit": "steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Philox prior, random-init weights seed 0)",
            "config": {"workload": "c2: 2D L=32 m2=-4 lam=8, 24 couplings, hidden 32, batch 1024, Adam lr 1e-3",
                       "batch": B, "l2": "flushed between timed steps"},
            "e2e": {"value": world * len(e2e) / (e2e_total / 1e3), "unit": "steps/s",
                    "h2d_bytes_per_step": B * shape.V * 4, "d2h_bytes_per_step": 8},
            # per step: prior + reverse-pass weight packing, 3 per layer forward, loss + mean,
            # 13 per layer backward, Adam + repack
            "gpu_launches": args.steps * (16 * shape.n_layers + 6),
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "traffic": None, "peak_kind": peak_kind,
                         "peak_derived": fp32_alu_peak_tflops(n_sm, pk.get("sm_max_mhz", 2070.0)),
                         "note": "algorithmic FLOP = 4 x forward (forward, recompute, "
                                 "data and weight gradients)"},
            "clocks": clk, "loss": float(loss.item())}


# --------------------------------------------------------------------------- GPU arm
def bench_gpu(args, rank, world, local):
    import torch
    import paper_2208_08903_gb300 as P

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = gi.WORKLOADS[args.workload]
    shape, phi4, B = W["shape"], W["phi4"], args.batch or W["batch"]
    prec = args.precision
    if prec == "auto":
        prec = "bf16" if P.tensor_core_supported(shape) else "fp32"
    flow = P.Flow(shape, gi.init_weights(shape, seed=0), precision=prec)
    V = shape.V
    out = P.SampleResult(phi=torch.empty(B, V, device=dev),
                         logq=torch.empty(B, device=dev, dtype=torch.float64),
                         S=torch.empty(B, device=dev, dtype=torch.float64),
                         logw=torch.empty(B, device=dev, dtype=torch.float64))
    state = P.new_mh_state(seed=12345, stream_id=rank, device=dev)
    idx = torch.empty(B, device=dev, dtype=torch.int64)
    acc = torch.empty(B, device=dev, dtype=torch.uint8)
    ws = torch.empty(max(P.mh_chain_workspace_bytes(B) // 8, 1), device=dev, dtype=torch.float64)
    flush = torch.empty(2 * L2_BYTES // 4, device=dev, dtype=torch.float32)
    stream = torch.cuda.current_stream()
    seed = 2024
    c0 = counter_base(rank)

    def step(i, z=None):
        flow.sample(B, seed=seed, counter0=c0 + i * B, phi4=phi4, z=z, out=out)
        P.mh_chain(state, out.logw, workspace=ws, chain_idx=idx, acc=acc)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    assert P.device_status() == 0

    # device-timed steps: inputs resident, L2 flushed between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    for i in range(args.steps):
        flush.fill_(float(i))
        e0, e1, e2 = ev[i]
        e0.record(stream)
        flow.sample(B, seed=seed, counter0=c0 + (args.warmup + i) * B, phi4=phi4, out=out)
        e1.record(stream)
        P.mh_chain(state, out.logw, workspace=ws, chain_idx=idx, acc=acc)
        e2.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    step_ms = [e0.elapsed_time(e2) for e0, e1, e2 in ev]
    flow_ms = [e0.elapsed_time(e1) for e0, e1, e2 in ev]
    total_ms = max_over_ranks(sum(step_ms), world)
    st = P.read_mh_state(state)

    # end-to-end through the public API with host buffers (pinned), copies timed
    z_host = torch.from_numpy(gi.random_field(shape.nd, shape.L, B, seed=99).astype(np.float32)).pin_memory()
    phi_host = torch.empty(B, V, dtype=torch.float32).pin_memory()
    small_host = torch.empty(4, B, dtype=torch.float64).pin_memory()
    idx_host = torch.empty(B, dtype=torch.int64).pin_memory()
    acc_host = torch.empty(B, dtype=torch.uint8).pin_memory()
    z_dev = torch.empty(B, V, device=dev)
    e2e_ms = []
    n_e2e = max(3, min(args.steps, 10))
    for i in range(n_e2e + 1):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        z_dev.copy_(z_host, non_blocking=True)
        step(10**6 + i, z=z_dev)
        phi_host.copy_(out.phi, non_blocking=True)
        small_host[0].copy_(out.logq, non_blocking=True)
        small_host[1].copy_(out.S, non_blocking=True)
        small_host[2].copy_(out.logw, non_blocking=True)
        idx_host.copy_(idx, non_blocking=True)
        acc_host.copy_(acc, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        if i > 0:                 # first iteration warms the pinned paths
            e2e_ms.append(a.elapsed_time(b))
    e2e_total = max_over_ranks(sum(e2e_ms), world)
    h2d = B * V * 4
    d2h = B * V * 4 + 3 * B * 8 + B * 8 + B

    pk, pk_kind = peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fpc = flops_per_config(shape)
    flow_avg_s = float(np.mean(flow_ms)) / 1e3
    achieved = fpc * B / flow_avg_s / 1e12
    if prec == "bf16":
        # Each flow launch is timed on its own (about 15 ms, one per step with an
        # L2 flush in between), so the burst peak is the denominator.
        peak = pk.get("bf16_tflops", 1900.0)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_kind": f"bf16 dense burst, {pk_kind} (each launch is timed alone)",
                "frac_of_sustained": achieved / pk.get("bf16_tflops_sustained", 1700.0)}
    else:
        mhz = pk.get("sm_max_mhz", 2070.0)
        peak, peak_kind = alu_peak(n_sm, mhz)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                "peak_derived": fp32_alu_peak_tflops(n_sm, mhz)}
    roof["kernel"] = "flow_fp32_kernel" if prec == "fp32" else "flow_bf16_kernel"
    roof["traffic"] = measured_traffic(roof["kernel"], B)
    pipe = measured_counter(roof["kernel"], "tensor_pipe_active_pct")
    if pipe is not None:
        roof["ncu_tensor_pipe_active_pct"] = pipe
    roof["flops_per_config"] = fpc
    value = world * B * args.steps / (total_ms / 1e3)
    res = {
        "metric": METRIC, "value": value, "unit": "configs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == "fp32" else "bf16",
        "data": "synthetic (seeded Philox prior, Kaiming-uniform random-init weights seed 0)",
        "config": {"workload": f"{args.workload}: {shape.nd}D phi^4 L={shape.L} m2={phi4.m2} lam={phi4.lam}, "
                               f"RealNVP {shape.n_layers} couplings, conv 1->{shape.c1}->{shape.c2}->2, "
                               f"batch {B}, MH chain over the batch",
                   "batch": B, "nd": shape.nd, "L": shape.L, "n_layers": shape.n_layers,
                   "hidden": [shape.c1, shape.c2], "precision": prec,
                   "l2": "flushed between timed steps (2x L2 buffer write)",
                   "parallelism": f"dp{world} (independent batches, one MH chain per rank)"},
        "e2e": {"value": world * B * n_e2e / (e2e_total / 1e3), "unit": "configs/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 3 * args.steps,
        "roofline": roof,
        "clocks": clk,
        "mh": {"steps": int(st.step), "accepted": int(st.n_acc),
               "acceptance": st.n_acc / max(1, st.step - 1)},
        "flow_kernel_ms": float(np.mean(flow_ms)),
    }
    del flush
    if world == 1 and not args.no_extra:
        flush2 = torch.empty(2 * L2_BYTES // 4, device=dev, dtype=torch.float32)
        res["extra"] = bench_extra(args, dev, flush2, pk)
        if "plain_fp32_unfused" in res["extra"]:
            pl = res["extra"]["plain_fp32_unfused"]["configs_per_s"]
            res["extra"]["speedup_vs_plain_fp32"] = value / pl
    return res


# --------------------------------------------------------------------------- secondary measurements
def _time_steps(fn, steps, warmup, flush=None):
    """Per-step CUDA-event times (ms) on the current stream, L2 flushed between steps."""
    import torch
    stream = torch.cuda.current_stream()
    for i in range(warmup):
        fn(i)
    torch.cuda.synchronize()
    ts = []
    for i in range(steps):
        if flush is not None:
            flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn(warmup + i)
        b.record(stream)
        ts.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ts]


def bench_extra(args, dev, flush, pk):
    """Secondary lines: plain FP32 arm, training step, HMC, action GB/s, MH, c1."""
    import torch
    import paper_2208_08903_gb300 as P
    out = {}
    W = gi.WORKLOADS[args.workload]
    shape, phi4, B = W["shape"], W["phi4"], args.batch or W["batch"]
    w = gi.init_weights(shape, seed=0)
    V = shape.V
    only = [x for x in (args.only_extra or "").split(",") if x]

    def want(name):
        return not only or name in only

    def sampling_rate(kind, steps=3):
        flow = P.Flow(shape, w, precision="fp32")
        res = P.SampleResult(phi=torch.empty(B, V, device=dev),
                             logq=torch.empty(B, device=dev, dtype=torch.float64),
                             S=torch.empty(B, device=dev, dtype=torch.float64),
                             logw=torch.empty(B, device=dev, dtype=torch.float64))
        st = P.new_mh_state(seed=12345, device=dev)
        ws = torch.empty(flow.unfused_workspace_bytes(B), device=dev, dtype=torch.uint8) if kind == "unfused" else None

        def step(i):
            if kind == "unfused":
                flow.sample_unfused(B, seed=2024, counter0=i * B, phi4=phi4, out=res, workspace=ws)
            else:
                flow.sample(B, seed=2024, counter0=i * B, phi4=phi4, out=res)
            P.mh_chain(st, res.logw)
        t = _time_steps(step, steps, 1, flush)
        s = P.read_mh_state(st)
        del ws
        return {"configs_per_s": B * len(t) / (sum(t) / 1e3), "ms_per_step": float(np.mean(t)),
                "acceptance": s.n_acc / max(1, s.step - 1)}

    if want("sampling"):
        out["plain_fp32_unfused"] = sampling_rate("unfused")
        out["fused_fp32"] = sampling_rate("fused")
        torch.cuda.empty_cache()

    if want("trained"):
        # equal acceptance on the trained 3D flow shipped in checkpoints/: the
        # tensor-core, fused FP32 and plain FP32 samplers on the same proposals
        if args.workload == "c3":
            out["trained_c3_equal_acceptance"] = trained_acceptance(shape, phi4, n=args.acceptance_proposals)
            torch.cuda.empty_cache()

    if want("train"):
        # reverse-KL training step, 2D L=32, 24 couplings, hidden 32, batch 1024, Adam
        W2 = gi.WORKLOADS["c2"]
        f2 = P.Flow(W2["shape"], gi.init_weights(W2["shape"]))
        m = torch.zeros(f2.n_params, device=dev)
        v = torch.zeros(f2.n_params, device=dev)
        ws2 = torch.empty(f2.train_workspace_bytes(W2["batch"]), device=dev, dtype=torch.uint8)
        t = _time_steps(lambda i: f2.train_step(W2["batch"], W2["phi4"], seed=12345, counter0=i * W2["batch"],
                                                lr=1e-3, adam_m=m, adam_v=v, adam_t=i + 1, workspace=ws2,
                                                grad=False), 3, 2, flush)
        fl = 4 * flops_per_config(W2["shape"]) * W2["batch"]
        out["train_c2"] = {"steps_per_s": 1e3 / float(np.mean(t)), "ms_per_step": float(np.mean(t)),
                           "approx_tflops": fl / (float(np.mean(t)) / 1e3) / 1e12,
                           "workload": "2D L=32, 24 couplings, hidden 32, batch 1024, forward+backward+Adam"}
        del ws2, f2
        torch.cuda.empty_cache()

    if want("hmc"):
        # HMC, 3D L=16, 512 chains, 20 leapfrog steps, eps 0.05, FP64
        W4 = gi.WORKLOADS["c4"]
        phi = torch.zeros(W4["chains"], W4["L"] ** 3, device=dev, dtype=torch.float64)
        t = _time_steps(lambda i: P.hmc_trajectory(3, W4["L"], W4["phi4"], phi, W4["n_steps"], W4["eps"], 7, i),
                        20, 3, None)
        traj_ms = float(np.mean(t))
        # FP64 FLOP per site and leapfrog step: force 20 (three directions of
        # 2 phi - two neighbours, 2 x lap + 2 m2 phi + 4 lam phi^3), kick 2, drift 2
        hmc_fl = 24.0 * W4["chains"] * W4["L"] ** 3 * W4["n_steps"]
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        dfma, dfma_kind = alu_peak(n_sm, pk.get("sm_max_mhz", 2070.0), fp64=True)
        ffma, ffma_kind = alu_peak(n_sm, pk.get("sm_max_mhz", 2070.0), fp64=False)
        hmc_tf = hmc_fl / (traj_ms / 1e3) / 1e12
        out["hmc_c4"] = {"trajectories_per_s": 1e3 / traj_ms, "ms_per_trajectory_all_chains": traj_ms,
                         "chain_trajectories_per_s": W4["chains"] * 1e3 / traj_ms,
                         "seconds_for_1000_trajectories": traj_ms,
                         "fp64_tflops": hmc_tf, "dfma_peak_tflops": dfma,
                         "frac_of_dfma": hmc_tf / dfma if dfma else None, "peak_kind": dfma_kind,
                         "flop_per_site_step": 24,
                         "workload": "3D L=16, 512 chains, 20 steps, eps=0.05, FP64"}
        try:
            f2 = max(P.api.alu_peak(packed=True, iters=1 << 17) for _ in range(3)) / 1e12
        except Exception:  # noqa: BLE001
            f2 = None
        out["alu_peaks_measured"] = {"ffma_tflops": ffma, "dfma_tflops": dfma, "ffma2_packed_tflops": f2,
                                     "ffma_kind": ffma_kind,
                                     "dfma_kind": dfma_kind,
                                     "ffma_derived_tflops": fp32_alu_peak_tflops(n_sm, pk.get("sm_max_mhz", 2070.0))}

    if want("action"):
        # standalone action of FP32 fields: fields larger than L2 (4 x the batch,
        # 268 MB) read in turn without a flush, as for the observables below
        Ba = 4 * B
        phi32 = torch.randn(Ba, V, device=dev)
        S = torch.empty(Ba, device=dev, dtype=torch.float64)
        t = _time_steps(lambda i: P.phi4_action(shape.nd, shape.L, phi4, phi32, out=S), 10, 3, None)
        gbs = (Ba * V * 4 + Ba * 8) / (float(np.mean(t)) / 1e3) / 1e9
        out["action_fp32"] = {"GB_per_s": gbs, "frac_of_hbm": gbs / pk.get("hbm_gbs", 6800.0),
                              "bytes_per_launch": Ba * V * 4 + Ba * 8, "ms": float(np.mean(t)),
                              "workload": f"{Ba} configurations of {shape.nd}D L={shape.L}",
                              "l2": "inputs 4x L2 size, read in turn, no flush"}
        del phi32

    if want("observables"):
        # chain observables: M and C(t) per configuration (HBM-bound read of the
        # fields), then the autocorrelation / tau_int of a 100k-step series and the ESS.
        # The fields here are larger than L2 (4 x the batch, 268 MB) and are read in
        # turn without a flush: a flush that writes L2 full leaves dirty lines whose
        # write-back would double the traffic of this read-only kernel.
        lib = P._abi.load()
        stream = torch.cuda.current_stream().cuda_stream
        Bo = 4 * B
        phi_o = torch.randn(Bo, V, device=dev)
        M = torch.empty(Bo, device=dev, dtype=torch.float64)
        Cc = torch.empty(Bo, shape.L, device=dev, dtype=torch.float64)

        def obs(i):
            P._abi.check("gf_observables", lib.gf_observables(shape.nd, shape.L, Bo, phi_o.data_ptr(), M.data_ptr(),
                                                              Cc.data_ptr(), stream))
        t = _time_steps(obs, 10, 3, None)
        ob_bytes = Bo * V * 4 + Bo * (shape.L + 1) * 8
        gbs = ob_bytes / (float(np.mean(t)) / 1e3) / 1e9
        out["observables"] = {"GB_per_s": gbs, "frac_of_hbm": gbs / pk.get("hbm_gbs", 6800.0),
                              "bytes_per_launch": ob_bytes, "ms": float(np.mean(t)),
                              "workload": f"M and C(t) of {Bo} configurations of {shape.nd}D L={shape.L}",
                              "l2": "inputs 4x L2 size, read in turn, no flush"}
        del phi_o
        y = torch.randn(100000, device=dev, dtype=torch.float64)
        t = _time_steps(lambda i: P.autocorr(y, 1000), 5, 2, None)
        out["autocorr"] = {"ms": float(np.mean(t)), "n": 100000, "t_max": 1000}
        t = _time_steps(lambda i: P.ess(y), 5, 2, None)
        out["ess"] = {"ms": float(np.mean(t)), "n": 100000}

    if want("eager"):
        # context: the same flow in eager PyTorch (cuDNN FP32 convolutions, TF32 off)
        out["torch_eager_fp32_context"] = torch_eager_rate(shape, phi4, w, min(B, 1024), dev, flush)
        torch.cuda.empty_cache()

    if want("mh"):
        # MH chain alone, 100k proposals
        n = 100000
        lw = torch.randn(n, device=dev, dtype=torch.float64) * 2 - 50
        st = P.new_mh_state(seed=1, device=dev)
        wsm = torch.empty(n, device=dev, dtype=torch.float64)
        t = _time_steps(lambda i: P.mh_chain(st, lw, workspace=wsm), 5, 2, None)
        out["mh_chain"] = {"ns_per_proposal": float(np.mean(t)) * 1e6 / n, "proposals": n}

    if want("serving"):
        # serving mix: resident random-init models; capacity, then a Poisson load sweep
        out["serving_c5"] = bench_serving(dev, n_requests=args.serving_requests)
        torch.cuda.empty_cache()

    if want("tc"):
        out["tensor_core_other_shapes"] = bench_tc_shapes(dev, flush, pk)
        torch.cuda.empty_cache()

    if want("c1"):
        # the paper's example workload (2D L=8, 16 couplings, hidden 8, batch 64)
        W1 = gi.WORKLOADS["c1"]
        f1 = P.Flow(W1["shape"], gi.init_weights(W1["shape"]))
        r1 = P.SampleResult(phi=torch.empty(64, 64, device=dev), logq=torch.empty(64, device=dev, dtype=torch.float64),
                            S=torch.empty(64, device=dev, dtype=torch.float64),
                            logw=torch.empty(64, device=dev, dtype=torch.float64))
        st1 = P.new_mh_state(seed=2, device=dev)

        def c1step(i):
            f1.sample(64, seed=3, counter0=64 * i, phi4=W1["phi4"], out=r1)
            P.mh_chain(st1, r1.logw)
        t = _time_steps(c1step, 50, 5, None)
        out["c1_sampling"] = {"configs_per_s": 64 / (float(np.mean(t)) / 1e3), "ms_per_step": float(np.mean(t))}
        # batch sweep of the c1 flow (fused FP32 sampler + MH): 64 configurations cannot fill 152 SMs
        sweep = {}
        for Bs in (64, 1024, 16384, 65536):
            rs = P.SampleResult(phi=torch.empty(Bs, 64, device=dev), logq=torch.empty(Bs, device=dev, dtype=torch.float64),
                                S=torch.empty(Bs, device=dev, dtype=torch.float64),
                                logw=torch.empty(Bs, device=dev, dtype=torch.float64))
            sts = P.new_mh_state(seed=3, device=dev)

            def sstep(i, Bs=Bs, rs=rs, sts=sts):
                f1.sample(Bs, seed=4, counter0=Bs * i, phi4=W1["phi4"], out=rs)
                P.mh_chain(sts, rs.logw)
            t = _time_steps(sstep, 10, 3, None)
            sweep[str(Bs)] = Bs / (float(np.mean(t)) / 1e3)
        out["c1_batch_sweep_configs_per_s"] = sweep
    return out


def bench_tc_shapes(dev, flush, pk):
    """The tensor-core kernel for the lattice shapes other than 3D L=16 C=32
    (gf_flow_tc.cu) next to the fused FP32 kernel on the same flows: per-launch
    CUDA-event time of gf_flow_sample (prior, coupling stack, log q, S, log w)
    with L2 flushed between launches, configs/s, algorithmic TFLOP/s and the
    fraction of the measured BF16 burst peak (each launch timed alone)."""
    import torch
    import paper_2208_08903_gb300 as P
    cases = [("2D L=32, 24 couplings, hidden 32", gi.FlowShape(2, 32, 24, 32, 32), 8192),
             ("2D L=64, 16 couplings, hidden 16", gi.FlowShape(2, 64, 16, 16, 16), 4096),
             ("2D L=16, 16 couplings, hidden 24", gi.FlowShape(2, 16, 16, 24, 24), 16384),
             ("3D L=8, 16 couplings, hidden 32", gi.FlowShape(3, 8, 16, 32, 32), 8192),
             ("3D L=12, 16 couplings, hidden 16", gi.FlowShape(3, 12, 16, 16, 16), 4096),
             ("2D L=32, 16 couplings, hidden 8", gi.FlowShape(2, 32, 16, 8, 8), 8192),
             ("3D L=16, 16 couplings, hidden 8", gi.FlowShape(3, 16, 16, 8, 8), 4096),
             ("3D L=8, 16 couplings, hidden 16", gi.FlowShape(3, 8, 16, 16, 16), 8192)]
    phi4 = (-4.0, 6.0)
    res = {"theory": "m2=-4, lam=6, random-init weights seed 0", "peak_tflops": pk["bf16_tflops"]}
    for name, shape, B in cases:
        w = gi.init_weights(shape, seed=0)
        line = {"batch": B, "flops_per_config": flops_per_config(shape)}
        for prec in ("bf16", "fp32"):
            flow = P.Flow(shape, w, precision=prec)
            r = P.SampleResult(phi=torch.empty(B, shape.V, device=dev),
                               logq=torch.empty(B, device=dev, dtype=torch.float64),
                               S=torch.empty(B, device=dev, dtype=torch.float64),
                               logw=torch.empty(B, device=dev, dtype=torch.float64))
            t = _time_steps(lambda i: flow.sample(B, seed=5, counter0=i * B, phi4=phi4, out=r),
                            5 if prec == "bf16" else 2, 2, flush)
            ms = float(np.mean(t))
            line[prec] = {"configs_per_s": B / (ms / 1e3), "ms_per_launch": ms,
                          "tflops": flops_per_config(shape) * B / (ms / 1e3) / 1e12}
            del flow, r
        line["bf16"]["frac_of_bf16_burst"] = line["bf16"]["tflops"] / pk["bf16_tflops"]
        line["speedup_vs_fused_fp32"] = line["bf16"]["configs_per_s"] / line["fp32"]["configs_per_s"]
        res[name] = line
    res["trained_2d_equal_acceptance"] = trained_2d_acceptance()
    assert P.device_status() == 0
    return res


def trained_2d_acceptance(n=65536):
    """Equal acceptance of the second tensor-core kernel: a 2D L=16 flow
    (12 couplings, hidden 16, m2=-4, lam=8) trained here with the reverse-KL
    step (3,000 Adam steps at batch 64, lr 1e-3, model seed 2021), then the
    tensor-core and fused FP32 samplers on the same n proposals (same prior
    counters and MH uniforms): acceptance with binomial errors, ESS, tau_int
    of |M|, decision agreement and each sampler's configs/s over the run."""
    import torch
    import paper_2208_08903_gb300 as P
    from paper_2208_08903_gb300 import train as T
    shape = gi.FlowShape(2, 16, 12, 16, 16)
    phi4 = (-4.0, 8.0)
    flow = P.Flow(shape, gi.init_weights(shape, seed=2021))
    t0 = time.perf_counter()
    st = T.train(flow, phi4, 30, 100, 64, lr=1e-3, seed=4242)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    tc = P.Flow(shape, flow.get_weights().double().cpu().numpy(), precision="bf16")
    for f in (flow, tc):               # first launches outside the timed runs
        T.evaluate(f, phi4, 4096, 4096, seed=1, sampler="fused")
    ev = {k: T.evaluate(f, phi4, n, 4096, seed=909, sampler="fused", keep_logw=True)
          for k, f in (("fp32", flow), ("tensor_core", tc))}
    out = {"flow": "2D L=16, 12 couplings, hidden 16, m2=-4, lam=8; 3,000 reverse-KL Adam steps at batch 64 "
                   f"({train_s:.1f} s), final loss {st.losses[-1]:.3f}",
           "proposals": n}
    for k, e in ev.items():
        out[k] = {"acceptance": e["acceptance"], "acceptance_binomial_err": e["acceptance_binomial_err"],
                  "ess": e["ess"], "tau_int_abs_M": e["tau_int_abs_M"], "tau_int_err": e["tau_int_err"],
                  "configs_per_s_incl_mh_observables": n / e["seconds"]}
    se = float(np.hypot(ev["fp32"]["acceptance_binomial_err"], ev["tensor_core"]["acceptance_binomial_err"]))
    out["acceptance_difference_sigma"] = (ev["tensor_core"]["acceptance"] - ev["fp32"]["acceptance"]) / max(se, 1e-300)
    out["decisions_same"] = T.decision_agreement(ev["tensor_core"], ev["fp32"])
    return out


def trained_acceptance(shape, phi4, n=32768):
    """MH acceptance (binomial error), ESS, tau_int(|M|) and configs/s of the
    three samplers on the trained 3D flow, all on the same n proposals."""
    import paper_2208_08903_gb300 as P
    from paper_2208_08903_gb300 import train as T
    w = T.load_weights(os.path.join(T.CHECKPOINT_DIR, "c3_L16_16layers_15k.npz"), shape)
    f32 = P.Flow(shape, w)
    arms = {"tensor_core": (P.Flow(shape, w, precision="bf16"), "fused"), "fused_fp32": (f32, "fused"),
            "plain_fp32": (f32, "unfused")}
    for f, kind in arms.values():      # first launches (module loading, attributes) outside the timed runs
        T.evaluate(f, phi4, 4096, 4096, seed=1, sampler=kind)
    ev = {k: T.evaluate(f, phi4, n, 4096, seed=12347, sampler=kind, keep_logw=True) for k, (f, kind) in arms.items()}
    res = {"checkpoint": "checkpoints/c3_L16_16layers_15k.npz (15,000 reverse-KL Adam steps, batch 64)",
           "proposals": n}
    for k, e in ev.items():
        res[k] = {kk: e[kk] for kk in ("acceptance", "acceptance_binomial_err", "ess", "abs_M", "tau_int_abs_M",
                                       "tau_int_err")}
        res[k]["configs_per_s"] = n / e["seconds"]
    res["tensor_core"]["decisions_same_as_fp32"] = T.decision_agreement(ev["tensor_core"], ev["fused_fp32"])
    res["plain_fp32"]["decisions_same_as_fused"] = T.decision_agreement(ev["plain_fp32"], ev["fused_fp32"])
    d = res["tensor_core"]["acceptance"] - res["fused_fp32"]["acceptance"]
    se = math.hypot(res["tensor_core"]["acceptance_binomial_err"], res["fused_fp32"]["acceptance_binomial_err"])
    res["acceptance_difference_sigma"] = d / se if se > 0 else None
    res["speedup_tensor_core_vs_plain_fp32"] = res["tensor_core"]["configs_per_s"] / res["plain_fp32"]["configs_per_s"]
    res["speedup_tensor_core_vs_plain_fp32_per_independent_sample"] = (
        res["speedup_tensor_core_vs_plain_fp32"] * res["plain_fp32"]["tau_int_abs_M"] / res["tensor_core"]["tau_int_abs_M"])
    return res


def torch_eager_flow(shape, phi4, w, dev):
    """The flow (sampling direction, log q, S) written with eager torch ops:
    circular padding + cuDNN convolutions in FP32.  Returns run(z) -> (phi,
    log q, S).  A context baseline only; it shares nothing with the library."""
    import torch
    import torch.nn.functional as F
    nd, L, V = shape.nd, shape.L, shape.V
    conv = F.conv3d if nd == 3 else F.conv2d
    k = (3,) * nd
    layers = []
    for l in range(shape.n_layers):
        d = gi.split_layer(shape, w, l)
        t = lambda a, shp: torch.tensor(a, dtype=torch.float32, device=dev).reshape(shp)
        layers.append((t(d["W1"], (shape.c1, 1) + k), t(d["b1"], (-1,)), t(d["W2"], (shape.c2, shape.c1) + k),
                       t(d["b2"], (-1,)), t(d["W3"], (2, shape.c2) + k), t(d["b3"], (-1,))))
    coords = torch.stack(torch.meshgrid(*[torch.arange(L, device=dev)] * nd, indexing="ij"))
    par = (coords.sum(0) % 2).reshape((1, 1) + (L,) * nd)
    pad = (1, 1) * nd

    def run(z):
        x = z.reshape((z.shape[0], 1) + (L,) * nd)
        logdet = torch.zeros(z.shape[0], device=dev, dtype=torch.float64)
        for l, (W1, b1, W2, b2, W3, b3) in enumerate(layers):
            frozen = (par == (l & 1)).float()
            h = F.leaky_relu(conv(F.pad(x * frozen, pad, mode="circular"), W1, b1), shape.leaky_slope)
            h = F.leaky_relu(conv(F.pad(h, pad, mode="circular"), W2, b2), shape.leaky_slope)
            st = conv(F.pad(h, pad, mode="circular"), W3, b3)
            s = torch.tanh(st[:, :1]) if shape.use_final_tanh else st[:, :1]
            act = 1.0 - frozen
            x = x * frozen + act * (x * torch.exp(s) + st[:, 1:])
            logdet += (s * act).flatten(1).double().sum(1)
        phi = x.flatten(1)
        logr = -0.5 * (z.double() ** 2).sum(1) - 0.5 * V * math.log(2 * math.pi)
        hop = sum(torch.roll(x, -1, dims=2 + a) for a in range(nd)).flatten(1).double()
        pd = phi.double()
        S = ((2 * nd + phi4.m2) * pd * pd + phi4.lam * pd ** 4 - 2 * pd * hop).sum(1)
        return phi, logr - logdet, S
    return run


def torch_eager_rate(shape, phi4, w, B, dev, flush):
    """Configs/s of torch_eager_flow with TF32 disabled (context figure)."""
    import torch
    torch.backends.cudnn.allow_tf32 = False
    torch.backends.cuda.matmul.allow_tf32 = False
    run = torch_eager_flow(shape, phi4, w, dev)
    gen = torch.Generator(device=dev).manual_seed(1)
    z = torch.randn(B, shape.V, device=dev, generator=gen)
    t = _time_steps(lambda i: run(z), 3, 1, flush)
    return {"configs_per_s": B / (float(np.mean(t)) / 1e3), "batch": B, "ms_per_step": float(np.mean(t)),
            "note": "eager torch, cuDNN FP32 (TF32 off), no MH; context only"}


def bench_serving(dev, n_requests=120, rate=200.0, n_models=16, seed=5):
    """Continuous-batching loop on the serving mix: the capacity (every
    request admitted at t=0), then p50/p99 latency, throughput and the overlap
    of requests' kernels at Poisson loads of 25 %, 50 %, 75 % and 90 % of that
    capacity and at the mix's nominal 200 req/s."""
    import torch
    import paper_2208_08903_gb300 as P
    from paper_2208_08903_gb300 import serving
    specs = gi.serving_models(n_models, seed)
    models = {}
    for name, shape, s in specs:
        prec = "bf16" if P.tensor_core_supported(shape) else "fp32"
        models[name] = serving.Model(name, shape, P.Flow(shape, gi.init_weights(shape, seed=s), precision=prec))
    mix = gi.serving_requests(n_requests, list(models), seed)

    def requests(rate_req_s):
        arr = serving.poisson_arrivals(n_requests, rate_req_s, seed) if rate_req_s else np.zeros(n_requests)
        return [serving.Request(i, name, m2, lam, b, sd, arrival=float(arr[i]))
                for i, (name, m2, lam, b, sd) in enumerate(mix)]

    out = {"mix": "2D L in {8,16,32,64}, 3D L in {8,12,16}, 12-24 couplings, hidden {8,16,24,32}, "
                  "batch 64-8192 log-uniform; tensor-core kernels where gf_flow_tensor_core_supported "
                  "(activations that fit a block), FP32 kernels otherwise",
           "precision_by_model": {name: ("bf16" if P.tensor_core_supported(shape) else "fp32")
                                  for name, shape, _ in specs},
           "models": n_models, "requests_per_load": n_requests,
           "mean_configs_per_request": float(np.mean([m[3] for m in mix]))}
    with serving.Server(models, hbm_budget_bytes=16 << 30, max_active=16, chunk=2048, device=dev) as srv:
        srv.run(requests(0)[:4], keep_results=False, realtime=False)      # warm-up
        _, cap = srv.run(requests(0), keep_results=False, realtime=False, timeline=True)
        cap_req_s = n_requests / cap["wall_s"]
        out["capacity"] = {"configs_per_s": cap["configs_per_s"], "requests_per_s": cap_req_s,
                           "overlapped_fraction": cap.get("overlapped_fraction"),
                           "max_requests_in_flight": cap.get("max_requests_in_flight")}
        loads = []
        for frac in (0.25, 0.5, 0.75, 0.9, None):
            r = rate if frac is None else frac * cap_req_s
            _, st = srv.run(requests(r), keep_results=False, realtime=True, timeline=True)
            loads.append({"offered_req_per_s": r, "fraction_of_capacity": r / cap_req_s,
                          "p50_latency_ms": st["p50_latency_ms"], "p99_latency_ms": st["p99_latency_ms"],
                          "configs_per_s": st["configs_per_s"], "failed_requests": st["failed_requests"],
                          "overlapped_fraction": st.get("overlapped_fraction"),
                          "max_requests_in_flight": st.get("max_requests_in_flight")})
        out["loads"] = loads
    return out


# --------------------------------------------------------------------------- CPU oracle
def oracle_rate(shape, phi4, n_cfg, seed=2024, counter0=0, nthreads=None):
    import oracle
    nthr = nthreads or oracle.default_threads()
    w = gi.init_weights(shape, seed=0)
    t0 = time.perf_counter()
    out = oracle.flow_sample(shape, w, phi4.m2, phi4.lam, n_cfg, seed=seed, counter0=counter0,
                             nthreads=nthr)
    st = oracle.new_mh_state(12345)
    oracle.mh_chain(st, out["logw"])
    dt = time.perf_counter() - t0
    return n_cfg / dt, dt, nthr


def cpu_sample_size(shape, phi4, target_s):
    r, dt, nthr = oracle_rate(shape, phi4, 1)
    per_cfg_serial = dt
    n = max(1, int(target_s * nthr / max(per_cfg_serial, 1e-6)))
    return min(n, 4096), nthr


def bench_cpu_baseline(args):
    W = gi.WORKLOADS[args.workload]
    shape, phi4 = W["shape"], W["phi4"]
    n, nthr = cpu_sample_size(shape, phi4, target_s=args.cpu_seconds)
    rate, dt, nthr = oracle_rate(shape, phi4, n, counter0=7)
    n1 = max(1, n // max(nthr, 1))
    rate1, dt1, _ = oracle_rate(shape, phi4, n1, counter0=7, nthreads=1)
    return {"value": rate, "unit": "configs/s", "cores": nthr, "kind": "oracle",
            "single_thread_value": rate1,
            "sample": f"{n} configurations of the same workload (FP64 C oracle, OpenMP over "
                      f"configurations) + MH over them, {dt:.1f} s; single thread: {n1} "
                      f"configurations, {dt1:.1f} s"}


def bench_reference(args, rank, world):
    if rank != 0:
        return None
    W = gi.WORKLOADS[args.workload]
    shape, phi4 = W["shape"], W["phi4"]
    budget = max(20.0, min(150.0, args.ref_seconds))
    per_step = budget / (args.steps + args.warmup)
    n, nthr = cpu_sample_size(shape, phi4, target_s=per_step)
    times = []
    for i in range(args.warmup + args.steps):
        r, dt, _ = oracle_rate(shape, phi4, n, counter0=1000 + i * n)
        if i >= args.warmup:
            times.append(dt)
    value = n * args.steps / sum(times)
    sample = f"{n} configurations per step (FP64 C oracle on {nthr} host threads) + MH over them"
    return {"metric": METRIC, "value": value, "unit": "configs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{args.workload}: {shape.nd}D phi^4 L={shape.L} m2={phi4.m2} "
                                   f"lam={phi4.lam}, RealNVP {shape.n_layers} couplings, conv "
                                   f"1->{shape.c1}->{shape.c2}->2, MH chain over the batch",
                       "batch_per_step": n, "nd": shape.nd, "L": shape.L, "n_layers": shape.n_layers,
                       "hidden": [shape.c1, shape.c2], "precision": "f64",
                       "parallelism": "rank 0 host cores (OpenMP over configurations)"},
            "cpu_baseline": {"value": value, "unit": "configs/s", "cores": nthr, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "configs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gfflow", choices=["gfflow", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16"])
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=120.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary measurements")
    ap.add_argument("--only-extra", default="",
                    help="comma list of secondary measurements to run (sampling, trained, train, hmc, action, "
                         "observables, eager, mh, serving, tc, c1); default all")
    ap.add_argument("--serving-requests", type=int, default=60)
    ap.add_argument("--acceptance-proposals", type=int, default=32768)
    args = ap.parse_args()
    if args.impl == "reference":
        # The oracle runs on the host cores of rank 0 only: no process group, no GPU.
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
        res = bench_reference(args, rank, world)
        if rank == 0:
            print(json.dumps(res), flush=True)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = dist_setup(args.gpus)
    if args.workload == "c2":
        res = bench_train(args, rank, world, local)
        if rank == 0:
            print(json.dumps(res), flush=True)
        return
    res = bench_gpu(args, rank, world, local)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            res["cpu_baseline"] = bench_cpu_baseline(args)
        else:
            res["cpu_baseline"] = None
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

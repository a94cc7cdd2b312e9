"""Continuous-batching request loop for flow sampling (host scheduler).

Requests ask for `batch` configurations from one of the resident flow models,
with their own (m2, lam), seed and Metropolis-Hastings chain.  The loop:

  * admits waiting requests in arrival order while the HBM budget (outputs,
    chain state and workspace of all admitted requests) and the number of
    request slots allow;
  * splits each admitted request into chunks of at most `chunk` proposals and
    keeps one chunk per request in flight on the request's own CUDA stream:
    gf_flow_sample for the chunk, then gf_mh_chain over its log weights, so a
    request's chain consumes its proposals in order while chunks of different
    requests overlap on the GPU;
  * retires a request when its last chunk's event completes, frees its slot
    and budget, and records its latency (completion - arrival);
  * attributes device-detected errors (a bounded wait of a kernel that ran
    out) to the request that caused them: each stream has its own status slot
    (gf_set_stream_status_slot), read and cleared when a request on it
    retires; a request whose slot is non-zero is reported failed (Result.error)
    and its outputs must not be used.

Results do not depend on what else is running: every random number is keyed
by the request's seed and the configuration's index inside the request, and
every kernel is deterministic.  Flow weights and chain state stay on the
device for the whole run.
"""
from __future__ import annotations

import dataclasses
import heapq
import time

import numpy as np
import torch

from . import api


@dataclasses.dataclass
class Model:
    """A flow resident on the device (weights uploaded once)."""
    name: str
    shape: object
    flow: api.Flow

    @property
    def V(self) -> int:
        return self.shape.L ** self.shape.nd


@dataclasses.dataclass
class Request:
    rid: int
    model: str
    m2: float
    lam: float
    batch: int
    seed: int
    arrival: float = 0.0        # seconds on the loop's clock


@dataclasses.dataclass
class Result:
    rid: int
    phi: torch.Tensor
    logq: torch.Tensor
    S: torch.Tensor
    logw: torch.Tensor
    chain_idx: torch.Tensor
    accepted: torch.Tensor
    mh_state: torch.Tensor
    arrival: float
    admitted: float
    done: float
    error: int = 0              # 0, or the gf_status a kernel of this request recorded

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class _Active:
    def __init__(self, req: Request, model: Model, device, stream, chunk: int, keep: bool):
        B, V = req.batch, model.V
        self.req, self.model, self.stream = req, model, stream
        self.chunk = chunk
        self.next = 0
        self.event = None
        with torch.cuda.stream(stream):
            self.phi = torch.empty(B, V, device=device)
            self.logq = torch.empty(B, device=device, dtype=torch.float64)
            self.S = torch.empty(B, device=device, dtype=torch.float64)
            self.logw = torch.empty(B, device=device, dtype=torch.float64)
            self.idx = torch.empty(B, device=device, dtype=torch.int64)
            self.acc = torch.empty(B, device=device, dtype=torch.uint8)
            self.ws = torch.empty(max(api.mh_chain_workspace_bytes(chunk) // 8, 1), device=device,
                                  dtype=torch.float64)
            self.state = api.new_mh_state(req.seed, req.rid, device=device)
        self.keep = keep

    @staticmethod
    def bytes_needed(req: Request, model: Model, chunk: int) -> int:
        B, V = req.batch, model.V
        return B * V * 4 + B * (8 * 4 + 1) + 8 * chunk + 48

    def launch_next(self, timeline=None):
        req, B = self.req, self.req.batch
        a = self.next
        b = min(B, a + self.chunk)
        phi4 = (req.m2, req.lam)
        with torch.cuda.stream(self.stream):
            if timeline is not None:
                t0 = torch.cuda.Event(enable_timing=True)
                t0.record(self.stream)
            out = api.SampleResult(phi=self.phi[a:b], logq=self.logq[a:b], S=self.S[a:b],
                                   logw=self.logw[a:b])
            self.model.flow.sample(b - a, seed=req.seed, counter0=a, phi4=phi4, out=out)
            api.mh_chain(self.state, self.logw[a:b], workspace=self.ws, chain_idx=self.idx[a:b],
                         acc=self.acc[a:b])
            self.event = torch.cuda.Event(enable_timing=timeline is not None)
            self.event.record(self.stream)
            if timeline is not None:
                timeline.append((self.req.rid, t0, self.event))
        self.next = b

    def finished(self) -> bool:
        return self.next >= self.req.batch and (self.event is None or self.event.query())

    def ready(self) -> bool:
        return self.next < self.req.batch and (self.event is None or self.event.query())


class Server:
    """Continuous-batching loop over resident models (see module docstring)."""

    def __init__(self, models: dict, hbm_budget_bytes: int = 8 << 30, max_active: int = 16,
                 chunk: int = 1024, device=None):
        self.models = models
        self.budget = int(hbm_budget_bytes)
        self.max_active = int(max_active)
        self.chunk = int(chunk)
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(self.max_active)]
        # one device status slot per stream: errors are attributed to the request on it
        self.slots = torch.zeros(self.max_active, dtype=torch.int32, device=self.device)
        for i, st in enumerate(self.streams):
            api.set_stream_status_slot(st, self.slots[i:i + 1])

    def close(self):
        """Removes the streams' status-slot associations (also done when the
        server is garbage collected).  The association belongs to the stream
        handle, and torch hands out pooled streams, so a server should be
        closed before another one is created on the same device."""
        for st in getattr(self, "streams", []) or []:
            if st is not None and getattr(self, "slots", None) is not None:
                api.set_stream_status_slot(st, None)
        self.slots = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _take_error(self, si: int) -> int:
        """Reads and clears stream si's status slot (its work has completed)."""
        return api.device_status(self.streams[si])

    def run(self, requests, keep_results: bool = True, realtime: bool = True, poll_s: float = 50e-6,
            timeline: bool = False):
        """Serves `requests` (arrival times relative to the start) and returns
        (results by rid, stats).  realtime=False admits every request at t=0.
        timeline=True records a CUDA event pair around every chunk (sample +
        MH chain on the request's stream) and adds to the stats how much of the
        GPU-busy time had chunks of two or more requests in flight at once."""
        chunks = [] if timeline else None
        ref = None
        if timeline:
            ref = torch.cuda.Event(enable_timing=True)
            ref.record(torch.cuda.current_stream(self.device))
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        pi = 0
        free_streams = list(range(self.max_active))
        active: dict[int, tuple[_Active, int, int]] = {}
        results: dict[int, Result] = {}
        used = 0
        peak_used = 0
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        admitted_at = {}
        max_concurrent = 0
        while pi < len(pending) or active:
            t = now()
            # admit in arrival order while the slot count and the HBM budget allow
            while pi < len(pending) and free_streams:
                r = pending[pi]
                if realtime and r.arrival > t:
                    break
                m = self.models[r.model]
                need = _Active.bytes_needed(r, m, self.chunk)
                if need > self.budget:
                    raise ValueError(f"request {r.rid} needs {need} bytes, budget {self.budget}")
                if used + need > self.budget:
                    break
                si = free_streams.pop()
                active[r.rid] = (_Active(r, m, self.device, self.streams[si], self.chunk, keep_results), si, need)
                admitted_at[r.rid] = t
                used += need
                peak_used = max(peak_used, used)
                pi += 1
            max_concurrent = max(max_concurrent, len(active))
            # keep one chunk in flight per active request
            progressed = False
            for rid, (st, si, need) in list(active.items()):
                if st.ready():
                    if chunks is not None:
                        st.launch_next(chunks)
                    else:
                        st.launch_next()
                    progressed = True
                elif st.finished():
                    done = now()
                    r = st.req
                    err = self._take_error(si)
                    if keep_results:
                        results[rid] = Result(rid, st.phi, st.logq, st.S, st.logw, st.idx, st.acc, st.state,
                                              r.arrival if realtime else 0.0, admitted_at[rid], done, err)
                    else:
                        results[rid] = Result(rid, None, None, None, None, None, None, None,
                                              r.arrival if realtime else 0.0, admitted_at[rid], done, err)
                    del active[rid]
                    free_streams.append(si)
                    used -= need
                    progressed = True
            if not progressed:
                if pi < len(pending) and not active and realtime:
                    wait = pending[pi].arrival - now()
                    if wait > 0:
                        time.sleep(min(wait, 1e-3))
                else:
                    time.sleep(poll_s)
        torch.cuda.synchronize(self.device)
        lat = np.array([r.latency for r in results.values()])
        wall = now()
        stats = {
            "requests": len(results),
            "wall_s": wall,
            "configs": int(sum(r.batch for r in requests)),
            "configs_per_s": float(sum(r.batch for r in requests) / wall) if wall > 0 else 0.0,
            "p50_latency_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
            "p99_latency_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
            "max_concurrent_requests": max_concurrent,
            "peak_budget_bytes": peak_used,
            "failed_requests": int(sum(1 for r in results.values() if r.error)),
        }
        if chunks:
            iv = [(rid, ref.elapsed_time(a), ref.elapsed_time(b)) for rid, a, b in chunks]
            stats.update(overlap_stats(iv))
        return results, stats


def overlap_stats(intervals):
    """From (request id, start ms, end ms) of every chunk: the GPU-busy time
    (union of the intervals), the part of it during which chunks of at least
    two different requests were in flight, and the most requests in flight at
    once."""
    ev = []
    for rid, a, b in intervals:
        ev.append((a, 1, rid))
        ev.append((b, -1, rid))
    ev.sort(key=lambda e: (e[0], e[1]))
    live = {}
    busy = multi = 0.0
    peak = 0
    last = None
    for t, d, rid in ev:
        if last is not None:
            n_req = sum(1 for v in live.values() if v > 0)
            if n_req >= 1:
                busy += t - last
            if n_req >= 2:
                multi += t - last
        live[rid] = live.get(rid, 0) + d
        peak = max(peak, sum(1 for v in live.values() if v > 0))
        last = t
    return {"gpu_busy_ms": busy, "overlapped_ms": multi,
            "overlapped_fraction": multi / busy if busy > 0 else 0.0, "max_requests_in_flight": peak}


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process (exponential gaps), seconds from 0."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))

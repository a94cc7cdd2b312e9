"""Host logic of the continuous-batching loop (serving.Server), on the CPU.

The device work of a request (chunks of gf_flow_sample + gf_mh_chain on its
own stream) is replaced by a stand-in whose chunks finish after a few polls, so
the admission policy, the HBM budget accounting, the request slots and the
retirement can be checked without a GPU.
"""
import pytest

import gf_inputs as gi
from paper_2208_08903_gb300 import serving as SV


class FakeActive:
    """Stand-in for serving._Active: a chunk 'runs' for two polls."""
    admitted = []

    def __init__(self, req, model, device, stream, chunk, keep):
        self.req, self.model, self.chunk, self.stream = req, model, chunk, stream
        self.next, self.inflight = 0, 0
        self.phi = self.logq = self.S = self.logw = self.idx = self.acc = self.state = None
        FakeActive.admitted.append(req.rid)

    bytes_needed = staticmethod(SV._Active.bytes_needed)

    def launch_next(self):
        self.next = min(self.req.batch, self.next + self.chunk)
        self.inflight = 2

    def ready(self):
        if self.inflight:
            self.inflight -= 1
            return False
        return self.next < self.req.batch

    def finished(self):
        return self.next >= self.req.batch and self.inflight == 0


@pytest.fixture
def server(monkeypatch):
    FakeActive.admitted = []
    monkeypatch.setattr(SV, "_Active", FakeActive)
    monkeypatch.setattr(SV.torch.cuda, "synchronize", lambda *a, **k: None)

    def make(budget, max_active, chunk=256):
        srv = object.__new__(SV.Server)
        shape = gi.FlowShape(2, 8, 4, 8, 8)
        srv.models = {"m": SV.Model("m", shape, None)}
        srv.budget, srv.max_active, srv.chunk = budget, max_active, chunk
        srv.device = "cpu"
        srv.streams = [None] * max_active
        srv._take_error = lambda si: 0            # no device: no kernel errors
        return srv
    return make


def requests(n, batch=1000):
    return [SV.Request(rid=i, model="m", m2=-4.0, lam=8.0, batch=batch + 37 * i, seed=i) for i in range(n)]


def test_every_request_completes_in_arrival_order(server):
    reqs = requests(9)
    srv = server(budget=1 << 30, max_active=3)
    results, stats = srv.run(list(reversed(reqs)), realtime=False)
    assert sorted(results) == list(range(9))
    assert FakeActive.admitted == list(range(9))          # (arrival, rid) order
    assert stats["requests"] == 9 and stats["configs"] == sum(r.batch for r in reqs)
    assert stats["max_concurrent_requests"] <= 3
    assert all(r.latency >= 0 for r in results.values())


def test_budget_bounds_the_admitted_requests(server):
    reqs = requests(6, batch=2000)
    shape = gi.FlowShape(2, 8, 4, 8, 8)
    need = [SV._Active.bytes_needed(r, SV.Model("m", shape, None), 256) for r in reqs]
    budget = need[4] + need[5] + 1                        # room for any two, not three
    srv = server(budget=budget, max_active=16)
    results, stats = srv.run(reqs, realtime=False)
    assert len(results) == 6
    assert stats["peak_budget_bytes"] <= budget
    assert stats["max_concurrent_requests"] == 2


def test_request_larger_than_the_budget_is_rejected(server):
    srv = server(budget=1000, max_active=4)
    with pytest.raises(ValueError):
        srv.run(requests(1), realtime=False)


def test_bytes_needed_counts_outputs_chain_and_workspace():
    shape = gi.FlowShape(3, 4, 4, 8, 8)
    r = SV.Request(rid=0, model="m", m2=0.0, lam=1.0, batch=100, seed=0)
    # phi FP32 [B][V] + log q, S, log w, chain index (8 B each) + accept flag (1 B)
    # + 8 B per proposal of one chunk's workspace + the chain state
    assert SV._Active.bytes_needed(r, SV.Model("m", shape, None), 64) == 100 * 64 * 4 + 100 * 33 + 8 * 64 + 48


def test_device_error_marks_only_its_request_failed(server):
    """The status slot read when a request retires belongs to that request's
    stream: a non-zero slot fails that request alone."""
    srv = server(budget=1 << 40, max_active=3)
    on_stream = {}

    def take_error(si):
        return on_stream.pop(si, 0)
    srv._take_error = take_error
    reqs = requests(6)
    orig_launch = FakeActive.launch_next

    def launch(self):
        orig_launch(self)
        if self.req.rid == 4:                 # a kernel of request 4 records GF_ETIMEOUT (-5)
            on_stream[srv.streams.index(self.stream)] = -5
    FakeActive.launch_next = launch
    srv.streams = [f"s{i}" for i in range(3)]
    try:
        res, stats = srv.run(reqs, realtime=False)
    finally:
        FakeActive.launch_next = orig_launch
    assert res[4].error == -5
    assert all(res[i].error == 0 for i in res if i != 4)
    assert stats["failed_requests"] == 1


def test_overlap_statistics():
    """Busy time is the union of the chunks' intervals; overlapped time counts
    only moments with chunks of two or more different requests in flight."""
    iv = [(1, 0.0, 10.0), (2, 5.0, 15.0), (3, 20.0, 30.0), (1, 25.0, 26.0), (1, 26.0, 27.0)]
    st = SV.overlap_stats(iv)
    assert st["gpu_busy_ms"] == 25.0
    assert st["overlapped_ms"] == 7.0
    assert st["max_requests_in_flight"] == 2
    one = SV.overlap_stats([(4, 0.0, 3.0), (4, 3.0, 5.0), (4, 4.0, 6.0)])   # one request's own chunks
    assert one["overlapped_ms"] == 0.0 and one["gpu_busy_ms"] == 6.0

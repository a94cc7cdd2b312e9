"""CPU model of the synchronisation protocol of the second tensor-core kernel
(paper_2208_08903_gb300/csrc/gf_flow_tc.cu; no GPU).

One block half runs: two MMA-issuing threads (tiles t = 0 and t = 1 mod 2,
each into the TMEM ring of its epilogue group), two epilogue groups, the
tensor-core work each issuer queued (completing in issue order per issuer, in
any order across them), the bulk weight copies and the thread 0 that stages
them; all of the half's threads meet at a barrier between the phases (conv1,
conv2, halo, head).  This model replays the kernel's loops, waits, arrivals,
commits and copies under many random schedules and checks:

* no deadlock;
* every mbarrier wait is by phase parity, which is correct only if the barrier
  has completed exactly n or n + 1 times when a thread waits for completion n;
* a TMEM accumulator is refilled only after its epilogue group has read it;
* h2 of a tile is written over h1 only when no queued conv2 MMA still reads
  those positions (the in-place rule with its lag of r tiles);
* W2 / W3 of the next layer are staged only when no MMA of this layer that
  reads them is still queued, and the FP32 part only into a buffer no thread
  still reads.

The failure path: a wait runs out at a random point (GF_ETIMEOUT, the abort
flag); every agent must leave its loops, the queued tensor-core work must be
complete before TMEM is freed, and no bulk copy may still be landing when the
half exits.  Planted mistakes (no in-place lag, no wait for a drained
accumulator, W2 staged before the conv2 phase ends) are caught.
"""
import random

import pytest


class Violation(AssertionError):
    pass


class Deadlock(Violation):
    pass


class Barrier:
    def __init__(self, name, count):
        self.name, self.count, self.arrived, self.done = name, count, 0, 0

    def arrive(self, k=1):
        self.arrived += k
        assert self.arrived <= self.count, self.name
        if self.arrived == self.count:
            self.arrived = 0
            self.done += 1


def geometry(nd, L):
    P = L + 2
    p_first = 1 + P + (P * P if nd == 3 else 0)
    p_last = p_first * L
    nt = (p_last - p_first + 1 + 95) // 96
    r = (p_first + 95) // 96
    return p_first, nt, r


class Half:
    """State shared by the agents of one block half."""

    def __init__(self, nd, L, n_cfg, n_layers, nb2, nb3, rng, mutation=None):
        self.p_first, self.nt, self.r = geometry(nd, L)
        self.n_cfg, self.nl, self.nb2, self.nb3 = n_cfg, n_layers, nb2, nb3
        self.rng, self.mut = rng, mutation
        self.total = n_cfg * n_layers
        self.B = {}
        for g in range(2):
            for i in range(nb2):
                self.B[f"full2_{g}_{i}"] = Barrier("full2", 1)
                self.B[f"empty2_{g}_{i}"] = Barrier("empty2", 1)     # the group (one arrival here)
            for i in range(nb3):
                self.B[f"full3_{g}_{i}"] = Barrier("full3", 1)
                self.B[f"empty3_{g}_{i}"] = Barrier("empty3", 1)
        for t in range(self.nt):
            self.B[f"done2_{t}"] = Barrier("done2", 1)
        for k in ("w2", "w3", "wf0", "wf1"):
            self.B[k] = Barrier(k, 2)            # expect_tx arrival + the copy's completion
        self.B["fin"] = Barrier("fin", 2)
        self.queues = {0: [], 1: []}             # queued MMA groups per issuer
        self.copies = []                         # bulk copies in flight: barrier names
        self.tmem = {}                           # (conv, ring, i) -> "filled"/"read"/"pending"
        self.abort = False
        self.status = None
        self.w2_layer = self.w3_layer = None     # step whose weights are staged
        self.wf_readers = {0: 0, 1: 0}

    # ---- mbarrier waits by parity
    def wait_ok(self, name, n):
        b = self.B[name]
        if b.done > n + 1 or b.done < n:
            raise Violation(f"parity wait on {name} for completion {n} with {b.done} completions")
        return b.done == n + 1

    def reads_positions(self, t):
        # conv2 tile t reads positions 96 t .. 96 t + 96 + 2 p_first - 1
        return 96 * t, 96 * t + 96 + 2 * self.p_first - 1

    def out_positions(self, t):
        lo = self.p_first + 96 * t
        return lo, lo + 95


def run(nd, L, n_cfg, n_layers, nb2, nb3, seed, mutation=None, abort_at=None):
    rng = random.Random(seed)
    h = Half(nd, L, n_cfg, n_layers, nb2, nb3, rng, mutation)
    nt, r = h.nt, h.r
    waits = {"n": 0}

    def wait(name, n):
        """generator: a bounded wait; returns False (and aborts) when abort_at fires"""
        waits["n"] += 1
        k = waits["n"]
        while True:
            if h.abort:
                return False
            if h.wait_ok(name, n):
                return True
            if abort_at is not None and k >= abort_at:
                h.abort, h.status = True, "GF_ETIMEOUT"
                return False
            h.blocked = True
            yield

    def stage(name, what, step):
        h.B[name].arrive()                       # expect_tx
        h.copies.append((name, what, step))

    sync = {"count": 0, "gen": 0, "abort": {}}
    n_agents = 5                                 # issuer 0, issuer 1, group 0, group 1, stager

    def half_sync():
        """the half's barrier; returns the abort flag as every thread reads it
        right after the barrier (a wait that runs out takes far longer than
        the other threads' read of the flag)"""
        g = sync["gen"]
        sync["count"] += 1
        if sync["count"] == n_agents:
            sync["count"] = 0
            sync["abort"][g] = h.abort
            sync["gen"] += 1
        while sync["gen"] == g:
            h.blocked = True
            yield
        return sync["abort"][g]

    def issuer(rg):
        i2 = i3 = 0
        k2 = k3 = 0
        for step in range(h.total):
            # conv1 phase (all threads) -> barrier
            if (yield from half_sync()):
                break
            ok = yield from wait("w2", step)
            for t in range(rg, nt, 2):
                if not ok:
                    break
                if k2 >= 1 and h.mut != "no_empty_wait":
                    ok = yield from wait(f"empty2_{rg}_{i2}", k2 - 1)
                    if not ok:
                        break
                key = ("c2", rg, i2)
                if h.tmem.get(key) in ("filled", "pending"):
                    raise Violation(f"conv2 accumulator {key} refilled before its epilogue read it")
                h.tmem[key] = "pending"
                h.queues[rg].append(dict(kind="c2", t=t, step=step, key=key, done=f"done2_{t}",
                                         full=f"full2_{rg}_{i2}", reads=h.reads_positions(t)))
                i2 += 1
                if i2 == nb2:
                    i2, k2 = 0, k2 + 1
                yield
            if (yield from half_sync()):         # end of the conv2 phase
                break
            yield from half_sync()               # end of the halo phase
            ok = yield from wait("w3", step)
            for t in range(rg, nt, 2):
                if not ok:
                    break
                if k3 >= 1:
                    ok = yield from wait(f"empty3_{rg}_{i3}", k3 - 1)
                    if not ok:
                        break
                key = ("c3", rg, i3)
                if h.tmem.get(key) in ("filled", "pending"):
                    raise Violation(f"head accumulator {key} refilled before its epilogue read it")
                h.tmem[key] = "pending"
                h.queues[rg].append(dict(kind="c3", t=t, step=step, key=key, done=None,
                                         full=f"full3_{rg}_{i3}", reads=None))
                i3 += 1
                if i3 == nb3:
                    i3, k3 = 0, k3 + 1
                yield
            if (yield from half_sync()):         # end of the head phase
                break
        # teardown: the final commit
        h.queues[rg].append(dict(kind="fin", full="fin"))
        h.done_agents.add(f"issuer{rg}")

    def group(eg):
        i2 = i3 = 0
        k2 = k3 = 0
        for step in range(h.total):
            if (yield from half_sync()):         # after conv1
                break
            dwaited = 0
            ok = True
            for t in range(eg, nt, 2):
                ok = yield from wait(f"full2_{eg}_{i2}", k2)
                if not ok:
                    break
                key = ("c2", eg, i2)
                if h.tmem.get(key) != "filled":
                    raise Violation(f"epilogue read {key} in state {h.tmem.get(key)}")
                h.tmem[key] = "read"
                h.B[f"empty2_{eg}_{i2}"].arrive()
                i2 += 1
                if i2 == nb2:
                    i2, k2 = 0, k2 + 1
                lag = r - 1 if h.mut == "short_lag" else r
                need = min(t + lag, nt - 1)
                if h.mut != "no_lag":
                    while ok and dwaited <= need:
                        ok = yield from wait(f"done2_{dwaited}", step)
                        dwaited += 1
                if not ok:
                    break
                lo, hi = h.out_positions(t)
                for q in h.queues.values():
                    for gr in q:
                        if gr["kind"] == "c2" and gr["step"] == step and not (gr["reads"][1] < lo or gr["reads"][0] > hi):
                            raise Violation(f"h2 of tile {t} written while conv2 of tile {gr['t']} still reads it")
                yield
            if (yield from half_sync()):         # end of the conv2 phase
                break
            yield from half_sync()               # end of the halo phase
            for t in range(eg, nt, 2):
                ok = yield from wait(f"full3_{eg}_{i3}", k3)
                if not ok:
                    break
                key = ("c3", eg, i3)
                if h.tmem.get(key) != "filled":
                    raise Violation(f"head epilogue read {key} in state {h.tmem.get(key)}")
                h.tmem[key] = "read"
                h.B[f"empty3_{eg}_{i3}"].arrive()
                i3 += 1
                if i3 == nb3:
                    i3, k3 = 0, k3 + 1
                yield
            if (yield from half_sync()):         # end of the head phase
                break
        h.done_agents.add(f"group{eg}")

    def stager():
        """thread 0's staging of the weight copies (thread 0 is also issuer 0
        in the kernel; its staging happens at these points of the phases)"""
        w2_i = w3_i = wf_i = -1
        if h.total > 0:
            stage("w2", "W2", 0); stage("w3", "W3", 0); stage("wf0", "wf", 0)
            w2_i = w3_i = wf_i = 0
        for step in range(h.total):
            ok = yield from wait(f"wf{step & 1}", step >> 1)
            if ok and step + 1 < h.total:
                if h.wf_readers[(step + 1) & 1]:
                    raise Violation("FP32 weights staged into a buffer still being read")
                stage(f"wf{(step + 1) & 1}", "wf", step + 1)
                wf_i = step + 1
            h.wf_readers[step & 1] += 1
            if h.mut == "early_w2" and step + 1 < h.total:
                stage("w2", "W2", step + 1)
                w2_i = step + 1
            if (yield from half_sync()):         # end of conv1
                h.wf_readers[step & 1] -= 1
                break
            if (yield from half_sync()):         # end of the conv2 phase
                h.wf_readers[step & 1] -= 1
                break
            if step + 1 < h.total and h.mut != "early_w2":
                for q in h.queues.values():
                    if any(g["kind"] == "c2" for g in q):
                        raise Violation("W2 of the next layer staged while conv2 MMAs are queued")
                stage("w2", "W2", step + 1)
                w2_i = step + 1
            yield from half_sync()               # end of the halo phase
            ab = yield from half_sync()          # end of the head phase
            h.wf_readers[step & 1] -= 1
            if ab:
                break
            if step + 1 < h.total:
                for q in h.queues.values():
                    if any(g["kind"] == "c3" for g in q):
                        raise Violation("W3 of the next layer staged while head MMAs are queued")
                stage("w3", "W3", step + 1)
                w3_i = step + 1
        # teardown: wait for the last copies and for the issuers' final commits
        for name, n in (("w2", w2_i), ("w3", w3_i), (f"wf{wf_i & 1}", wf_i >> 1)):
            if n >= 0:
                while h.B[name].done < n + 1:
                    h.blocked = True
                    yield
        while h.B["fin"].done < 1:
            h.blocked = True
            yield
        if any(h.queues[q] for q in h.queues):
            raise Violation("TMEM freed with tensor-core work still queued")
        if h.copies:
            raise Violation("exit with a bulk copy still landing")
        h.done_agents.add("stager")

    def tensor_core():
        while True:
            live = [q for q in (0, 1) if h.queues[q]]
            h.blocked = not live and not h.copies
            if live:
                q = rng.choice(live)
                gr = h.queues[q].pop(0)
                if gr["kind"] == "fin":
                    h.B["fin"].arrive()
                else:
                    if gr["kind"] == "c2" and h.w2_layer != gr["step"]:
                        raise Violation(f"conv2 MMA of step {gr['step']} read W2 of step {h.w2_layer}")
                    if gr["kind"] == "c3" and h.w3_layer != gr["step"]:
                        raise Violation(f"head MMA of step {gr['step']} read W3 of step {h.w3_layer}")
                    h.tmem[gr["key"]] = "filled"
                    h.B[gr["full"]].arrive()
                    if gr["done"]:
                        h.B[gr["done"]].arrive()
            if h.copies and rng.random() < 0.5:
                name, what, step = h.copies.pop(0)
                if what == "W2":
                    h.w2_layer = step
                elif what == "W3":
                    h.w3_layer = step
                h.B[name].arrive()
            yield

    h.done_agents = set()
    agents = [issuer(0), issuer(1), group(0), group(1), stager()]
    tc = tensor_core()
    live = list(range(len(agents)))
    # deadlock: a long run of scheduler steps in which every step found its
    # agent spinning in a wait (or the tensor cores with nothing to do)
    stall = 0
    while live:
        pick = rng.choice(live + [-1, -1])
        h.blocked = False
        if pick == -1:
            next(tc)
        else:
            try:
                next(agents[pick])
            except StopIteration:
                live.remove(pick)
        stall = stall + 1 if h.blocked else 0
        if stall > 20000:
            raise Deadlock(f"deadlock: {sorted(h.done_agents)} finished")
    # the tensor cores finish whatever is left (only the final commits)
    for _ in range(1000):
        next(tc)
    return h


SHAPES = [(2, 32), (2, 64), (3, 8), (3, 12), (2, 8)]


@pytest.mark.parametrize("nd,L", SHAPES)
# TMEM rings of the launches: width 32 (1 or 2 buffers per group with two or
# one halves), 16 (2 / 5), 8 (4 / 8); plus small and odd sizes
@pytest.mark.parametrize("nb2,nb3", [(1, 8), (2, 2), (5, 16), (4, 8), (8, 8)])
def test_protocol_random_schedules(nd, L, nb2, nb3):
    for seed in range(6):
        h = run(nd, L, n_cfg=2, n_layers=3, nb2=nb2, nb3=nb3, seed=seed)
        assert h.status is None and h.done_agents == {"issuer0", "issuer1", "group0", "group1", "stager"}


@pytest.mark.parametrize("nd,L", [(2, 32), (3, 12)])
def test_protocol_abort_anywhere(nd, L):
    rng = random.Random(5)
    for k in range(40):
        h = run(nd, L, n_cfg=2, n_layers=2, nb2=1, nb3=8, seed=100 + k, abort_at=rng.randint(1, 60))
        assert h.done_agents == {"issuer0", "issuer1", "group0", "group1", "stager"}


@pytest.mark.parametrize("mutation", ["no_lag", "short_lag", "no_empty_wait", "early_w2"])
def test_protocol_catches_planted_mistakes(mutation):
    caught = False
    for seed in range(40):
        try:
            run(3, 12, n_cfg=2, n_layers=3, nb2=1, nb3=8, seed=seed, mutation=mutation)
        except Violation:
            caught = True
            break
    assert caught, mutation


def lag_fits(r, nb2):
    """The conv2 schedule's condition: an epilogue group holding tile t's
    store waits for tile t + r's MMAs, which need the TMEM buffer of tile
    t + r - 2 nb2 drained; with r even that tile belongs to the same group, so
    it must be tile t or earlier; with r odd, the other group's current tile
    t + 1 or earlier."""
    return r <= 2 * nb2 + (r & 1)


@pytest.mark.parametrize("nd,L", [(2, 64), (3, 8), (3, 12), (3, 16)])
@pytest.mark.parametrize("nb2", [1, 2, 3, 5, 8])
def test_protocol_deadlocks_exactly_when_the_ring_is_short_for_the_lag(nd, L, nb2):
    _, _, r = geometry(nd, L)
    for seed in range(3):
        if lag_fits(r, nb2):
            run(nd, L, n_cfg=2, n_layers=2, nb2=nb2, nb3=8, seed=seed)
        else:
            with pytest.raises(Deadlock):
                run(nd, L, n_cfg=2, n_layers=2, nb2=nb2, nb3=8, seed=seed)


def test_launch_rings_fit_the_lag():
    """Every shape the kernel takes (gf_flow_tensor_core_supported, less the
    3D L=16 width-32 shape, which has its own kernel), with the TMEM rings its
    launch gives it (512 columns, or 256 per half with two halves; conv2
    accumulators of 3 Cp columns, 32 at width 8; at most 8 per group),
    satisfies the condition; the launcher also refuses any launch that would
    not (GF_EUNSUPPORTED)."""
    import ctypes as C
    from paper_2208_08903_gb300 import _abi
    lib = _abi.load()

    def ex(nd, L, c):
        hid = (C.c_int32 * _abi.GF_MAX_HIDDEN)(*([c, c] + [0] * (_abi.GF_MAX_HIDDEN - 2)))
        return _abi.FlowShapeExC(nd, L, 4, 2, hid, 3, 1, 0.01)

    n = 0
    for nd, Ls in ((2, range(4, 66, 2)), (3, range(4, 18, 2))):
        for L in Ls:
            for c in (8, 16, 24, 32):
                if (nd, L, c) == (3, 16, 32) or not lib.gf_flow_tensor_core_supported(C.byref(ex(nd, L, c))):
                    continue
                n2 = 32 if c == 8 else (48 if c == 16 else 96)
                _, _, r = geometry(nd, L)
                for cols in (512, 256):
                    nb2 = min(8, cols // (2 * n2))
                    assert nb2 >= 1 and lag_fits(r, nb2), (nd, L, c, cols, r, nb2)
                n += 1
    assert n >= 20

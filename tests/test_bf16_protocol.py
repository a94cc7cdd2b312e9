"""CPU model of the BF16 flow kernel's synchronisation protocol (no GPU).

The kernel (paper_2208_08903_gb300/csrc/gf_flow_bf16.cu) runs eight kinds of
agents that meet only through mbarriers: four MMA-issuing threads (conv2 of
M-tile 0 and 1, conv3 batches, conv1), the conv1 workers, the epilogue, the
tensor-core work each issuer queued (completing in issue order) and the bulk
weight copies.  This model replays their loops exactly as the kernel orders its
waits, arrivals and commits, under many random schedules, and checks:

* no deadlock;
* every mbarrier wait is by phase parity, which is correct only if the barrier
  has completed exactly n or n+1 times when a thread waits for completion n;
* no buffer is overwritten while an earlier reader may still read it (h1 and h2
  slots, the conv1 operand buffers, the TMEM accumulators and batch regions,
  the staged weights of each layer);
* conv1 reads each field slice only after the previous layer has updated it, and
  a layer updates a slice only after the previous layer's conv1 reads of it.

It also replays the failure path: one role's wait runs out at a random point
(the kernel then records GF_ETIMEOUT and raises the CTA's abort flag; every
other wait gives up once it sees the flag), and checks that every role leaves
its loops, that the tensor-core work still queued is complete before TMEM is
freed (the issuers' final commit to bar_fin) and that no bulk weight copy is
still writing shared memory when the CTA exits.

Several workers or epilogue warps act as one agent here (their per-thread
arrivals are one arrival); the model checks the protocol, not the arithmetic.
Planted mistakes (a skipped wait, weights staged early, no slice rotation) are
caught.  The field checkpoints turn out to be implied by the h1-slot waits (a
checkpoint planted too early goes unnoticed); the kernel keeps them as an
explicit guard.
"""
import random

import pytest

L = 16                       # slices per layer
C1_PER_LAYER, C2_PER_LAYER = 20, 18


class Violation(AssertionError):
    pass


class Barrier:
    def __init__(self, name, count):
        self.name, self.count, self.arrived, self.done = name, count, 0, 0

    def arrive(self):
        self.arrived += 1
        if self.arrived == self.count:
            self.arrived = 0
            self.done += 1


class Model:
    def __init__(self, n_configs, n_layers, seed):
        self.rng = random.Random(seed)
        self.nc, self.nl = n_configs, n_layers
        B = {}
        for i in range(4):
            B[f"h1{i}"] = Barrier(f"h1{i}", 1)
            B[f"m2{i}"] = Barrier(f"m2{i}", 1)
            B[f"x{i}"] = Barrier(f"x{i}", 1)
        for i in range(3):
            B[f"h2{i}"] = Barrier(f"h2{i}", 1)
            B[f"t3{i}"] = Barrier(f"t3{i}", 1)
        for i in range(2):
            B[f"m3{i}"] = Barrier(f"m3{i}", 1)
            B[f"t2{i}"] = Barrier(f"t2{i}", 1)
            B[f"b1{i}"] = Barrier(f"b1{i}", 1)
            B[f"c1{i}"] = Barrier(f"c1{i}", 1)
        B["w2"] = Barrier("w2", 2)          # expect_tx arrival + copy completion
        B["w3"] = Barrier("w3", 2)
        self.B = B
        self.queues = {k: [] for k in ("qA", "qB", "qC", "qD", "copy")}
        # resource state: version held and readers still pending per version
        self.h1 = [None] * 4
        self.h2 = [None] * 3
        self.im2col = [None] * 2
        self.tm_c1 = [None] * 2           # conv1 accumulators: version written (None = drained)
        self.tm_c2 = [None] * 2           # conv2 tile buffers
        self.tm_c3 = [None] * 3           # conv3 batch regions
        self.c3_left = {}                 # batch -> slices still to read it
        self.w = {"W1": None, "W2": None, "W3": None, "wf": None}
        self.pending = []                 # queued tensor-core groups: dict(reads=..., ...)
        self.x = {}                       # (slice, parity) -> global layer that last wrote it
        self.x_reads = {}                 # (slice, parity) -> layers whose conv1 still may read it

    # ---- helpers
    def check_wait(self, name, n):
        b = self.B[name]
        if b.done not in (n, n + 1):
            raise Violation(f"parity wait on {name} for completion {n} with {b.done} completions")
        return b.done == n + 1

    def pending_reads(self, pred):
        return any(pred(g) for g in self.pending)


def frozen_of(s_local):
    return s_local & 1


def rot(li):
    return (4 * li) & 15


def run(n_configs, n_layers, seed, mutation=None, abort_at=None):
    """Replays the kernel's loops; `mutation` plants one protocol mistake (for the
    tests that show the model catches it).  abort_at = (agent, k): the first wait
    of that agent from its k-th on that is not already satisfied runs out.
    Returns the status word (None or "GF_ETIMEOUT")."""
    m = Model(n_configs, n_layers, seed)
    B = m.B
    nl = n_layers
    m.abort = False
    m.status = None
    n_waits = {}

    waiting = {}
    current = [None]

    def wait(name, n, who=None):
        """True once completion n of `name` is seen; False when this wait runs
        out (abort_at) or gives up because another thread aborted."""
        me = current[0]
        n_waits[me] = n_waits.get(me, 0) + 1
        while True:
            if m.check_wait(name, n):
                return True
            if m.abort:                      # the flag is polled while the wait spins
                return False
            if abort_at is not None and abort_at[0] == me and n_waits[me] >= abort_at[1]:
                m.abort = True
                m.status = "GF_ETIMEOUT"
                return False
            waiting[me] = (name, n, B[name].done)
            yield

    def issue(queue, group):
        # a queued group may read its inputs and write its outputs any time until it completes
        m.pending.append(group)
        m.queues[queue].append(group)

    # ---------------- agents
    def conv2_issuer(t, cfg):
        q = "qA" if t == 0 else "qB"
        for li in range(nl):
            s = cfg * nl + li
            c0, g20 = s * C1_PER_LAYER, s * C2_PER_LAYER
            if not (yield from wait("w2", s)):
                return
            if m.w["W2"] != s:
                raise Violation("conv2 issued before its W2")
            for u in range(-1, L + 1):
                for v in (range(-2, 1) if u == -1 else [u + 1]):
                    c = c0 + v + 2
                    if not (yield from wait(f"h1{c & 3}", c >> 2)):
                        return
                g2 = g20 + u + 1
                if g2 >= 1 and mutation != "no_t2_wait":
                    if not (yield from wait(f"t2{t}", g2 - 1)):
                        return
                reads = [c0 + v + 2 for v in (u - 1, u, u + 1)]
                for c in reads:
                    if m.h1[c & 3] != c:
                        raise Violation(f"conv2 {g2} reads h1 slot {c & 3} holding {m.h1[c & 3]}, wants {c}")
                if m.tm_c2[t] is not None:
                    raise Violation(f"conv2 {g2} tile {t} overwrites undrained {m.tm_c2[t]}")
                m.tm_c2[t] = g2
                issue(q, dict(kind="conv2", t=t, g2=g2, h1=reads, W2=s, commit=f"m2{2 * t + (g2 & 1)}"))
                yield

    def conv3_issuer(cfg):
        for li in range(nl):
            s = cfg * nl + li
            g20 = s * C2_PER_LAYER
            if not (yield from wait("w3", s)):
                return
            if m.w["W3"] != s:
                raise Violation("conv3 issued before its W3")
            for ub in range(-1, L + 1):
                gh = g20 + ub + 1
                if not (yield from wait(f"h2{gh % 3}", gh // 3)):
                    return
                if gh >= 3 and mutation != "no_t3_wait":
                    if not (yield from wait(f"t3{gh % 3}", (gh - 3) // 3)):
                        return
                if m.h2[gh % 3] != gh:
                    raise Violation(f"batch {gh} reads h2 slot holding {m.h2[gh % 3]}")
                if m.c3_left.get(gh - 3, 0) > 0:
                    raise Violation(f"batch {gh} overwrites region of batch {gh - 3} still to be read")
                m.tm_c3[gh % 3] = gh
                # slices ub-1, ub, ub+1 of the layer read it (those that exist)
                m.c3_left[gh] = sum(1 for w in (ub - 1, ub, ub + 1) if 0 <= w < L)
                issue("qC", dict(kind="conv3", gh=gh, h2=gh, W3=s, commit=f"m3{gh & 1}"))
                yield

    def conv1_issuer(cfg):
        for li in range(nl):
            s = cfg * nl + li
            c0 = s * C1_PER_LAYER
            for v in range(-2, L + 2):
                c = c0 + v + 2
                b = c & 1
                if not (yield from wait(f"b1{b}", c >> 1)):
                    return
                if m.im2col[b] != c or m.w["W1"] != s:
                    raise Violation(f"conv1 {c} reads operand {m.im2col[b]} / W1 {m.w['W1']}")
                if m.tm_c1[b] is not None:
                    raise Violation(f"conv1 {c} overwrites undrained accumulator {m.tm_c1[b]}")
                m.tm_c1[b] = c
                issue("qD", dict(kind="conv1", c=c, im2col=c, W1=s, commit=f"c1{b}"))
                yield

    def copy(resource, version, barrier, pred_readers):
        if m.pending_reads(pred_readers):
            raise Violation(f"bulk copy of {resource} {version} while a queued MMA still reads the old one")
        m.queues["copy"].append(dict(kind="copy", res=resource, ver=version, commit=barrier))
        m.last_copy[barrier] = B[barrier].done     # the completion this copy will bring
        B[barrier].arrive()          # expect_tx arrival

    def workers(cfg):
        kx = 0
        step = 4 if mutation != "rot0" else 0
        for li in range(nl):
            s = cfg * nl + li
            c0, g20 = s * C1_PER_LAYER, s * C2_PER_LAYER
            fr, R = frozen_of(li), (step * li) & 15
            if li == 0:
                copy("W2", s, "w2", lambda g: g["kind"] == "conv2")
                copy("W3", s, "w3", lambda g: g["kind"] == "conv3")
            if m.pending_reads(lambda g: g["kind"] == "conv1"):
                raise Violation("conv1 B operand restaged while a conv1 MMA is queued")
            m.w["W1"] = s
            xseen = L if li == 0 else 0
            kx = 0

            ok = [True]

            def build(v):
                # as the kernel: the checkpoint waits stop at an abort, the operand is
                # still built and signalled (its buffer was drained before)
                nonlocal xseen, kx
                c = c0 + v + 2
                while xseen <= min(v + 5, L - 1) and ok[0]:
                    ok[0] = yield from wait(f"x{kx}", s - 1)
                    xseen = (L - 1 if kx == 3 else 5 + 4 * kx) + 1
                    kx += 1
                for d in (-1, 0, 1):
                    z = (v + R + d) & 15
                    want = s - 1 if li > 0 else ("prior", cfg)
                    if ok[0] and m.x.get((z, fr)) != want:
                        raise Violation(f"conv1 of layer {s} reads slice {z} written by {m.x.get((z, fr))}")
                    m.x_reads.setdefault((z, fr), set()).add(s)
                b = c & 1
                if m.pending_reads(lambda g: g["kind"] == "conv1" and g["im2col"] == c - 2):
                    raise Violation(f"operand {c} overwrites one a queued conv1 still reads")
                m.im2col[b] = c
                B[f"b1{b}"].arrive()
            yield from build(-2)
            yield from build(-1)
            for v in range(-2, L + 2):
                if not ok[0]:
                    return
                c = c0 + v + 2
                if not (yield from wait(f"c1{c & 1}", c >> 1)):
                    return
                if m.tm_c1[c & 1] != c:
                    raise Violation("conv1 drain of the wrong accumulator")
                m.tm_c1[c & 1] = None
                if v == L + 1:       # this layer's conv1 reads are all done
                    for key in list(m.x_reads):
                        m.x_reads[key].discard(s)
                if v + 2 <= L + 1:
                    yield from build(v + 2)
                if not ok[0]:
                    return
                if v >= 2:
                    g2 = g20 + v - 2
                elif li > 0:
                    g2 = g20 - C2_PER_LAYER + min(v + 17, 16) + 1
                else:
                    g2 = -1
                if g2 >= 0 and mutation != "no_slot_wait":
                    if not ((yield from wait(f"m2{g2 & 1}", g2 >> 1)) and
                            (yield from wait(f"m2{2 + (g2 & 1)}", g2 >> 1))):
                        return
                old = m.h1[c & 3]
                if old is not None and m.pending_reads(lambda g: g["kind"] == "conv2" and old in g["h1"]):
                    raise Violation(f"h1 {c} overwrites {old} still read by a queued conv2")
                m.h1[c & 3] = c
                B[f"h1{c & 3}"].arrive()
                if li > 0 and v == (-2 if mutation == "w2_early" else -1):
                    copy("W2", s, "w2", lambda g: g["kind"] == "conv2")
                    if m.wf_reader_pending:
                        raise Violation("biases restaged before the epilogue read the previous ones")
                elif li > 0 and v == 2:
                    gb = g20 - 1
                    if not (yield from wait(f"m3{gb & 1}", gb >> 1)):
                        return
                    copy("W3", s, "w3", lambda g: g["kind"] == "conv3")
                yield

    m.wf_reader_pending = False

    def epilogue(cfg):
        for li in range(nl + 1):
            s = cfg * nl + li
            g20 = s * C2_PER_LAYER
            for u in range(-1, (L if li < nl else 0) + 1):
                g2 = g20 + u + 1
                tail, own = (u <= 0 and li > 0), u >= 3
                if (li > 0 or u >= 1) and not (mutation == "no_batch_wait" and not (tail or own)):
                    gb = g2 - 2
                    if not (yield from wait(f"m3{gb & 1}", gb >> 1)):
                        return
                if tail or own:
                    lj = li - 1 if tail else li
                    w = L - 1 + u if tail else u - 3
                    gj = (cfg * nl + lj) * C2_PER_LAYER + w + 1
                    for gb in (gj - 1, gj, gj + 1):
                        if m.tm_c3[gb % 3] != gb:
                            raise Violation(f"slice {w} of layer {lj} reads region holding {m.tm_c3[gb % 3]}, wants {gb}")
                        m.c3_left[gb] -= 1
                    B[f"t3{(gj - 1) % 3}"].arrive()
                    if w == L - 1:
                        B[f"t3{gj % 3}"].arrive()
                        B[f"t3{(gj + 1) % 3}"].arrive()
                    z, act = (w + ((4 if mutation != "rot0" else 0) * lj)) & 15, 1 - frozen_of(lj)
                    sl = cfg * nl + lj
                    readers = m.x_reads.get((z, act), set())
                    if sl - 1 in readers:
                        raise Violation(f"layer {sl} updates slice {z} before layer {sl - 1}'s conv1 read it")
                    m.x[(z, act)] = sl
                    if w == L - 1:
                        B["x3"].arrive()
                    if w >= 5 and (w & 3) == 1:
                        B[f"x{(w - 5) >> 2}"].arrive()
                if li == nl:
                    continue
                if u == -1:
                    if not (yield from wait("w2", s)):
                        return
                    if m.w["wf"] != s:
                        raise Violation("epilogue reads biases of another layer")
                for t in (0, 1):
                    if not (yield from wait(f"m2{2 * t + (g2 & 1)}", g2 >> 1)):
                        return
                    if m.tm_c2[t] != g2:
                        raise Violation(f"drain of tile {t} finds {m.tm_c2[t]}, wants {g2}")
                    m.tm_c2[t] = None
                    B[f"t2{t}"].arrive()
                slot = (g2 + 2) % 3
                old = m.h2[(g2) % 3]
                if old is not None and m.pending_reads(lambda g: g["kind"] == "conv3" and g["h2"] == old):
                    raise Violation(f"h2 {g2} overwrites {old} still read by a queued batch")
                m.h2[g2 % 3] = g2
                B[f"h2{g2 % 3}"].arrive()
                yield

    def complete_one(qname):
        g = m.queues[qname].pop(0)
        if g["kind"] == "copy":
            if g["res"] == "W2":
                m.w["W2"] = g["ver"]
                m.w["wf"] = g["ver"]
            else:
                m.w[g["res"]] = g["ver"]
        else:
            m.pending.remove(g)
        B[g["commit"]].arrive()

    m.last_copy = {}                   # barrier -> completion its last issued copy brings
    for cfg in range(n_configs):
        if m.abort:
            break
        # the prior (all threads, then a CTA barrier)
        for z in range(L):
            for p in (0, 1):
                m.x[(z, p)] = ("prior", cfg)
        m.x_reads = {}
        agents = {"A": conv2_issuer(0, cfg), "Bt": conv2_issuer(1, cfg), "C": conv3_issuer(cfg),
                  "D": conv1_issuer(cfg), "W": workers(cfg), "E": epilogue(cfg)}
        steps = 0
        # each agent and queue runs at its own random speed in this configuration
        speed = {k: m.rng.choice([0.05, 0.3, 1.0, 3.0]) for k in list(agents) + list(m.queues)}
        while agents or any(m.queues.values()):
            choices = list(agents) + [q for q, v in m.queues.items() if v]
            k = m.rng.choices(choices, weights=[speed[c] for c in choices])[0]
            steps += 1
            if steps > 2_000_000:
                raise Violation(f"no progress: {waiting}")
            if k in agents:
                current[0] = k
                try:
                    next(agents[k])
                except StopIteration:
                    del agents[k]
            else:
                complete_one(k)
            if not agents and not any(m.queues.values()):
                break
            if m.abort and not agents:
                break                  # every role has left its loops; queued work may remain
            # deadlock: every live agent blocked and nothing queued
        if not m.abort:
            # the CTA barrier at the end of the configuration needs every queued MMA done
            assert not m.pending

    # teardown (after the loop over configurations, normal or aborted): the four
    # issuers commit to bar_fin and one thread waits for it, i.e. for every
    # tensor-core group they queued; the staging thread waits for the
    # completions its last W2 / W3 copies bring.  Meanwhile queued copies and MMAs
    # keep completing in any order.
    def drain(until):
        guard = 0
        while not until():
            live = [q for q, v in m.queues.items() if v]
            if not live:
                raise Violation("teardown waits for work that was never queued")
            complete_one(m.rng.choice(live))
            guard += 1
            if guard > 100_000:
                raise Violation("teardown does not finish")
    drain(lambda: not any(m.queues[q] for q in ("qA", "qB", "qC", "qD")))
    if mutation != "no_copy_drain":
        drain(lambda: all(B[b].done > n for b, n in m.last_copy.items()))
    # TMEM is freed and the CTA exits: nothing may still use either
    if m.pending:
        raise Violation("TMEM freed while tensor-core work is queued")
    if m.queues["copy"]:
        raise Violation("CTA exits while a bulk weight copy still writes shared memory")
    return m.status


@pytest.mark.parametrize("seed", range(24))
def test_protocol_random_schedules(seed):
    run(n_configs=2, n_layers=4, seed=seed)


@pytest.mark.parametrize("mutation", ["no_slot_wait", "no_t2_wait", "no_t3_wait", "w2_early",
                                      "no_batch_wait", "rot0"])
def test_model_catches_planted_mistakes(mutation):
    """Each planted mistake must break some schedule: the model is not vacuous."""
    for seed in range(40):
        try:
            run(n_configs=2, n_layers=3, seed=seed, mutation=mutation)
        except Violation:
            return
    raise AssertionError(f"{mutation} went unnoticed")


AGENTS = ["A", "Bt", "C", "D", "W", "E"]


@pytest.mark.parametrize("seed", range(24))
def test_abort_at_a_random_wait(seed):
    """A random role's wait runs out at a random point: every role leaves its
    loops, the status word says GF_ETIMEOUT, queued tensor-core work is done
    before TMEM is freed and no copy is in flight when the CTA exits."""
    rng = random.Random(1000 + seed)
    who, k = rng.choice(AGENTS), rng.randint(1, 400)
    st = run(n_configs=2, n_layers=3, seed=seed, abort_at=(who, k))
    # a wait that is never blocked from its k-th on cannot run out: then no abort
    assert st in (None, "GF_ETIMEOUT")


def test_abort_happens_in_most_draws():
    """The abort schedules are not vacuous: most draws do abort."""
    hits = 0
    for seed in range(30):
        rng = random.Random(5000 + seed)
        if run(n_configs=1, n_layers=3, seed=seed, abort_at=(rng.choice(AGENTS), rng.randint(1, 200))):
            hits += 1
    assert hits >= 15, hits


def test_missing_copy_drain_is_caught():
    """Without the staging thread's wait for its last copies, some abort leaves
    a bulk copy writing shared memory after the CTA exits."""
    for seed in range(200):
        rng = random.Random(9000 + seed)
        try:
            run(n_configs=1, n_layers=3, seed=seed, abort_at=(rng.choice(["A", "Bt", "C", "E"]), rng.randint(1, 3)),
                mutation="no_copy_drain")
        except Violation as e:
            assert "bulk weight copy" in str(e)
            return
    raise AssertionError("a copy in flight at exit went unnoticed")

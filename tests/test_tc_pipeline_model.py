"""CPU model check of the tensor-core transforms' producer schedule
(`tc_forward_range` / `tc_adjoint_range` in csrc/tc_kernels.cuh, and the
moment pass's copy of the forward schedule in csrc/tc_grad.cu).

The kernels run without a CTA barrier in their main loop: four warps each
read their TMEM lanes of a chunk's accumulator, count themselves on a
per-buffer shared counter, and go on to the arithmetic. The warp counted
last issues the MMAs up to two chunks ahead; the warp counted first refills
the operand rings (forward: B of chunk c + NBB and the nearfield of chunk
c + KF into an NF = KF + 3 slot ring; adjoint: B of chunk c + NB and A of
group s + 2). Correctness rests on how far apart the warps can drift, so
this test plays the schedule under random interleavings of warps, copy
completions and MMA completions and checks, at every step:

* no copy or MMA overwrites a ring slot or TMEM buffer whose contents are
  still needed (by an MMA in flight, a warp yet to read it, or an MMA yet
  to be issued that expects it);
* every read sees the chunk (or block, group) it expects;
* no interleaving deadlocks (some action is always enabled until every
  warp has finished its range).

The model follows the kernels' control flow step for step: the range's
chunk -> (block, pixel chunk) or (group, spot chunk) mapping, the issue
loop's block-change rule (a new spot block's A is reloaded only once every
MMA of the old block has been released by all warps), the waits the
kernels make and the order in which lane 0 acts on the arrival count.
"""
import random

import pytest

WARPS = 4


class Violation(AssertionError):
    pass


def check(cond, what):
    if not cond:
        raise Violation(what)


class Pipeline:
    """Shared pieces: asynchronous copies (land in any order) and MMAs
    (complete in issue order: one thread issues them and commits each)."""

    def __init__(self, rng, nc):
        self.rng = rng
        self.nc = nc
        self.copies = []            # pending (ring, slot, tag)
        self.mma_queue = []         # issued, not complete
        self.mma_done = [False] * nc
        self.tmem = [None, None]    # chunk whose MMA owns the buffer
        self.cnt = [0, 0]
        self.released = [-1] * WARPS   # last chunk each warp has read from TMEM
        self.finished = [-1] * WARPS   # last chunk each warp has finished
        self.rings = {}

    def ring(self, name, n):
        self.rings[name] = [(None, False)] * n

    def start_copy(self, name, slot, tag):
        self.rings[name][slot] = (tag, False)
        self.copies.append((name, slot, tag))

    def landed(self, name, slot, tag):
        t, ok = self.rings[name][slot]
        return t == tag and ok

    def holds(self, name, slot, tag):
        return self.rings[name][slot][0] == tag

    def all_released(self, c):
        return all(r >= c for r in self.released)

    def all_finished(self, c):
        return all(f >= c for f in self.finished)

    def issue_mma(self, k):
        # the TMEM buffer k & 1 was last written by MMA(k - 2): every warp
        # must have read it
        check(k < 2 or self.all_released(k - 2), f"MMA({k}) overwrites TMEM of chunk {k - 2} before all warps read it")
        self.tmem[k & 1] = k
        self.mma_queue.append(k)

    def async_actions(self):
        acts = []
        for i in range(len(self.copies)):
            acts.append(("copy", i))
        if self.mma_queue:
            acts.append(("mma", 0))
        return acts

    def run_async(self, act):
        kind, i = act
        if kind == "copy":
            name, slot, tag = self.copies.pop(i)
            check(self.rings[name][slot][0] == tag, f"{name} slot {slot} rewritten while its copy of {tag} was in flight")
            self.rings[name][slot] = (tag, True)
        else:
            k = self.mma_queue.pop(0)
            self.check_mma_operands(k)
            self.mma_done[k] = True


class ForwardModel(Pipeline):
    """tc_forward_range: spot blocks of nq pixel chunks; this range covers
    units u0 .. u0 + nc - 1 (unit u = block u // nq, pixel chunk u % nq)."""

    NBB, KF, NF = 4, 5, 8

    def __init__(self, rng, nc, nq, u0):
        super().__init__(rng, nc)
        self.nq, self.u0 = nq, u0
        self.ring("A", 1)
        self.ring("B", self.NBB)
        self.ring("F", self.NF)
        self.b0 = u0 // nq
        # producer state of the issuing thread: next MMA chunk, block in A, A unchecked
        self.k, self.ab, self.fresh = 0, self.b0, True
        self.start_copy("A", 0, self.b0)
        for c in range(min(self.NBB, nc)):
            self.start_copy("B", c % self.NBB, c)
        for c in range(min(self.KF, nc)):
            self.start_copy("F", c % self.NF, c)
        # warp 0's thread 0 runs issue_upto(1, -1) before the loop
        self.warps = [{"c": 0, "st": "wait_full"} for _ in range(WARPS)]
        self.warps[0] = {"c": 0, "st": "issue", "upto": 1, "rel": -1, "next": "wait_full", "sub": "top"}

    def block(self, c):
        return (self.u0 + c) // self.nq

    def check_mma_operands(self, k):
        check(self.landed("A", 0, self.block(k)), f"MMA({k}) ran with A of another block")
        check(self.landed("B", k % self.NBB, k), f"MMA({k}) ran with B of another chunk")

    def issue_step(self, w):
        """One step of issue_upto(upto, released); returns False if blocked."""
        s = self.warps[w]
        k = self.k
        if s["sub"] == "top":
            if k > s["upto"] or k >= self.nc:
                s["st"] = s["next"]
                return True
            b = self.block(k)
            if b != self.ab:
                if k - 1 > s["rel"]:
                    s["st"] = s["next"]          # an MMA of the old block may still run
                    return True
                check(k == 0 or self.mma_done[k - 1], f"A reloaded for block {b} while MMA({k - 1}) runs")
                self.start_copy("A", 0, b)
                self.ab, self.fresh = b, True
            s["sub"] = "wait_b"
            return True
        if s["sub"] == "wait_b":
            if not self.landed("B", k % self.NBB, k):
                return False
            s["sub"] = "wait_a" if self.fresh else "mma"
            return True
        if s["sub"] == "wait_a":
            if not self.landed("A", 0, self.block(k)):
                return False
            self.fresh = False
            s["sub"] = "mma"
            return True
        self.issue_mma(k)
        self.k += 1
        s["sub"] = "top"
        return True

    def warp_step(self, w):
        s = self.warps[w]
        c = s["c"]
        st = s["st"]
        if st == "done":
            return False
        if st == "issue":
            return self.issue_step(w)
        if st == "wait_full":
            if c >= self.nc:
                s["st"] = "done"
                return True
            if not self.mma_done[c]:
                return False
            check(self.tmem[c & 1] == c, f"TMEM buffer {c & 1} holds chunk {self.tmem[c & 1]}, warp expects {c}")
            s["st"] = "arrive"
            self.released[w] = c
            return True
        if st == "arrive":
            order = self.cnt[c & 1] % WARPS
            self.cnt[c & 1] += 1
            if order == WARPS - 1:
                s.update(st="issue", upto=c + 2, rel=c, next="wait_f", sub="top")
            elif order == 0:
                s["st"] = "load_b"
            else:
                s["st"] = "wait_f"
            return True
        if st == "load_b":
            if c + self.NBB < self.nc:
                slot = (c + self.NBB) % self.NBB
                check(self.mma_done[c], f"B slot {slot} reloaded while MMA({c}) may read it")
                self.start_copy("B", slot, c + self.NBB)
            s["st"] = "load_f"
            return True
        if st == "load_f":
            if c + self.KF < self.nc:
                slot = (c + self.KF) % self.NF
                prev = c + self.KF - self.NF
                check(prev < 0 or self.all_finished(prev), f"f slot {slot} reloaded while a warp still needs chunk {prev}")
                self.start_copy("F", slot, c + self.KF)
            s["st"] = "wait_f"
            return True
        if st == "wait_f":
            if not self.landed("F", c % self.NF, c):
                return False
            s["st"] = "compute"
            return True
        if st == "compute":
            check(self.landed("F", c % self.NF, c), f"f slot of chunk {c} rewritten during its use")
            self.finished[w] = c
            s["c"] = c + 1
            s["st"] = "wait_full"
            return True
        raise AssertionError(st)

    def done(self):
        return all(s["st"] == "done" for s in self.warps)


class AdjointModel(Pipeline):
    """tc_adjoint_range: pixel groups of nch spot chunks; this range covers
    units u0 .. u0 + nc - 1 (unit u = group u // nch, spot chunk u % nch)."""

    NB = 2

    def __init__(self, rng, nc, nch, u0):
        super().__init__(rng, nc)
        self.nch, self.u0 = nch, u0
        self.s0 = u0 // nch
        self.s_last = (u0 + nc - 1) // nch
        self.ring("A", 2)
        self.ring("B", self.NB)
        self.start_copy("A", 0, self.s0)
        if self.s0 + 1 <= self.s_last:
            self.start_copy("A", 1, self.s0 + 1)
        for c in range(min(self.NB, nc)):
            self.start_copy("B", c % self.NB, c)
        self.k = 0
        self.warps = [{"c": 0, "st": "wait_full"} for _ in range(WARPS)]
        self.warps[0] = {"c": 0, "st": "issue", "upto": 1, "next": "wait_full", "sub": "top"}

    def group(self, c):
        return (self.u0 + c) // self.nch

    def spot_chunk(self, c):
        return (self.u0 + c) % self.nch

    def a_slot(self, s):
        return (s - self.s0) & 1

    def check_mma_operands(self, k):
        s = self.group(k)
        check(self.landed("A", self.a_slot(s), s), f"MMA({k}) ran with A of another group")
        check(self.landed("B", k % self.NB, k), f"MMA({k}) ran with B of another chunk")

    def issue_step(self, w):
        s = self.warps[w]
        k = self.k
        if s["sub"] == "top":
            if k > s["upto"] or k >= self.nc:
                s["st"] = s["next"]
                return True
            s["sub"] = "wait_b"
            return True
        if s["sub"] == "wait_b":
            if not self.landed("B", k % self.NB, k):
                return False
            s["sub"] = "wait_a" if (k == 0 or self.spot_chunk(k) == 0) else "mma"
            return True
        if s["sub"] == "wait_a":
            g = self.group(k)
            if not self.landed("A", self.a_slot(g), g):
                return False
            s["sub"] = "mma"
            return True
        self.issue_mma(k)
        self.k += 1
        s["sub"] = "top"
        return True

    def warp_step(self, w):
        s = self.warps[w]
        c = s["c"]
        st = s["st"]
        if st == "done":
            return False
        if st == "issue":
            return self.issue_step(w)
        if st == "wait_full":
            if c >= self.nc:
                s["st"] = "done"
                return True
            if not self.mma_done[c]:
                return False
            check(self.tmem[c & 1] == c, f"TMEM buffer {c & 1} holds chunk {self.tmem[c & 1]}, warp expects {c}")
            self.released[w] = c
            s["st"] = "arrive"
            return True
        if st == "arrive":
            order = self.cnt[c & 1] % WARPS
            self.cnt[c & 1] += 1
            if order == WARPS - 1:
                s.update(st="issue", upto=c + 2, next="compute", sub="top")
            elif order == 0:
                s["st"] = "loads"
            else:
                s["st"] = "compute"
            return True
        if st == "loads":
            g = self.group(c)
            last_of_group = self.spot_chunk(c) == self.nch - 1 or c == self.nc - 1
            if c + self.NB < self.nc:
                check(self.mma_done[c], f"B slot {c % self.NB} reloaded while MMA({c}) may read it")
                self.start_copy("B", (c + self.NB) % self.NB, c + self.NB)
            if last_of_group and g + 2 <= self.s_last:
                # every MMA of group g is complete (they end with MMA(c))
                check(self.mma_done[c] and all(not (self.group(k) == g) for k in self.mma_queue),
                      f"A slot of group {g} reloaded while its MMAs may run")
                self.start_copy("A", self.a_slot(g), g + 2)
            s["st"] = "compute"
            return True
        if st == "compute":
            self.finished[w] = c
            s["c"] = c + 1
            s["st"] = "wait_full"
            return True
        raise AssertionError(st)

    def done(self):
        return all(s["st"] == "done" for s in self.warps)


def play(model, rng, max_steps=200000):
    for _ in range(max_steps):
        if model.done() and not model.mma_queue:
            return
        acts = [("warp", w) for w in range(WARPS)] + model.async_actions()
        rng.shuffle(acts)
        progressed = False
        for a in acts:
            if a[0] == "warp":
                if model.warp_step(a[1]):
                    progressed = True
                    break
            else:
                model.run_async(a)
                progressed = True
                break
        check(progressed, "deadlock: no warp, copy or MMA can proceed")
    raise AssertionError("no termination within the step bound")


def _cases(seed0, n):
    rng = random.Random(seed0)
    for i in range(n):
        yield rng.randrange(1 << 30), rng.randint(1, 40), rng.randint(1, 9), rng.randint(0, 30)


@pytest.mark.parametrize("seed,nc,per,u0", list(_cases(11, 150)))
def test_forward_schedule(seed, nc, per, u0):
    rng = random.Random(seed)
    play(ForwardModel(rng, nc, per, u0), rng)


@pytest.mark.parametrize("seed,nc,per,u0", list(_cases(12, 150)))
def test_adjoint_schedule(seed, nc, per, u0):
    rng = random.Random(seed)
    play(AdjointModel(rng, nc, per, u0), rng)


# Planted mistakes: each must be caught on some interleaving.

class ForwardRingTooSmall(ForwardModel):
    NF = ForwardModel.KF + 2     # the nearfield ring one slot short of the drift bound


class ForwardThreeAhead(ForwardModel):
    def warp_step(self, w):
        s = self.warps[w]
        if s["st"] == "arrive" and self.cnt[s["c"] & 1] % WARPS == WARPS - 1:
            c = s["c"]
            self.cnt[c & 1] += 1
            s.update(st="issue", upto=c + 3, rel=c, next="wait_f", sub="top")
            return True
        return super().warp_step(w)


class AdjointEarlyA(AdjointModel):
    def warp_step(self, w):
        # A of group s + 2 loaded at the first arrival of s's second-to-last chunk
        s = self.warps[w]
        if s["st"] == "loads":
            c = s["c"]
            g = self.group(c)
            if self.spot_chunk(c) == self.nch - 2 and g + 2 <= self.s_last:
                self.start_copy("A", self.a_slot(g), g + 2)
        return super().warp_step(w)


def _caught(cls, per_range):
    for seed, nc, _per, u0 in _cases(99, 400):
        rng = random.Random(seed)
        try:
            play(cls(rng, max(nc, 8), per_range, u0), rng)
        except Violation:
            return True
    return False


@pytest.mark.parametrize("cls,per", [(ForwardRingTooSmall, 5), (ForwardThreeAhead, 5), (AdjointEarlyA, 3)])
def test_planted_schedule_mistakes_are_caught(cls, per):
    assert _caught(cls, per)


# SM-aware range claiming of the forward (tc_claim_range): G CTAs claim G
# ranges, [0, n_full) of the full spot blocks and one per SM of the
# replicated last block. Every range must be run exactly once whatever the
# placement; with per_sm CTAs on every SM, each SM runs exactly one
# replicated range.

def claim_ranges(placement, n_full, G, order):
    """placement[c] = SM of CTA c; order: the order in which CTAs claim."""
    per_sm_ctr, pools = {}, [0, 0]
    n_rep = G - n_full
    per_sm = G // n_rep if n_rep > 0 else 1
    got = {}
    for c in order:
        sm = placement[c]
        slot = per_sm_ctr.get(sm, 0)
        per_sm_ctr[sm] = slot + 1
        rep_first = slot % per_sm == per_sm - 1
        got[c] = -1
        for pas in range(2):
            rep = (pas == 0) == rep_first
            k = pools[1 if rep else 0]
            pools[1 if rep else 0] += 1
            if k < (n_rep if rep else n_full):
                got[c] = n_full + k if rep else k
                break
    return got


@pytest.mark.parametrize("seed", range(40))
def test_claimed_ranges_cover_every_range_once(seed):
    rng = random.Random(seed)
    sms, per_sm = rng.choice([(152, 4), (148, 4), (20, 2), (7, 3)])
    G = sms * per_sm
    n_full = G - sms
    if seed % 2:
        placement = [c // per_sm for c in range(G)]            # per_sm CTAs on every SM
        rng.shuffle(placement)
    else:
        placement = [rng.randrange(sms) for _ in range(G)]     # uneven placement
    order = list(range(G))
    rng.shuffle(order)
    got = claim_ranges(placement, n_full, G, order)
    assert sorted(got.values()) == list(range(G))
    if seed % 2:
        rep_per_sm = {}
        for c, r in got.items():
            if r >= n_full:
                rep_per_sm[placement[c]] = rep_per_sm.get(placement[c], 0) + 1
        assert sorted(rep_per_sm.values()) == [1] * sms

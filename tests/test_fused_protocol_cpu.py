"""The step protocol of the multi-step fused kernel (steps_fused_advdiff in
csrc/at_fused.cu), modelled on the CPU.

C CTAs on a ring (periodic domain).  Before step n (not the first of the
launch) CTA c waits until its two neighbour CTAs have published level n (they
finished step n-1).  During step n it reads, from the start of the step until
it publishes: the u^n of itself and of both neighbours (the strips) in buffer
i % 2 (i = n - level0), and ring slots of the neighbours' and its own edge
windows at levels n-d, 1 <= d <= k_max + q, every stage.  It writes ring slots
of level n (stages 1..S-1) stage by stage, then u^{n+1} into buffer (i+1) % 2
and ring level n+1 stage 0, then publishes n+1.  The ring has R = k_max + q +
3 levels per (PE, stage): slot L mod R.

The model runs those events under random interleavings and checks that every
run ends (no deadlock), that every read finds the version it needs and keeps
it until the reader publishes (no write lands on a location a CTA inside its
step still reads), and that neighbours are never more than one step apart.
A weakened wait rule must fail it.  It models the kernel's protocol, written
out by hand: a change to one needs the same change to the other."""
import random

import pytest


def simulate(C, K, S, kq, level0, seed, wait_rule="both", withheld=None, spare=2, max_events=200000):
    """Returns (finished: bool, violations: list of str)."""
    rng = random.Random(seed)
    R = kq + 1 + spare
    # buffer versions: buf[b][c] = level held by CTA c's region of buffer b
    buf = [[level0] * C, [None] * C]
    # ring versions: ring[(c, slot, s)] = level held; the state before the
    # launch: stage 0 holds levels <= level0, stages >= 1 levels <= level0 - 1
    ring = {}
    for c in range(C):
        for s in range(S):
            top = level0 if s == 0 else level0 - 1
            for L in range(top - R + 1, top + 1):
                ring[(c, L % R, s)] = L
    done = [level0] * C
    step = [0] * C          # steps finished within the launch
    phase = [None] * C      # None: before the step's wait; else index into its event list
    reading = [None] * C    # read set of a CTA inside its step
    viol = []

    def nbrs(c):
        return (c - 1) % C, (c + 1) % C

    def events(c):
        n = level0 + step[c]
        ev = [("read",)]
        for s in range(1, S):
            ev.append(("wring", n % R, s, n))
        ev.append(("wbuf", (step[c] + 1) % 2, n + 1))
        ev.append(("wring", (n + 1) % R, 0, n + 1))
        ev.append(("publish", n + 1))
        return ev

    def read_set(c):
        n = level0 + step[c]
        b = step[c] % 2
        rs = []
        for x in {c, *nbrs(c)}:
            rs.append(("buf", b, x, n))
            for s in range(S):
                for d in range(1, kq + 1):
                    if n - d >= 0:
                        rs.append(("ring", (x, (n - d) % R, s), n - d))
        return rs

    def can_start(c):
        if step[c] == 0:
            return True
        n = level0 + step[c]
        cl, cr = nbrs(c)
        if wait_rule == "both":
            return done[cl] >= n and done[cr] >= n
        if wait_rule == "left":
            return done[cl] >= n
        if wait_rule == "one_behind":
            return done[cl] >= n - 1 and done[cr] >= n - 1
        raise ValueError(wait_rule)

    evs = [None] * C
    for _ in range(max_events):
        if all(step[c] == K for c in range(C)):
            return True, viol
        runnable = []
        for c in range(C):
            if step[c] == K:
                continue
            if phase[c] is None:
                if can_start(c):
                    runnable.append(c)
            else:
                runnable.append(c)
        if not runnable:
            return False, viol
        c = rng.choice(runnable)
        if phase[c] is None:
            evs[c] = events(c)
            phase[c] = 0
            continue
        e = evs[c][phase[c]]
        phase[c] += 1
        n = level0 + step[c]
        if e[0] == "read":
            reading[c] = read_set(c)
            for r in reading[c]:
                have = buf[r[1]][r[2]] if r[0] == "buf" else ring.get(r[1])
                if have != r[-1]:
                    viol.append("CTA %d step %d reads %s: holds %s" % (c, n, r[:-1], have))
        elif e[0] in ("wring", "wbuf"):
            loc = ("ring", (c, e[1], e[2])) if e[0] == "wring" else ("buf", e[1], c)
            for o in range(C):
                if reading[o] is None:
                    continue
                for r in reading[o]:
                    key = ("ring", r[1]) if r[0] == "ring" else ("buf", r[1], r[2])
                    if key == loc:
                        viol.append("CTA %d step %d overwrites %s while CTA %d reads it" % (c, n, loc, o))
            if e[0] == "wring":
                ring[(c, e[1], e[2])] = e[3]
            else:
                buf[e[1]][c] = e[2]
        elif e[0] == "publish":
            reading[c] = None
            if c != withheld:
                done[c] = e[1]
            step[c] += 1
            phase[c] = None
            for o in nbrs(c):
                if abs(step[o] - step[c]) > 1 and o != c and withheld is None:
                    viol.append("CTAs %d and %d are %d steps apart" % (c, o, abs(step[o] - step[c])))
    return False, viol + ["event limit"]


@pytest.mark.parametrize("C", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("S,kq", [(4, 5), (3, 2), (2, 1), (4, 2)])
def test_fused_protocol_completes_without_hazards(C, S, kq):
    for seed in range(60):
        level0 = (seed * 7) % 11
        ok, viol = simulate(C, 6, S, kq, level0, seed)
        assert ok, (C, S, kq, seed)
        assert not viol, viol[:3]


def test_withheld_cta_blocks_its_neighbours():
    """A CTA that never publishes leaves its neighbours waiting (in the kernel
    the bounded waits then run out and raise the abort flag)."""
    ok, viol = simulate(5, 6, 4, 5, 3, seed=1, withheld=2)
    assert not ok and not viol


@pytest.mark.parametrize("rule", ["left", "one_behind"])
def test_weaker_wait_rules_are_caught(rule):
    """Waiting for one neighbour only, or for the step before last, lets a CTA
    read a strip that is not there yet or overwrite one still being read."""
    found = False
    for seed in range(200):
        ok, viol = simulate(4, 6, 4, 5, 2, seed, wait_rule=rule)
        if viol:
            found = True
            break
    assert found


def test_ring_without_spare_levels_is_caught():
    """With R = k_max + q + 1 a step's write of level n+1 lands on the slot of
    level n - k_max - q that a neighbour at the same step still reads."""
    found = any(simulate(3, 6, 4, 5, 6, seed, spare=0)[1] for seed in range(200))
    assert found

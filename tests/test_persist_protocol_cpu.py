"""The named-barrier protocol of the persistent kernel (csrc/at_persist.cu),
modelled on the CPU.  The halo warp runs one stage ahead of the worker
warps; stage t of parity p uses barrier 1 + p (halo ready: the halo warp
arrives, the workers sync), 3 + p (the workers are done with G[p]: they
arrive after stage t when t + 2 < T, the halo warp syncs before filling G[p]
for stage t + 2) and 5 (workers only).  A failed neighbour wait at stage t_a
makes the halo warp record t_a, arrive, consume the workers' last pending
arrival and stop; the workers stop at t_a.  The model replays exactly that
sequence of barrier operations under random interleavings of the two
groups and checks that every run ends with no deadlock, no barrier taking
more arrivals than its count in one phase, and no arrivals left over.  It
models the kernel's control flow, written out by hand: a change to one
needs the same change to the other."""
import random

import pytest

COUNT = {0: 288, 1: 288, 2: 288, 3: 288, 4: 288, 5: 256}   # 8 worker warps + 1 halo warp


def programs(T, abort_at):
    halo, work = [], []
    for t in range(T):
        p = t & 1
        if t >= 2:
            halo.append(("sync", 3 + p, 32))
        if t == abort_at:
            halo.append(("set_abort", t))
        halo.append(("arrive", 1 + p, 32))
        if t == abort_at:
            if t >= 1 and t + 1 < T:
                halo.append(("sync", 3 + ((t - 1) & 1), 32))
            break
    halo.append(("sync", 0, 32))
    for t in range(T):
        p = t & 1
        work.append(("sync", 1 + p, 256))
        work.append(("check_abort", t))
        work.append(("sync", 5, 256))
        if t + 2 < T:
            work.append(("arrive", 3 + p, 256))
    work.append(("sync", 0, 256))
    return halo, work


def run(T, abort_at, seed, make=programs):
    rng = random.Random(seed)
    progs = dict(zip(("h", "w"), make(T, abort_at)))
    pc = {"h": 0, "w": 0}
    waiting, done = {}, set()
    arrived = {b: 0 for b in COUNT}
    gen = {b: 0 for b in COUNT}
    abort = None
    for _ in range(100000):
        if len(done) == 2:
            break
        for a, (b, g) in list(waiting.items()):
            if gen[b] > g:
                del waiting[a]
                if pc[a] == len(progs[a]):
                    done.add(a)
        if len(done) == 2:
            break
        ready = [a for a in ("h", "w") if a not in done and a not in waiting]
        if not ready:
            return "deadlock"
        a = rng.choice(ready)
        prog = progs[a]
        op = prog[pc[a]]
        pc[a] += 1
        if op[0] == "set_abort":
            abort = op[1]
        elif op[0] == "check_abort":
            if abort is not None and op[1] >= abort:
                pc[a] = len(prog) - 1          # leave the loop: only the final barrier remains
        else:
            b, c = op[1], op[2]
            arrived[b] += c
            if arrived[b] > COUNT[b]:
                return "overflow on barrier %d" % b
            if arrived[b] == COUNT[b]:
                arrived[b] = 0
                gen[b] += 1
            elif op[0] == "sync":
                waiting[a] = (b, gen[b])
        if pc[a] == len(prog) and a not in waiting:
            done.add(a)
    else:
        return "no progress"
    if any(arrived.values()):
        return "arrivals left over %s" % arrived
    return "ok"


@pytest.mark.parametrize("T", range(1, 10))
def test_barrier_protocol_completes_for_every_abort_stage(T):
    for abort_at in [None] + list(range(T)):
        for seed in range(100):
            assert run(T, abort_at, seed) == "ok", (T, abort_at, seed)


def test_model_detects_a_broken_protocol():
    """The same model flags the protocol without the per-stage abort check
    (workers stopping at any recorded abort): the halo warp runs ahead, so
    its arrival for the failed stage may never be consumed."""
    def broken(T, abort_at):
        halo, work = programs(T, abort_at)
        return halo, [("check_abort", 10 ** 9) if op[0] == "check_abort" else op for op in work]
    results = {run(3, 2, seed, broken) for seed in range(200)}
    assert any(r != "ok" for r in results)

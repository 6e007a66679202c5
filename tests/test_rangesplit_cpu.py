"""One domain split over CPU ranks by PE ranges (gloo, no GPU).

Each rank steps its contiguous PE range with the oracle (a window problem
with global PE indices in the delay counter and open outer ends) and trades
the edge windows of every stage argument with its neighbours through gloo
point-to-point messages, under the Philox delays.  The gathered state must
equal, bit for bit, the one-process oracle run of the whole domain: with two
ranks (each rank both neighbours of the other), three ranks (distinct
neighbours, uneven ranges), for central (AT6 + RK4, reacting flow) and WENO
(AT-WENO5 + RK3-TVD, detonation) schemes, and with windows held back on the
host for several stages.  A window that is lost while a neighbour's delay
needs it makes that neighbour stop with AT_ETIMEOUT within its wait limit.
"""
import os
import socket

import numpy as np
import pytest

from paper_2204_01133_gb300 import rangesplit as RS


def test_pe_ranges_cover_and_balance():
    for P, world in ((24, 2), (16, 3), (7, 7), (1000, 6)):
        rs = RS.pe_ranges(P, world)
        assert rs[0][0] == 0 and rs[-1][1] == P
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        sizes = [hi - lo for lo, hi in rs]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        RS.pe_ranges(3, 4)


def test_levels_read_follow_the_nonzero_weights():
    import oracle
    for q in (1, 2, 3):
        for k in range(5):
            w = oracle.lagrange_weights(q, k)
            want = [10 - k - l for l in range(q + 1) if w[l] != 0.0]
            assert RS.levels_read("at", q, 10, k) == want
    assert RS.levels_read("as", 2, 10, 3) == [7]
    assert RS.levels_read("sync", 2, 10, 3) == [10]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem(name):
    from paper_2204_01133_gb300 import workloads as W
    if name == "rns":
        pb, u0 = W.rns(case="flame", n=1536, pe_size=64, mode="at", k_max=4, seed=5, dt=0.003)
        return pb, u0, 30
    if name == "rns-as":
        pb, u0 = W.rns(case="ignition", n=1024, pe_size=32, order=4, mode="as", k_max=3, seed=6, dt=0.003)
        return pb, u0, 25
    if name == "detonation":
        pb, u0 = W.detonation(n=4096, pe_size=256, mode="at", k_max=4, seed=7)
        return pb, u0, 20
    pb, u0 = W.advdiff(n=1024, pe_size=32, mode="at", k_max=3, seed=8, cfl=0.05)
    return pb, u0, 40


def _worker(rank, world, port, name, hold, wait_limit, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2204_01133_gb300 import api
    oracle.set_threads(1)
    pb, u0, steps = _problem(name)
    P, B = pb["n"] // pb["pe_size"], pb["pe_size"]
    lo, hi = RS.pe_ranges(P, world)[rank]
    sub = dict(pb, n=(hi - lo) * B, pe_base=lo, pe_total=P, open_ends=1)
    eng = oracle.Oracle(sub, u0[:, lo * B:hi * B])
    qq = 1 if pb["pde"] == "euler" else pb["order"] // 2
    rr = RS.RangeRank(eng, rank, world, pb["mode"], qq, pb["k_max"], wait_limit=wait_limit,
                      hold=hold.get(rank, {}))
    code, msg = 0, ""
    try:
        rr.run(steps)
    except api.AtError as e:
        code, msg = e.code, str(e)
    rr.drain()
    out = (rank, code, msg, eng.state() if code == 0 else None, eng.delays() if code == 0 else None, lo, hi,
           rr.waits)
    gathered = [None] * world
    dist.all_gather_object(gathered, out)
    if rank == 0:
        q.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def _launch(name, world, hold=None, wait_limit=20.0):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, hold or {}, wait_limit, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return sorted(res, key=lambda r: r[0])


def _one_process(name):
    import oracle
    pb, u0, steps = _problem(name)
    o = oracle.Oracle(pb, u0)
    assert o.run(steps) == 0
    return pb, o.state(), o.delays()


@pytest.mark.parametrize("name,world", [("rns", 2), ("rns", 3), ("detonation", 2), ("rns-as", 3),
                                        ("advdiff", 4)])
def test_split_run_equals_one_process_bitwise(name, world):
    res = _launch(name, world)
    pb, ref, ref_d = _one_process(name)
    B = pb["pe_size"]
    for rank, code, msg, st, dl, lo, hi, _ in res:
        assert code == 0, msg
        assert np.array_equal(st, ref[:, lo * B:hi * B]), (rank, np.abs(st - ref[:, lo * B:hi * B]).max())
        assert np.array_equal(dl, ref_d[:, lo:hi, :]), rank


def test_windows_held_back_within_the_delays_change_nothing():
    """Windows held back on the host for 3 to 6 stages (longer than a step
    of 4 stages).  Three of them are read at delay 0 by the receiving rank at
    the very stage they were held back at, so it cannot go on before they
    arrive; two more are read later from the kept versions, at larger
    delays.  The result is still the one-process run bit for bit."""
    pb, _, _ = _problem("rns")
    P = pb["n"] // pb["pe_size"]
    lo1 = RS.pe_ranges(P, 2)[1][0]
    a = _zero_delay_stage("rns", lo1, RS.LEFT, start=3)      # rank 1's first PE reads rank 0's right edge
    b = _zero_delay_stage("rns", P - 1, RS.RIGHT, start=8)   # rank 1's last PE reads rank 0's left edge
    c = _zero_delay_stage("rns", 0, RS.LEFT, start=5)        # rank 0's first PE reads rank 1's right edge
    hold = {0: {a + (RS.RIGHT,): 3, b + (RS.LEFT,): 6, (12, 2, RS.RIGHT): 4, (20, 1, RS.LEFT): 5},
            1: {c + (RS.RIGHT,): 4}}
    res = _launch("rns", 2, hold=hold)
    pb, ref, _ = _one_process("rns")
    B = pb["pe_size"]
    for rank, code, msg, st, _, lo, hi, waits in res:
        assert code == 0, msg
        assert np.array_equal(st, ref[:, lo * B:hi * B]), rank
        print("rank %d waited at %d stages" % (rank, waits))


def _zero_delay_stage(name, rank_pe, side, start=6):
    """A (level, stage) at which global PE `rank_pe` draws delay 0 on `side`."""
    import oracle
    pb, u0, steps = _problem(name)
    o = oracle.Oracle(pb, u0)
    for n in range(start, steps):
        for s in range(o.stages):
            if o.delay(n, s, rank_pe, side) == 0:
                return n, s
    raise AssertionError("no zero delay found")


def test_lost_window_stops_the_neighbour_with_a_timeout():
    """Rank 0 never sends (until the drain) the right edge window of a stage
    at which rank 1's first PE draws delay 0 on its left side: rank 1 must
    stop with AT_ETIMEOUT, and every rank must still leave cleanly."""
    from paper_2204_01133_gb300 import api
    pb, _, _ = _problem("advdiff")
    P = pb["n"] // pb["pe_size"]
    lo1 = RS.pe_ranges(P, 2)[1][0]
    n0, s0 = _zero_delay_stage("advdiff", lo1, RS.LEFT)
    res = _launch("advdiff", 2, hold={0: {(n0, s0, RS.RIGHT): None}}, wait_limit=0.5)
    code1, msg1 = res[1][1], res[1][2]
    assert code1 == api.AT_ETIMEOUT, msg1
    assert "(%d, %d, 0)" % (n0, s0) in msg1

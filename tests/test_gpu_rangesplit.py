"""One domain split over ranks by PE ranges, each rank a library context on
the GPU (AT_OPT_OPEN_ENDS, global PE indices), exchanging the edge windows of
every stage argument through gloo point-to-point messages between stages
(paper_2204_01133_gb300.rangesplit).  The ranks are processes on the one GPU
of the box; none of their kernels waits on another rank (every wait is on
the host, with a time limit).  The gathered state and delay logs must equal,
bit for bit, one context running the whole domain on the per-stage path,
also with windows held back on the host; a lost window that a zero delay
needs stops the neighbour with AT_ETIMEOUT."""
import os
import socket

import numpy as np
import pytest

from paper_2204_01133_gb300 import rangesplit as RS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2204_01133_gb300 import build
    build.build()


def _problem(name):
    from paper_2204_01133_gb300 import workloads as W
    if name == "rns":
        pb, u0 = W.rns(case="flame", n=1536, pe_size=64, mode="at", k_max=4, seed=5, dt=0.003)
        return pb, u0, 30
    if name == "detonation":
        pb, u0 = W.detonation(n=4096, pe_size=256, mode="at", k_max=4, seed=7)
        return pb, u0, 20
    pb, u0 = W.advdiff(n=1024, pe_size=32, mode="at", k_max=3, seed=8, cfl=0.05)
    return pb, u0, 40


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, name, hold, wait_limit, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2204_01133_gb300 import api
    pb, u0, steps = _problem(name)
    P, B = pb["n"] // pb["pe_size"], pb["pe_size"]
    lo, hi = RS.pe_ranges(P, world)[rank]
    sub = dict(pb, n=(hi - lo) * B, pe_base=lo, pe_total=P, open_ends=1)
    solver = api.Solver(sub, u0[:, lo * B:hi * B], path="stage")
    q_ = 1 if pb["pde"] == "euler" else pb["order"] // 2
    rr = RS.RangeRank(RS.ContextEngine(solver), rank, world, pb["mode"], q_, pb["k_max"], wait_limit=wait_limit,
                      hold=hold.get(rank, {}))
    code, msg = 0, ""
    try:
        rr.run(steps)
    except api.AtError as e:
        code, msg = e.code, str(e)
    rr.drain()
    out = (rank, code, msg, solver.read_state() if code == 0 else None,
           solver.read_delays() if code == 0 else None, lo, hi)
    gathered = [None] * world
    dist.all_gather_object(gathered, out)
    if rank == 0:
        q.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def _launch(name, world, hold=None, wait_limit=30.0):
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


def _one_context(name):
    from paper_2204_01133_gb300.api import Solver
    pb, u0, steps = _problem(name)
    s = Solver(pb, u0, path="stage")
    s.run(steps)
    return pb, s.read_state(), s.read_delays()


@pytest.mark.parametrize("name,world", [("rns", 2), ("rns", 3), ("detonation", 2), ("advdiff", 3)])
def test_split_on_gpu_contexts_equals_one_context_bitwise(name, world):
    res = _launch(name, world)
    pb, ref, ref_d = _one_context(name)
    B = pb["pe_size"]
    for rank, code, msg, st, dl, lo, hi in res:
        assert code == 0, msg
        assert np.array_equal(st, ref[:, lo * B:hi * B]), (rank, np.abs(st - ref[:, lo * B:hi * B]).max())
        assert np.array_equal(dl, ref_d[:, lo:hi, :]), rank


def _zero_delay_stage(name, pe, side, start):
    import oracle
    pb, u0, steps = _problem(name)
    o = oracle.Oracle(pb, u0)
    for n in range(start, steps):
        for s in range(o.stages):
            if o.delay(n, s, pe, side) == 0:
                return n, s
    raise AssertionError("no zero delay found")


def test_held_back_windows_change_nothing_and_a_lost_one_times_out():
    from paper_2204_01133_gb300 import api
    pb, _, _ = _problem("rns")
    P = pb["n"] // pb["pe_size"]
    lo1 = RS.pe_ranges(P, 2)[1][0]
    a = _zero_delay_stage("rns", lo1, RS.LEFT, 3)
    b = _zero_delay_stage("rns", 0, RS.LEFT, 5)
    res = _launch("rns", 2, hold={0: {a + (RS.RIGHT,): 3, (12, 2, RS.LEFT): 5}, 1: {b + (RS.RIGHT,): 4}})
    pb, ref, _ = _one_context("rns")
    B = pb["pe_size"]
    for rank, code, msg, st, _, lo, hi in res:
        assert code == 0, msg
        assert np.array_equal(st, ref[:, lo * B:hi * B]), rank
    res = _launch("rns", 2, hold={0: {a + (RS.RIGHT,): None}}, wait_limit=1.0)
    assert res[1][1] == api.AT_ETIMEOUT, res[1][2]

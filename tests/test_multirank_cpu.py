"""The N > 1 path on CPU: two gloo ranks share a batch of independent
instances by the LPT partition, each solves its share (through the oracle,
no GPU), and the gathered results equal one process solving everything;
the timing reduction takes the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

from paper_2204_01133_gb300 import shard


def test_lpt_partition_covers_and_balances():
    rng = np.random.default_rng(0)
    costs = rng.integers(1, 1000, size=257).tolist()
    for world in (1, 2, 3, 8):
        parts = shard.lpt_partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)  # LPT bound
    with pytest.raises(ValueError):
        shard.lpt_partition(costs, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _instances():
    from paper_2204_01133_gb300 import workloads as W
    out = []
    for i, (n, B) in enumerate([(256, 16), (512, 32), (192, 16), (768, 64), (320, 16)]):
        pb, init = W.advdiff(n=n, pe_size=B, mode="at", k_max=3, seed=11 + i, cfl=0.05)
        out.append((dict(pb, instance=i), init, 30 + 5 * i))
    return out


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    inst = _instances()
    parts = shard.lpt_partition([pb["n"] * n for pb, _, n in inst], world)
    mine = {}
    for i in parts[rank]:
        pb, init, n = inst[i]
        o = oracle.Oracle(pb, init)
        assert o.run(n) == 0
        mine[i] = o.state()
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = shard.max_over_ranks(float(rank + 1) * 0.5)
    if rank == 0:
        res = {}
        for g in gathered:
            res.update(g)
        q.put((res, t, parts))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_solve_their_shares():
    import torch.multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res, t, parts = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == 1.0                          # max over ranks of 0.5 and 1.0
    assert all(len(p) > 0 for p in parts)    # both ranks got work
    inst = _instances()
    assert sorted(res) == list(range(len(inst)))
    for i, (pb, init, n) in enumerate(inst):
        o = oracle.Oracle(pb, init)
        assert o.run(n) == 0
        assert np.array_equal(res[i], o.state())

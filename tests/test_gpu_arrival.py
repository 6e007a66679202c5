"""Delays by arrival (real asynchrony on the persistent path) and the delay
trace.  With AT_OPT_ARRIVAL each PE boundary uses the freshest neighbour
stage argument that has arrived, so runs depend on timing; the trace records
every delay used, and the oracle replaying that trace must reproduce the GPU
result within the run tolerance.  In Philox mode the trace must equal the
oracle's draws bit for bit, on both paths."""
import numpy as np
import pytest

import oracle
from paper_2204_01133_gb300 import workloads as W

pytestmark = pytest.mark.gpu

from parity import TOL_RUN, check


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2204_01133_gb300 import build
    build.build()


def _oracle_delays(pb, u0, steps):
    o = oracle.Oracle(pb, u0)
    out = []
    for _ in range(steps):
        assert o.run(1) == 0
        out.append(o.delays())
    return np.stack(out)


@pytest.mark.parametrize("path", ["stage", "persistent"])
@pytest.mark.parametrize("maker", ["rns", "advdiff", "detonation"])
def test_trace_equals_the_drawn_delays(path, maker):
    from paper_2204_01133_gb300.api import Solver
    if maker == "rns":
        pb, u0 = W.rns(case="flame", n=4096, pe_size=64, mode="at", k_max=4, seed=3, dt=0.003)
    elif maker == "advdiff":
        pb, u0 = W.advdiff(n=2048, pe_size=64, mode="as", k_max=3, seed=2, cfl=0.05)
    else:
        if path == "persistent":
            pytest.skip("WENO runs on the per-stage path only")
        pb, u0 = W.detonation(n=4096, pe_size=512, mode="at", k_max=4, seed=1)
    steps = 40
    s = Solver(pb, u0, path=path)
    s.run(5)
    s.trace_delays(steps + 10)   # longer than the run: the tail stays untouched
    s.run(steps)
    tr = s.read_trace()
    ref = _oracle_delays(pb, u0, 5 + steps)[5:]
    assert np.array_equal(tr[:steps], ref)
    assert not tr[steps:].any()


@pytest.mark.parametrize("maker", ["rns-flame", "rns-ignition", "advdiff"])
def test_arrival_run_replays_on_the_oracle(maker):
    from paper_2204_01133_gb300.api import OPT_ARRIVAL, Solver
    if maker == "advdiff":
        pb, u0 = W.advdiff(n=2048, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075)
        steps = 400
    else:
        pb, u0 = W.rns(case=maker.split("-")[1], n=16384, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
        steps = 150
    s = Solver(pb, u0, path="persistent")
    s.set_option(OPT_ARRIVAL, 1)
    s.trace_delays(steps)
    s.run(steps)
    g = s.read_state()
    tr = s.read_trace()
    # every delay is within k_max and the start-up clamp
    q = pb["order"] // 2
    for n in range(steps):
        assert tr[n].max() <= min(pb["k_max"], max(0, n - q))
    o = oracle.Oracle(pb, u0)
    o.set_delay_trace(tr, 0)
    assert o.run(steps) == 0
    check(pb, g, o.state(), TOL_RUN, "%s replay" % maker)
    print("arrival delays %s: histogram %s" % (maker, np.bincount(tr.ravel(), minlength=pb["k_max"] + 1)))


def test_arrival_needs_the_persistent_path():
    from paper_2204_01133_gb300 import api
    pb, u0 = W.rns(case="flame", n=4096, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
    s = api.Solver(pb, u0, path="stage")
    s.set_option(api.OPT_ARRIVAL, 1)
    with pytest.raises(api.AtError) as ei:
        s.run(1)
    assert ei.value.code == api.AT_EINVAL
    with pytest.raises(api.AtError):
        s.set_option(api.OPT_ARRIVAL, 2)


def test_arrival_wait_runs_out_without_fault():
    """A PE that never announces its progress: with delays by arrival its
    neighbours wait for data no older than k_max, run out, and report
    AT_ETIMEOUT; the context then runs again."""
    from paper_2204_01133_gb300 import api
    pb, u0 = W.rns(case="flame", n=16384, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
    s = api.Solver(pb, u0, path="persistent")
    s.set_option(api.OPT_ARRIVAL, 1)
    s.set_option(api.OPT_WAIT_LIMIT, 20000)
    s.set_option(api.OPT_WITHHOLD_PE, 5)
    with pytest.raises(api.AtError) as ei:
        s.run(50)
    assert ei.value.code == api.AT_ETIMEOUT
    s.set_option(api.OPT_WITHHOLD_PE, -1)
    s.set_option(api.OPT_WAIT_LIMIT, 4000000)
    s.set_problem(u0)
    s.set_delays()
    s.trace_delays(20)
    s.run(20)
    o = oracle.Oracle(pb, u0)
    o.set_delay_trace(s.read_trace(), 0)
    assert o.run(20) == 0
    check(pb, s.read_state(), o.state(), TOL_RUN, "after the timeout")

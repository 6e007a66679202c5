"""Step-fused path (one launch per RK step, all stages in one pass, the outer
neighbours' edge points recomputed by each CTA): bit for bit the per-stage
path, over split and odd-length runs, alternating with the other paths, and
within the run bound of the oracle."""
import numpy as np
import pytest

from paper_2204_01133_gb300 import workloads as W

from test_gpu_parity import parity

pytestmark = pytest.mark.gpu

PATH_ID = {"stage": 1, "persistent": 2, "fused": 3}


def _run(pb, init, chunks, path):
    from paper_2204_01133_gb300.api import Solver
    s = Solver(pb, init, path=path)
    for c in chunks:
        s.run(c)
    assert s.stats().path == PATH_ID[path]
    out = s.read_state(), s.read_delays()
    s.close()
    return out


@pytest.mark.parametrize("pe_size,pes,order,mode,rk,per_stage", [
    (64, 32, 4, "at", "rk4", 1), (32, 5, 6, "at", "rk4", 1), (128, 40, 2, "as", "rk3tvd", 1),
    (256, 3, 4, "at", "rk2", 1), (64, 64, 4, "sync", "rk4", 1), (32, 1, 4, "at", "rk4", 1),
    (64, 33, 6, "at", "rk4", 0), (32, 17, 6, "at", "rk3tvd", 1), (64, 2, 2, "at", "rk4", 1),
    (64, 300, 4, "at", "rk4", 1)])
def test_fused_equals_per_stage_bitwise(pe_size, pes, order, mode, rk, per_stage):
    """PEs per CTA from 1 to 16 (a partial last CTA, one PE that is its own
    neighbour, two PEs that are each other's outer neighbours), orders 2/4/6,
    AT/AS/SYNC, RK2/3/4, delays per stage and per step."""
    cfl = 0.01 if order == 6 else 0.05
    pb, u0 = W.advdiff(n=pe_size * pes, pe_size=pe_size, order=order, mode=mode, k_max=3, seed=7, cfl=cfl, rk=rk,
                       per_stage=per_stage)
    a_state, a_del = _run(pb, u0, [150], "stage")
    b_state, b_del = _run(pb, u0, [37, 1, 112], "fused")  # odd chunks end with the copy back
    assert np.array_equal(a_state, b_state) and np.array_equal(a_del, b_del)


@pytest.mark.parametrize("order,rk", [(4, "rk4"), (6, "rk3tvd")])
def test_fused_parity_with_oracle(order, rk):
    cfl = 0.01 if order == 6 else 0.075
    pb, u0 = W.advdiff(n=2048, pe_size=64, order=order, mode="at", k_max=3, seed=0, cfl=cfl, rk=rk)
    parity(pb, u0, 400, path="fused")


def test_fused_alternates_with_other_paths():
    """The ring and the state are handed over between paths at at_step
    boundaries."""
    from paper_2204_01133_gb300.api import Solver
    pb, u0 = W.advdiff(n=4096, pe_size=64, mode="at", k_max=3, seed=1, cfl=0.075)
    ref, _ = _run(pb, u0, [300], "stage")
    s = Solver(pb, u0, path="fused")
    s.run(101)
    s.set_path("stage")
    s.run(50)
    s.set_path("fused")
    s.run(50)
    s.set_path("persistent")
    s.run(49)
    s.set_path("fused")
    s.run(50)
    assert np.array_equal(s.read_state(), ref)


def test_fused_full_size_equals_per_stage():
    """2^27 points in 2^21 PEs of 64 (the HBM-sized advection-diffusion run):
    the whole state bit for bit after a few steps."""
    pb, u0 = W.advdiff(n=1 << 27, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075)
    a_state, a_del = _run(pb, u0, [6], "stage")
    b_state, b_del = _run(pb, u0, [6], "fused")
    assert np.array_equal(a_state, b_state) and np.array_equal(a_del, b_del)


def test_fused_rejects_what_it_does_not_take():
    from paper_2204_01133_gb300.api import Solver, OPT_ARRIVAL
    pb, u0 = W.rns(case="flame", n=4096, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
    s = Solver(pb, u0, path="fused")
    with pytest.raises(RuntimeError):
        s.run(1)
    pb, u0 = W.advdiff(n=960, pe_size=48, mode="at", k_max=3, seed=0, cfl=0.05)
    s = Solver(pb, u0, path="fused")
    with pytest.raises(RuntimeError):
        s.run(1)
    pb, u0 = W.advdiff(n=2048, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.05)
    s = Solver(pb, u0, path="fused")
    s.set_option(OPT_ARRIVAL, 1)
    with pytest.raises(RuntimeError):
        s.run(1)


def test_fused_per_step_launches_beyond_one_cooperative_launch():
    """8,192 PEs need more CTAs than the GPU holds at once: one launch per
    step (the multi-step kernel is not used), bitwise the per-stage path."""
    pb, u0 = W.advdiff(n=1 << 19, pe_size=64, mode="at", k_max=3, seed=4, cfl=0.075)
    from paper_2204_01133_gb300.api import Solver
    s = Solver(pb, u0, path="fused")
    s.run(3)
    s.run(2)
    assert s.stats().kernels_launched == 5  # one launch per step
    ref, _ = _run(pb, u0, [5], "stage")
    assert np.array_equal(s.read_state(), ref)


def test_fused_wait_runs_out_without_fault():
    """Fault injection on the multi-step fused kernel: one CTA never publishes
    its progress, its neighbours' bounded waits run out, at_run reports
    AT_ETIMEOUT, and the context then runs correctly again."""
    from paper_2204_01133_gb300 import api
    pb, u0 = W.advdiff(n=16384, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075)
    s = api.Solver(pb, u0, path="fused")
    s.set_option(api.OPT_WAIT_LIMIT, 20000)
    s.set_option(api.OPT_WITHHOLD_PE, 100)  # a PE in the middle of the ring of CTAs
    with pytest.raises(api.AtError) as ei:
        s.run(50)
    assert ei.value.code == api.AT_ETIMEOUT
    s.set_option(api.OPT_WITHHOLD_PE, -1)
    s.set_option(api.OPT_WAIT_LIMIT, 4000000)
    s.set_problem(u0)
    s.set_delays()
    s.set_path("fused")
    s.run(50)
    ref, _ = _run(pb, u0, [50], "stage")
    assert np.array_equal(s.read_state(), ref)

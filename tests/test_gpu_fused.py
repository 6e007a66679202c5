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
    pb, u0 = W.adv_weno(n=512, pe_size=32, mode="at", k_max=3, seed=4, dt_coef=2.0, weno="interpolate")
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


# --------------------------------------------------------------------------
# the reacting flow: the tile-fused kernel (a tile of PEs plus recomputed
# strips of the neighbours, all stages of a step in shared memory)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("pe_size,pes,order,mode,rk,per_stage,case", [
    (64, 256, 6, "at", "rk4", 1, "flame"),         # config 1: 64 tiles of 4 PEs
    (64, 13, 6, "at", "rk4", 1, "ignition"),       # a partial last tile (4, 4, 4, 1)
    (32, 20, 4, "as", "rk4", 1, "flame"),          # tiles of 8 PEs
    (128, 6, 6, "at", "rk3tvd", 0, "ignition"),    # tiles of 2, one delay per step
    (256, 3, 4, "sync", "rk2", 1, "flame"),        # one PE per tile
    (512, 2, 2, "at", "rk4", 1, "flame"),          # a PE larger than the tile target
    (64, 1, 6, "at", "rk4", 1, "flame"),           # one PE, its own neighbour
])
def test_tile_fused_reacting_flow_equals_per_stage_bitwise(pe_size, pes, order, mode, rk, per_stage, case):
    pb, u0 = W.rns(case=case, n=pe_size * pes, pe_size=pe_size, order=order, mode=mode, k_max=4, seed=9,
                   dt=0.003, per_stage=per_stage)
    pb = dict(pb, rk=rk)
    a_state, a_del = _run(pb, u0, [40], "stage")
    b_state, b_del = _run(pb, u0, [13, 1, 26], "fused")  # odd chunks end with the copy back
    assert np.array_equal(a_state, b_state) and np.array_equal(a_del, b_del)


def test_tile_fused_parity_with_oracle():
    pb, u0 = W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
    parity(pb, u0, 150, path="fused", what="tile-fused flame")


def test_tile_fused_alternates_with_other_paths():
    from paper_2204_01133_gb300.api import Solver
    pb, u0 = W.rns(case="flame", n=16384, pe_size=64, mode="at", k_max=4, seed=2, dt=0.003)
    ref, _ = _run(pb, u0, [100], "stage")
    s = Solver(pb, u0, path="fused")
    s.run(31)
    s.set_path("stage")
    s.run(20)
    s.set_path("persistent")
    s.run(19)
    s.set_path("fused")
    s.run(30)
    assert np.array_equal(s.read_state(), ref)


def test_tile_fused_full_size_equals_per_stage_and_the_oracle():
    """The reacting flame at N = 2^24 (2^18 PEs of 64, the size of the large
    per-stage benchmark run): the whole state bit for bit the per-stage path's
    after 6 steps, and sampled PEs against the oracle on 5-PE windows."""
    import oracle
    from parity import TOL_RUN, check
    pb, u0 = W.rns(case="flame", n=1 << 24, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
    a_state, a_del = _run(pb, u0, [6], "stage")
    b_state, b_del = _run(pb, u0, [6], "fused")
    assert np.array_equal(a_state, b_state) and np.array_equal(a_del, b_del)
    P, B = pb["n"] // pb["pe_size"], pb["pe_size"]
    for p in (0, 77777, P - 1):
        idx = np.arange(p - 2, p + 3) % P
        sub = np.concatenate([u0[:, i * B:(i + 1) * B] for i in idx], axis=1)
        o = oracle.Oracle(dict(pb, n=5 * B, pe_base=p - 2, pe_total=P), sub)
        assert o.run(6) == 0
        check(pb, b_state[:, p * B:(p + 1) * B], o.state()[:, 2 * B:3 * B], TOL_RUN, "tile-fused PE %d" % p)


# --------------------------------------------------------------------------
# the WENO PDEs (the detonation): a tile is one window of the per-stage
# kernels plus recomputed strips
# --------------------------------------------------------------------------
@pytest.mark.parametrize("maker,steps", [
    ("det-1024", 40), ("det-512", 40), ("det-96", 30), ("det-1024-sync", 30), ("det-512-as-perstep", 30),
    ("det-one-pe", 30), ("adv", 60), ("burgers", 60)])
def test_tile_fused_weno_equals_per_stage_bitwise(maker, steps):
    """Windows of 256 in PEs of 1024 and 512 (inner windows: the strips are
    the same PE's neighbouring windows), PEs of 96 (one window, both strips
    from the neighbouring PEs), SYNC, AS with one delay per step, one PE that
    is its own neighbour; scalar advection and Burgers."""
    if maker.startswith("det"):
        B = {"det-1024": 1024, "det-512": 512, "det-96": 96, "det-1024-sync": 1024, "det-512-as-perstep": 512,
             "det-one-pe": 512}[maker]
        pes = 1 if maker == "det-one-pe" else 8
        mode = "sync" if "sync" in maker else ("as" if "-as" in maker else "at")
        pb, u0 = W.detonation(n=B * pes, pe_size=B, mode=mode, k_max=4, seed=3,
                              per_stage=0 if "perstep" in maker else 1)
    elif maker == "adv":
        pb, u0 = W.adv_weno(n=512, pe_size=32, mode="at", k_max=3, seed=4, dt_coef=2.0)
    else:
        pb, u0 = W.burgers(n=1024, pe_size=64, mode="at", k_max=3, seed=6, dt_coef=1.0)
    a_state, a_del = _run(pb, u0, [steps], "stage")
    b_state, b_del = _run(pb, u0, [7, 1, steps - 8], "fused")
    assert np.array_equal(a_state, b_state) and np.array_equal(a_del, b_del)


def test_tile_fused_detonation_full_size():
    """The N = 2^24 detonation: the whole state bit for bit the per-stage
    path's after 6 steps."""
    pb, u0 = W.detonation()
    a_state, a_del = _run(pb, u0, [6], "stage")
    b_state, b_del = _run(pb, u0, [6], "fused")
    assert np.array_equal(a_state, b_state) and np.array_equal(a_del, b_del)

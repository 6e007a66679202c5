"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element, on the same seeded inputs and delay streams.

Tolerance (FP64), per variable (``parity.errors``: each variable against its
own largest |value|, momentum against max(|rho u|, rho c)): <= 1e-12 after
one step and <= 1e-10 after the whole run.  Delays are integers and must
agree bitwise.

Shock-carrying runs (the detonation) amplify round-off: the WENO-JS weights
respond steeply where a smoothness indicator is near eps (an absolute 1e-6
against fluxes of order 10^3), so two correct FP64 implementations drift
apart.  Each such case has a fixed bound, 20 times the drift of the oracle
against itself under a 1e-15 relative perturbation of its initial state
(largest of four seeded perturbations and of the four variables, rounded
up); tests/test_parity_bounds_cpu.py measures those drifts again on the
CPU and checks that every bound stays between 10 and 40 times its drift.
"""
import numpy as np
import pytest

import oracle
from paper_2204_01133_gb300 import workloads as W
from parity import (DET_CASES, DET_FULL_SHOCK, DET_FULL_STEPS, DET_RUN, DET_STEP, TOL_RUN, TOL_STEP, check,
                    detonation_window, scales)

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2204_01133_gb300 import build
    build.build()


def parity(pb, init, steps, first_tol=TOL_STEP, run_tol=TOL_RUN, check_delays=True, path="auto", what=""):
    """Run the GPU path and the oracle side by side: one step, then the rest;
    per-variable errors within first_tol / run_tol (scalars or one bound per
    variable), delay logs bitwise."""
    from paper_2204_01133_gb300.api import Solver
    s = Solver(pb, init, path=path)
    o = oracle.Oracle(pb, init)
    s.run(1)
    assert o.run(1) == 0
    check(pb, s.read_state(), o.state(), first_tol, "%s step 1" % what)
    if check_delays:
        assert np.array_equal(s.read_delays(), o.delays())
    if steps > 1:
        s.run(steps - 1)
        assert o.run(steps - 1) == 0
        check(pb, s.read_state(), o.state(), run_tol, "%s step %d" % (what, steps))
        if check_delays:
            assert np.array_equal(s.read_delays(), o.delays())
    return s, o


@pytest.mark.parametrize("path", ["stage", "persistent"])
def test_advdiff_literal_config_full_run(path):
    """N = 2048, 32 PEs of 64, AT4 + RK4, k uniform on {0..3}, seed 0, 10,000 steps."""
    pb, u0 = W.advdiff(n=2048, pe_size=64, order=4, mode="at", k_max=3, seed=0, cfl=0.075)
    parity(pb, u0, 10000, path=path)


@pytest.mark.parametrize("mode", ["sync", "as", "at"])
@pytest.mark.parametrize("order,cfl", [(2, 0.05), (4, 0.05), (6, 0.01)])
def test_advdiff_modes_orders(mode, order, cfl):
    pb, u0 = W.advdiff(n=960, pe_size=48, order=order, mode=mode, k_max=3, seed=11, cfl=cfl)
    parity(pb, u0, 300)


@pytest.mark.parametrize("rk", ["rk2", "rk3tvd", "rk4"])
@pytest.mark.parametrize("per_stage", [0, 1])
def test_advdiff_rk_and_delay_granularity(rk, per_stage):
    pb, u0 = W.advdiff(n=512, pe_size=16, order=4, mode="at", k_max=2, seed=5, cfl=0.04, rk=rk,
                       per_stage=per_stage, dist="table", prob=[0.4, 0.5, 0.1])
    parity(pb, u0, 200)


@pytest.mark.parametrize("pe_size,n", [(8, 8), (16, 16 * 7), (1024, 3072), (520, 1040), (263, 789)])
def test_advdiff_edge_shapes(pe_size, n):
    """Degenerate decompositions: one PE (its own neighbour), an odd PE count,
    PEs split into several windows, a window length that is not a power of
    two, a prime PE size (one window of 263 points)."""
    pb, u0 = W.advdiff(n=n, pe_size=pe_size, order=4, mode="at", k_max=3, seed=3, cfl=0.05)
    parity(pb, u0, 60)


@pytest.mark.parametrize("pe_size,pes,order,mode,rk,cfl", [
    (32, 5, 6, "at", "rk4", 0.01), (32, 1, 4, "at", "rk4", 0.05), (64, 13, 4, "sync", "rk4", 0.05),
    (128, 11, 2, "as", "rk3tvd", 0.05), (256, 9, 4, "at", "rk2", 0.04), (64, 17, 6, "as", "rk4", 0.01)])
def test_advdiff_warp_per_pe_kernel(pe_size, pes, order, mode, rk, cfl):
    """PEs of 32, 64, 128 or 256 points take the one-warp-per-PE kernel on the
    per-stage path: PE counts that leave warps of the last CTA idle, a single
    PE, every order, mode and RK scheme."""
    pb, u0 = W.advdiff(n=pe_size * pes, pe_size=pe_size, order=order, mode=mode, k_max=3, seed=4, cfl=cfl,
                       rk=rk)
    parity(pb, u0, 120, path="stage")


@pytest.mark.parametrize("path", ["stage", "persistent"])
@pytest.mark.parametrize("case", ["flame", "ignition"])
def test_rns_literal_size(case, path):
    """Reacting N-S at N = 16,384 (256 PEs of 64), AT6 + RK4, k uniform on {0..4}."""
    pb, u0 = W.rns(case=case, n=16384, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
    parity(pb, u0, 150, path=path)


@pytest.mark.parametrize("case,mode,n,B,order", [
    ("flame", "at", 16384, 64, 6), ("ignition", "at", 16384, 64, 6), ("flame", "sync", 2048, 64, 6),
    ("flame", "as", 2048, 32, 4), ("ignition", "at", 1536, 48, 2), ("flame", "at", 2048, 32, 4)])
def test_rns_chain_rule_form(case, mode, n, B, order):
    """The chain-rule form of Sec. 4 (primitives differentiated and
    extrapolated), per-stage path, against the oracle's chain-rule RHS."""
    pb, u0 = W.rns(case=case, n=n, pe_size=B, order=order, mode=mode, k_max=4, seed=3, dt=0.003, form="chain")
    parity(pb, u0, 150)


@pytest.mark.parametrize("mode", ["sync", "as"])
def test_rns_modes(mode):
    pb, u0 = W.rns(case="flame", n=2048, pe_size=64, mode=mode, k_max=4, seed=2, dt=0.003)
    parity(pb, u0, 100)


@pytest.mark.parametrize("case", ["weno-1024", "weno-512", "weno-96"])
def test_detonation_weno(case):
    """Reactive Euler, WENO5 + AT-WENO5, RK3-TVD, k geometric(0.5) on {0..4};
    PEs of 1024 and 512 points (4 and 2 windows of 256) and of 96 (one
    window of a length that is not a power of two)."""
    kw, steps = DET_CASES[case]
    pb, u0 = W.detonation(**kw)
    parity(pb, u0, steps, first_tol=DET_STEP, run_tol=DET_RUN[case], what=case)


@pytest.mark.parametrize("mode", ["sync", "as"])
def test_detonation_modes(mode):
    kw, steps = DET_CASES[mode]
    pb, u0 = W.detonation(**kw)
    parity(pb, u0, steps, first_tol=DET_STEP, run_tol=DET_RUN[mode], what=mode)


@pytest.mark.parametrize("mode", ["sync", "as", "at"])
def test_scalar_weno(mode):
    pb, u0 = W.adv_weno(n=512, pe_size=32, mode=mode, k_max=3, seed=4, dt_coef=2.0)
    parity(pb, u0, 100)


@pytest.mark.parametrize("mode", ["sync", "as", "at"])
def test_burgers_weno(mode):
    pb, u0 = W.burgers(n=1024, pe_size=64, mode=mode, k_max=3, seed=6, dt_coef=1.0)
    parity(pb, u0, 150)


def test_detonation_full_size_sampled_pes():
    """The N = 2^24, 16,384-PE detonation in the launch configuration the
    benchmark times, 40 steps.  The oracle recomputes sampled PEs on a 5-PE
    window of the domain (with the global PE index in the delay counter):
    after s steps only points within 9 s of the window's outer edges can
    differ, 360 points here, less than the two PEs on each side of the
    middle one.  PE 0 holds the shock and PE 16,383 the rarefaction behind
    the slab; they take their fixed shock bounds, the PEs in constant flow
    (1, 2, 7777, 12345, 16382) the plain run bound."""
    from paper_2204_01133_gb300.api import Solver
    steps = DET_FULL_STEPS
    pb, u0 = W.detonation()
    P, B = pb["n"] // pb["pe_size"], pb["pe_size"]
    s = Solver(pb, u0)
    s.run(steps)
    g = s.read_state()
    gd = s.read_delays()
    for p in (0, 1, 2, 7777, 12345, P - 2, P - 1):
        spb, sub = detonation_window(pb, u0, p)
        o = oracle.Oracle(spb, sub)
        assert o.run(steps) == 0
        tol = DET_RUN[DET_FULL_SHOCK[p]] if p in DET_FULL_SHOCK else TOL_RUN
        check(spb, g[:, p * B:(p + 1) * B], o.state()[:, 2 * B:3 * B], tol, "PE %d step %d" % (p, steps))
        assert np.array_equal(gd[:, p, :], o.delays()[:, 2, :])


def _sampled_full_size(pb, u0, steps, pes):
    """Run the full problem on the GPU, then recompute the given PEs with the
    oracle on a 5-PE window (global PE indices in the delay counter).  After
    `steps` steps only points within S H steps of the window's outer edges can
    differ, which stays outside the middle PE for the step counts used."""
    from paper_2204_01133_gb300.api import Solver
    P, B = pb["n"] // pb["pe_size"], pb["pe_size"]
    s = Solver(pb, u0)
    s.run(steps)
    g = s.read_state()
    gd = s.read_delays()
    s.close()
    for p in pes:
        idx = np.arange(p - 2, p + 3) % P
        sub = np.concatenate([u0[:, i * B:(i + 1) * B] for i in idx], axis=1)
        o = oracle.Oracle(dict(pb, n=5 * B, pe_base=p - 2, pe_total=P), sub)
        assert o.run(steps) == 0
        check(pb, g[:, p * B:(p + 1) * B], o.state()[:, 2 * B:3 * B], TOL_RUN, "PE %d step %d" % (p, steps))
        assert np.array_equal(gd[:, p, :], o.delays()[:, 2, :])


def test_advdiff_full_size_sampled_pes():
    """Advection-diffusion at N = 2^27 (2^21 PEs of 64), the size and launch
    configuration of the HBM benchmark run; 12 steps move information at most
    96 points, less than two PEs."""
    pb, u0 = W.advdiff(n=1 << 27, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075)
    P = pb["n"] // pb["pe_size"]
    _sampled_full_size(pb, u0, 12, (0, 1, 123457, P - 1))


def test_rns_full_size_sampled_pes():
    """Reacting N-S flame at N = 2^24 (2^18 PEs of 64), per-stage launches as
    benchmarked; 6 steps move information at most 72 points."""
    pb, u0 = W.rns(case="flame", n=1 << 24, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
    P = pb["n"] // pb["pe_size"]
    _sampled_full_size(pb, u0, 6, (0, 77777, P // 2, P - 1))


@pytest.mark.parametrize("path,maker", [("stage", "rns"), ("persistent", "rns"), ("stage", "detonation"),
                                        ("persistent", "advdiff"), ("stage", "advdiff-rk3")])
def test_ring_holds_the_owners_stage_arguments(path, maker):
    """The history ring (the per-step message of S stages of Sec. 2.3): after a
    run, every slot holds the owner PE's edge window of its stage argument
    U^{m,(s)} as the oracle computes it, for every level both keep."""
    import ctypes
    from paper_2204_01133_gb300 import api
    if maker == "rns":
        pb, u0 = W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=1, dt=0.003)
    elif maker == "detonation":
        pb, u0 = W.detonation(**DET_CASES["ring"][0])
    elif maker == "advdiff":
        pb, u0 = W.advdiff(n=1024, pe_size=32, mode="as", k_max=3, seed=3, cfl=0.05)
    else:
        pb, u0 = W.advdiff(n=960, pe_size=48, order=6, mode="at", k_max=2, seed=4, cfl=0.01, rk="rk3tvd")
    steps = 25
    tol = DET_RUN["ring"] if maker == "detonation" else TOL_RUN
    s = api.Solver(pb, u0, path=path)
    s.run(steps)
    st = s.stats()
    R, S, H, nv = st.ring_levels, st.stages, st.halo, st.nvar
    P, B = pb["n"] // pb["pe_size"], pb["pe_size"]
    ring = np.empty((R, S, P, 2, H, nv), dtype=np.float64)
    api.check(api.lib().at_read(s._h, api.READ_RING, ctypes.c_void_p(ring.ctypes.data), ring.nbytes, 0))
    o = oracle.Oracle(pb, u0)
    assert o.run(steps) == 0
    idx = np.arange(P)[:, None] * B
    left = idx + np.arange(H)[None, :]
    right = idx + (B - H) + np.arange(H)[None, :]
    checked = 0
    for m in range(steps - R + 1, steps + 1):
        for stage in range(S):
            if m == steps and stage > 0:
                continue  # not produced yet
            U = o.history(m, stage)
            if U is None:
                continue
            g = ring[m % R, stage]                       # [P][2][H][nvar]
            ref = np.stack([U[:, left], U[:, right]], axis=0).transpose(2, 0, 3, 1)  # [P][2][H][nvar]
            # per variable, each against the scale of its whole field
            err = np.abs(g - ref).max(axis=(0, 1, 2)) / scales(pb, U)
            assert np.all(err <= tol), (m, stage, err, tol)
            checked += 1
    assert checked >= S * 2


def test_deterministic_and_seeded():
    from paper_2204_01133_gb300.api import Solver
    pb, u0 = W.advdiff(n=2048, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075)
    a = Solver(pb, u0)
    a.run(500)
    b = Solver(pb, u0)
    b.run(500)
    assert np.array_equal(a.read_state(), b.read_state())
    c = Solver(dict(pb, seed=1), u0)
    c.run(500)
    assert not np.array_equal(a.read_state(), c.read_state())


def test_unstable_run_reports_status():
    """A time step far beyond the AT stability limit makes the state blow up;
    the device flag turns that into AT_EUNSTABLE (no fault, no hang)."""
    from paper_2204_01133_gb300 import api
    pb, u0 = W.advdiff(n=2048, pe_size=64, mode="at", k_max=3, seed=0, cfl=2.0)
    s = api.Solver(pb, u0)
    with pytest.raises(api.AtError) as ei:
        s.run(3000)
    assert ei.value.code == api.AT_EUNSTABLE
    assert s.stats().status == api.AT_EUNSTABLE


# --------------------------------------------------------------------------
# persistent, neighbour-synchronised path
# --------------------------------------------------------------------------
def _run(pb, init, chunks, path):
    from paper_2204_01133_gb300.api import Solver
    s = Solver(pb, init, path=path)
    for c in chunks:
        s.run(c)
    assert s.stats().path == {"stage": 1, "persistent": 2}[path]
    return s.read_state(), s.read_delays()


@pytest.mark.parametrize("maker", ["advdiff", "rns", "advdiff-as", "advdiff-rk3-step", "rns-order4-sync"])
def test_persistent_equals_per_stage_bitwise(maker):
    """Same arithmetic in the same order: the two paths agree bit for bit,
    also when a run is split over several at_step calls."""
    if maker == "advdiff":
        pb, u0 = W.advdiff(n=2048, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075)
    elif maker == "rns":
        pb, u0 = W.rns(case="flame", n=16384, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
    elif maker == "advdiff-as":
        pb, u0 = W.advdiff(n=960, pe_size=48, order=6, mode="as", k_max=3, seed=2, cfl=0.01)
    elif maker == "advdiff-rk3-step":
        pb, u0 = W.advdiff(n=512, pe_size=16, order=2, mode="at", k_max=2, seed=3, cfl=0.04, rk="rk3tvd",
                           per_stage=0)
    else:
        pb, u0 = W.rns(case="ignition", n=4096, pe_size=32, order=4, mode="sync", k_max=2, seed=1, dt=0.003)
    a_state, a_del = _run(pb, u0, [200], "stage")
    b_state, b_del = _run(pb, u0, [200], "persistent")
    c_state, c_del = _run(pb, u0, [3, 1, 96, 100], "persistent")
    assert np.array_equal(a_state, b_state) and np.array_equal(a_del, b_del)
    assert np.array_equal(a_state, c_state) and np.array_equal(a_del, c_del)


@pytest.mark.parametrize("pe_size,pes,order,mode,rk", [
    (64, 32, 4, "at", "rk4"), (32, 5, 6, "at", "rk4"), (128, 12, 2, "as", "rk3tvd"), (256, 3, 4, "at", "rk2"),
    (64, 64, 4, "sync", "rk4"), (32, 1, 4, "at", "rk4"), (64, 48, 6, "as", "rk4"), (128, 32, 6, "at", "rk4"),
    (256, 32, 2, "at", "rk3tvd"), (128, 16, 4, "at", "rk2"), (256, 16, 6, "at", "rk4")])
def test_cluster_kernel_equals_per_stage_bitwise(pe_size, pes, order, mode, rk):
    """Advection-diffusion on at most 64 PEs of 32..256 points takes the
    one-cluster kernel on the persistent path (ring in distributed shared
    memory, one cluster barrier per stage; 1 to 4 PEs per CTA, 1 to 8
    warps per PE): bit for bit the per-stage result, also over split runs,
    and within the run bound of the oracle."""
    cfl = 0.01 if order == 6 else 0.05
    pb, u0 = W.advdiff(n=pe_size * pes, pe_size=pe_size, order=order, mode=mode, k_max=3, seed=6, cfl=cfl, rk=rk)
    a_state, a_del = _run(pb, u0, [150], "stage")
    b_state, b_del = _run(pb, u0, [37, 1, 112], "persistent")
    assert np.array_equal(a_state, b_state) and np.array_equal(a_del, b_del)
    parity(pb, u0, 150, path="persistent")


def test_cluster_kernel_and_per_stage_alternate():
    """Switching between the one-cluster kernel and per-stage launches
    mid-run: the history ring is handed over through global memory."""
    from paper_2204_01133_gb300.api import Solver
    pb, u0 = W.advdiff(n=2048, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075)
    ref, _ = _run(pb, u0, [300], "stage")
    s = Solver(pb, u0, path="persistent")
    s.run(100)
    s.set_path("stage")
    s.run(50)
    s.set_path("persistent")
    s.run(150)
    assert np.array_equal(s.read_state(), ref)


def test_persistent_after_per_stage_steps():
    from paper_2204_01133_gb300.api import Solver
    pb, u0 = W.rns(case="flame", n=16384, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
    ref, _ = _run(pb, u0, [120], "stage")
    s = Solver(pb, u0, path="stage")
    s.run(50)
    s.set_path("persistent")
    s.run(40)
    s.set_path("stage")
    s.run(30)
    assert np.array_equal(s.read_state(), ref)


def test_persistent_wait_runs_out_without_fault():
    """Fault injection: one PE never announces its progress.  Its neighbours'
    bounded waits run out, the kernel ends, at_run reports AT_ETIMEOUT, and
    the same context then runs correctly again."""
    from paper_2204_01133_gb300 import api
    pb, u0 = W.rns(case="flame", n=16384, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
    s = api.Solver(pb, u0, path="persistent")
    s.set_option(api.OPT_WAIT_LIMIT, 20000)
    s.set_option(api.OPT_WITHHOLD_PE, 17)
    with pytest.raises(api.AtError) as ei:
        s.run(50)
    assert ei.value.code == api.AT_ETIMEOUT
    assert s.stats().status == api.AT_ETIMEOUT
    # recover: restore the initial state, clear the fault, rerun
    s.set_option(api.OPT_WITHHOLD_PE, -1)
    s.set_option(api.OPT_WAIT_LIMIT, 4000000)
    s.set_problem(u0)
    s.set_delays()
    s.set_path("persistent")
    s.run(50)
    ref, _ = _run(pb, u0, [50], "stage")
    assert np.array_equal(s.read_state(), ref)


def test_contexts_of_different_pe_sizes_interleaved():
    """Several contexts set up first and stepped afterwards, with different
    PE sizes (and so different shared-memory needs) on the persistent path."""
    from paper_2204_01133_gb300.api import Solver
    probs = [W.rns(case="flame", n=2048, pe_size=B, mode="at", k_max=4, seed=B, dt=0.003) for B in (64, 32, 128)]
    solvers = [Solver(pb, u0) for pb, u0 in probs]
    for s in solvers:
        s.run(20)
    for (pb, u0), s in zip(probs, solvers):
        assert s.stats().path == 2
        assert np.array_equal(s.read_state(), _run(pb, u0, [20], "stage")[0])

"""Batched solves on the GPU: every instance of a mixed batch must equal,
bit for bit, the same instance solved alone through a context (same
kernels' arithmetic, same delay stream), whatever the chunking, slot reuse,
launch configuration or graph replay; and a seeded sample of instances with
the shapes of the 4,096-instance reacting batch is checked against the CPU
oracle directly, in both batch modes."""
import numpy as np
import pytest

import oracle
from paper_2204_01133_gb300 import workloads as W
from parity import TOL_RUN, check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2204_01133_gb300 import build
    build.build()


def mixed_instances():
    out = []
    for i, (pb, init, _) in enumerate(W.batched_rns(count=10, seed=3, nsteps=0, n_max=2048)):
        out.append((pb, init, 23 + 7 * i))
    pb, init = W.rns(case="flame", n=1536, pe_size=48, order=4, mode="as", k_max=3, seed=5, dt=0.003, instance=77)
    out.append((pb, init, 40))
    pb, init = W.advdiff(n=2048, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075)
    out.append((dict(pb, instance=78), init, 60))
    pb, init = W.advdiff(n=960, pe_size=48, order=2, mode="sync", k_max=1, seed=2, cfl=0.05, rk="rk2")
    out.append((dict(pb, instance=79), init, 33))
    pb, init = W.detonation(n=4096, pe_size=512, mode="at", k_max=4, seed=9)
    out.append((dict(pb, instance=80), init, 25))
    pb, init = W.adv_weno(n=512, pe_size=32, mode="at", k_max=3, seed=4, dt_coef=2.0)
    out.append((dict(pb, instance=81), init, 30))
    pb, init = W.burgers(n=768, pe_size=48, mode="at", k_max=2, seed=7, dt_coef=1.0)
    out.append((dict(pb, instance=82), init, 35))
    pb, init = W.rns(case="ignition", n=1024, pe_size=32, order=6, mode="at", k_max=3, seed=8, dt=0.003,
                     instance=83, form="chain")
    out.append((pb, init, 28))
    return out


def alone(pb, init, nsteps):
    from paper_2204_01133_gb300.api import Solver
    s = Solver(pb, init, path="stage")
    s.run(nsteps)
    return s.read_state(), s.read_delays()


@pytest.mark.parametrize("config", [(0, 256, 3, True), (0, 128, 6, False), (0, 256, 1, True), (1, 256, 1, True),
                                    (1, 128, 1, False)])
def test_batch_equals_alone_bitwise(config):
    from paper_2204_01133_gb300.batch import Batch
    inst = mixed_instances()
    ref = [alone(pb, init, n)[0] for pb, init, n in inst]
    b = Batch(capacity=len(inst) + 3)
    b.set_config(*config)
    for i, (pb, init, n) in enumerate(inst):
        b.bind(i, pb, init, n)
    while any(b.query(i).left > 0 for i in range(len(inst))):
        b.run(9)
    for i, (pb, init, n) in enumerate(inst):
        info = b.query(i)
        assert info.level == n and info.left == 0 and info.status == 0
        got = b.state(i).cpu().numpy()
        assert np.array_equal(got, ref[i]), (i, pb["pde"], np.abs(got - ref[i]).max())


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_slot_reuse_and_late_admission(mode):
    """Continuous batching: a finished instance's slot is released and a new
    instance bound while the others are mid-run; every result still equals
    the instance solved alone."""
    from paper_2204_01133_gb300.batch import Batch
    inst = mixed_instances()[:6]
    extra = W.batched_rns(count=12, seed=8, nsteps=0, n_max=1024)[10:]
    b = Batch(capacity=6)
    b.set_config(mode, 256, 3, True)
    for i, (pb, init, n) in enumerate(inst):
        b.bind(i, pb, init, n)
    b.run(25)                        # instance 0 (23 steps) is done
    assert b.query(0).left == 0
    done0 = b.release(0)
    got0 = done0["state"].cpu().numpy()
    assert np.array_equal(got0, alone(*inst[0])[0])
    pb, init, _ = extra[0]
    b.bind(0, pb, init, 31)          # late admission into the freed slot
    while any(b.query(i).left > 0 for i in range(6)):
        b.run(10)
    assert np.array_equal(b.state(0).cpu().numpy(), alone(pb, init, 31)[0])
    for i in range(1, 6):
        assert np.array_equal(b.state(i).cpu().numpy(), alone(*inst[i])[0])


def test_autotuner_keeps_results_and_picks_a_candidate(tmp_path, monkeypatch):
    from paper_2204_01133_gb300 import batch as BT
    monkeypatch.setenv("AT_TUNE_CACHE", str(tmp_path / "tune.json"))
    inst = W.batched_rns(count=24, seed=11, nsteps=0, n_max=4096)
    b = BT.Batch(capacity=24)
    for i, (pb, init, _) in enumerate(inst):
        b.bind(i, pb, init, 40)
    cands = [(BT.INSTANCE, 256, 2), (BT.INSTANCE, 128, 4), (BT.FLAT, 256, 1)]
    res = BT.autotune(b, chunk=2, candidates=cands)
    assert (res["mode"], res["block"], res["ctas_per_sm"]) in cands
    while any(b.query(i).left > 0 for i in range(24)):
        b.run(7)
    for i in (0, 5, 23):
        pb, init, _ = inst[i]
        assert np.array_equal(b.state(i).cpu().numpy(), alone(pb, init, 40)[0])
    again = BT.autotune(b, chunk=2, candidates=cands)
    assert again["cached"] and again["block"] == res["block"] and again["mode"] == res["mode"]


def test_flat_mode_window_map_limit():
    from paper_2204_01133_gb300 import api
    from paper_2204_01133_gb300.batch import Batch
    b = Batch(capacity=4, max_windows=40)
    pb, init = W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)  # 32 windows
    b.bind(0, pb, init, 5)
    with pytest.raises(api.AtError) as ei:
        b.bind(1, pb, init, 5)
    assert ei.value.code == api.AT_ENOMEM
    b.release(0)
    b.bind(1, pb, init, 5)  # fits again once the first is released


def config2_sample():
    """Instances with the shapes of the batched reacting workload: the
    smallest size (N = 256, PEs of 32) at every largest delay 2, 3, 4, as a
    flame and as an ignition, with T0 (K-equivalent / 300) and the fuel
    fraction 0.5 phi drawn as the batch draws them; one instance with the
    largest Philox instance word; the largest size of the mix (N = 8192,
    PEs of 64)."""
    rng = np.random.default_rng(2204)
    out = []
    for k_max in (2, 3, 4):
        for case in ("flame", "ignition"):
            T0 = float(rng.uniform(900.0, 1400.0)) / 300.0
            phi = float(rng.uniform(0.5, 1.5))
            out.append(W.rns(case=case, n=256, pe_size=32, mode="at", k_max=k_max, seed=1000 + len(out), dt=0.002,
                             T_init=T0, T_unburnt=T0, Y_init=0.5 * phi, instance=len(out)))
    out.append(W.rns(case="flame", n=512, pe_size=64, mode="at", k_max=4, seed=77, dt=0.002, T_init=3.5,
                     T_unburnt=3.5, Y_init=0.6, instance=0xFFFFFFFF))
    out.append(W.rns(case="ignition", n=8192, pe_size=64, mode="at", k_max=3, seed=78, dt=0.002, T_init=4.2,
                     T_unburnt=4.2, Y_init=0.4, instance=4096))
    return out


@pytest.mark.parametrize("mode", [0, 1])
def test_batched_config2_instances_match_the_oracle(mode):
    """200 RK4 steps of every sampled instance in one batch (instance mode:
    one CTA per instance; flat mode: one launch per stage over all windows),
    each against its own oracle run, per variable within the run bound."""
    from paper_2204_01133_gb300.batch import Batch
    steps = 200
    inst = config2_sample()
    b = Batch(capacity=len(inst))
    b.set_config(mode, 256, 3, True)
    for i, (pb, init) in enumerate(inst):
        b.bind(i, pb, init, steps)
    while any(b.query(i).left > 0 for i in range(len(inst))):
        b.run(50)
    for i, (pb, init) in enumerate(inst):
        assert b.query(i).status == 0
        o = oracle.Oracle(pb, init)
        assert o.run(steps) == 0
        check(pb, b.state(i).cpu().numpy(), o.state(), TOL_RUN,
              "batch mode %d instance %d (n=%d, k_max=%d, word %d)" % (mode, i, pb["n"], pb["k_max"], pb["instance"]))

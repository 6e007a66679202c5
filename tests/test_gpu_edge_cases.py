"""Edge cases of the GPU path against the oracle: the smallest PE the
stencils allow (pe_size = 2H) for every PDE, that PE alone (its own
neighbour on both sides), the largest single window (a prime PE size of
1021, one window per PE, the largest shared-memory request of the WENO
kernel), a zero-step call (state and delay log unchanged, bit for bit, on
every path), a negative step count (refused) and forced maximum delays
(every drawn delay at k_max, the oldest levels the ring keeps).  The Euler cases use the
smooth entropy wave, so the plain per-variable bounds (1e-12 after one
step, 1e-10 after the run) apply."""
import numpy as np
import pytest

from paper_2204_01133_gb300 import workloads as W
from test_gpu_parity import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2204_01133_gb300 import build
    build.build()


def _case(name, pes):
    if name == "advdiff-order2":
        return W.advdiff(n=2 * pes, pe_size=2, order=2, mode="at", k_max=3, seed=21, cfl=0.05), 200
    if name == "advdiff-order6":
        return W.advdiff(n=6 * pes, pe_size=6, order=6, mode="at", k_max=3, seed=22, cfl=0.01), 200
    if name == "rns-order6":
        return W.rns(case="flame", n=6 * pes, pe_size=6, order=6, mode="at", k_max=4, seed=23, dt=0.003), 60
    if name == "rns-order2-ignition":
        return W.rns(case="ignition", n=2 * pes, pe_size=2, order=2, mode="at", k_max=2, seed=24, dt=0.003), 60
    if name == "euler-weno":
        return W.entropy_wave(n=6 * pes, pe_size=6, mode="at", k_max=2, seed=25), 60
    return W.adv_weno(n=6 * pes, pe_size=6, mode="at", k_max=2, seed=26), 60


CASES = ["advdiff-order2", "advdiff-order6", "rns-order6", "rns-order2-ignition", "euler-weno", "adv-weno"]


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("pes", [1, 40])
def test_smallest_pe_matches_the_oracle(name, pes):
    (pb, u0), steps = _case(name, pes)
    assert pb["pe_size"] == 2 * (3 if pb["pde"] in ("euler", "adv_weno") else pb["order"] // 2)
    parity(pb, u0, steps, what="%s, %d PE(s) of %d" % (name, pes, pb["pe_size"]))


@pytest.mark.parametrize("name", ["advdiff-order6", "rns-order6"])
def test_smallest_pe_on_the_persistent_path(name):
    (pb, u0), steps = _case(name, 40)
    s, _ = parity(pb, u0, steps, path="persistent", what="%s persistent" % name)
    assert s.stats().path == 2


@pytest.mark.parametrize("pes", [1, 3])
def test_largest_window_matches_the_oracle(pes):
    """A prime PE size of 1021 has no divisor in [2H, 256]: the PE is one
    window of 1021 points (about 190 KB of shared memory per CTA)."""
    pb, u0 = W.entropy_wave(n=1021 * pes, pe_size=1021, mode="at", k_max=3, seed=27)
    parity(pb, u0, 40, what="entropy wave, %d PE(s) of 1021" % pes)


@pytest.mark.parametrize("path,maker", [("stage", "rns"), ("persistent", "rns"), ("fused", "advdiff"),
                                        ("stage", "detonation"), ("fused", "rns")])
def test_zero_steps_change_nothing(path, maker):
    from paper_2204_01133_gb300.api import Solver
    if maker == "rns":
        pb, u0 = W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=3, dt=0.003)
    elif maker == "advdiff":
        pb, u0 = W.advdiff(n=8192, pe_size=64, mode="at", k_max=3, seed=3, cfl=0.075)
    else:
        pb, u0 = W.detonation(n=4096, pe_size=256, mode="at", k_max=4, seed=3)
    s = Solver(pb, u0, path=path)
    s.run(5)
    st, dl = s.read_state(), s.read_delays()
    s.run(0)
    assert np.array_equal(s.read_state(), st)
    assert np.array_equal(s.read_delays(), dl)
    # and the run continues exactly as one without the empty call
    r = Solver(pb, u0, path=path)
    r.run(5)
    r.run(7)
    s.run(7)
    assert np.array_equal(s.read_state(), r.read_state())


def test_negative_step_count_is_refused():
    from paper_2204_01133_gb300 import api
    pb, u0 = W.advdiff(n=2048, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075)
    s = api.Solver(pb, u0)
    st = s.read_state()
    with pytest.raises(api.AtError) as ei:
        s.run(-1)
    assert ei.value.code == api.AT_EINVAL
    assert np.array_equal(s.read_state(), st)


@pytest.mark.parametrize("name", ["advdiff", "rns", "entropy-wave"])
def test_every_delay_at_its_maximum(name):
    """Forced maximum delays (a delay table with all its mass at k_max): the
    buffer points extrapolate from the oldest levels the ring keeps at every
    step after the start-up clamp.  The AT schemes are built to take that
    (Sec. 2.2); the run matches the oracle and the delay log shows k_max."""
    if name == "advdiff":
        pb, u0 = W.advdiff(n=1024, pe_size=32, order=4, mode="at", k_max=3, seed=31, cfl=0.05, dist="table",
                           prob=[0.0, 0.0, 0.0, 1.0])
    elif name == "rns":
        pb, u0 = W.rns(case="flame", n=1536, pe_size=64, mode="at", k_max=4, seed=32, dt=0.003, dist="table",
                       prob=[0.0, 0.0, 0.0, 0.0, 1.0])
    else:
        pb, u0 = W.entropy_wave(n=960, pe_size=96, mode="at", k_max=4, seed=33, dist="table",
                                prob=[0.0, 0.0, 0.0, 0.0, 1.0])
    s, _ = parity(pb, u0, 60, what="all delays at k_max, %s" % name)
    assert (s.read_delays() == pb["k_max"]).all()


@pytest.mark.parametrize("path", ["stage", "persistent"])
def test_homogeneous_ignition_at_error_stays_at_pe_edges(path):
    """The separable AT-error check on the GPU: a homogeneous igniting gas
    under AT equals the synchronous run bit for bit while the start-up clamp
    holds every delay at 0 (steps 0..q), then, at the first delayed step,
    moves only within S H points of a PE edge; and it matches the oracle."""
    from paper_2204_01133_gb300.api import Solver
    prm = W.rns_prm()
    n, B, T0, q, S, H = 128, 32, 6.0, 3, 4, 3
    rho = 1.0 / T0
    u0 = W.rns_conserved(np.full(n, rho), np.zeros(n), np.full(n, T0), np.ones(n), prm)

    def pb(mode):
        return W.base_problem(pde="rns", order=6, rk="rk4", n=n, pe_size=B, dx=1.0, dt=0.08, prm=prm, mode=mode,
                              k_max=2, dist="table", prob=[0.0, 0.0, 1.0])
    at, sync = Solver(pb("at"), u0, path=path), Solver(pb("sync"), u0, path=path)
    at.run(q + 1)
    sync.run(q + 1)
    assert np.array_equal(at.read_state(), sync.read_state())
    at.run(1)
    sync.run(1)
    dev = np.abs(at.read_state() - sync.read_state()).max(axis=0)
    j = np.arange(n) % B
    dist = np.minimum(j, B - 1 - j)
    assert (dev[dist >= S * H] == 0.0).all()
    assert (dev[dist < H] > 1e-13).all()
    parity(pb("at"), u0, q + 2, what="homogeneous ignition AT, %s" % path)

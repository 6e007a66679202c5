"""Reading A of the stage history on the GPU (AT_OPT_HISTORY =
AT_HIST_RECOMPUTE): a buffer point of stage s at a delayed level m reads the
neighbour's stage values formed again from its u^m (Sec. 2.3), recomputed by
a kernel on a strip around every PE boundary after each step, instead of
the stage arguments the neighbour computed.  Checked against the oracle's
reading A (per-variable bounds of test_gpu_parity), bit for bit against
reading B when no delay occurs, and refused where it is not built."""
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


def _a(pb):
    return dict(pb, history="recompute")


@pytest.mark.parametrize("case", ["advdiff-config0", "advdiff-as-order6-rk3", "advdiff-order2-rk2-pe16",
                                  "rns-flame", "rns-ignition-order4", "advdiff-one-pe"])
def test_reading_a_matches_the_oracle(case):
    if case == "advdiff-config0":
        pb, u0 = W.advdiff(n=2048, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075)
        steps = 2000
    elif case == "advdiff-as-order6-rk3":
        pb, u0 = W.advdiff(n=960, pe_size=48, order=6, mode="as", k_max=3, seed=2, cfl=0.01, rk="rk3tvd")
        steps = 300
    elif case == "advdiff-order2-rk2-pe16":
        pb, u0 = W.advdiff(n=512, pe_size=16, order=2, mode="at", k_max=2, seed=5, cfl=0.04, rk="rk2",
                           per_stage=0)
        steps = 300
    elif case == "rns-flame":
        pb, u0 = W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
        steps = 150
    elif case == "rns-ignition-order4":
        pb, u0 = W.rns(case="ignition", n=1536, pe_size=48, order=4, mode="at", k_max=3, seed=3, dt=0.003)
        steps = 150
    else:  # one PE, its own neighbour: the strip wraps around the whole domain
        pb, u0 = W.advdiff(n=64, pe_size=64, order=4, mode="at", k_max=3, seed=9, cfl=0.05)
        steps = 200
    s, _ = parity(_a(pb), u0, steps, what="reading A " + case)
    assert s.stats().path == 1  # the per-stage path


@pytest.mark.parametrize("maker", ["advdiff", "rns"])
def test_reading_a_without_delays_is_reading_b_bitwise(maker):
    from paper_2204_01133_gb300.api import Solver
    for kw in (dict(mode="sync"), dict(mode="at", k_max=0)):
        if maker == "advdiff":
            pb, u0 = W.advdiff(n=2048, pe_size=64, seed=0, cfl=0.075, **kw)
        else:
            pb, u0 = W.rns(case="flame", n=2048, pe_size=64, seed=0, dt=0.003, **kw)
        a = Solver(_a(pb), u0)
        b = Solver(pb, u0, path="stage")
        a.run(60)
        b.run(60)
        assert np.array_equal(a.read_state(), b.read_state()), (maker, kw)
    pb, u0 = (W.advdiff(n=2048, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075) if maker == "advdiff" else
              W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003))
    a, b = Solver(_a(pb), u0), Solver(pb, u0, path="stage")
    a.run(60)
    b.run(60)
    assert not np.array_equal(a.read_state(), b.read_state())
    assert np.array_equal(a.read_delays(), b.read_delays())


def test_reading_a_split_runs_and_restart():
    """Split at_step calls and a second at_set_delays (which restarts the
    run at level 0) give the same values as one call."""
    from paper_2204_01133_gb300.api import Solver
    pb, u0 = W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=1, dt=0.003)
    a = Solver(_a(pb), u0)
    a.run(80)
    b = Solver(_a(pb), u0)
    for k in (1, 2, 37, 40):
        b.run(k)
    assert np.array_equal(a.read_state(), b.read_state())
    b.set_problem(u0)
    b.set_delays()
    b.run(80)
    assert np.array_equal(a.read_state(), b.read_state())


def test_reading_a_is_refused_where_it_is_not_built():
    from paper_2204_01133_gb300 import api
    pb, u0 = W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
    s = api.Solver(_a(pb), u0, path="persistent")
    with pytest.raises(api.AtError) as ei:
        s.run(1)
    assert ei.value.code == api.AT_EINVAL
    pb, u0 = W.detonation(n=2048, pe_size=256, mode="at", k_max=4, seed=0)
    s = api.Solver(_a(pb), u0)
    with pytest.raises(api.AtError) as ei:
        s.run(1)
    assert ei.value.code == api.AT_EINVAL
    with pytest.raises(api.AtError):
        s.set_option(api.OPT_HISTORY, 2)

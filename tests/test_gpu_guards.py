"""Canary zones of the workspace (at_check_guards): after runs on every path
(per-stage, persistent, one-cluster, step-fused, tile-fused, reading A,
arrival-order delays, a stage-by-stage PE range with outside windows, a
checkpoint restore) no kernel has written past its slice of the workspace;
a write over the zones is reported as AT_ECORRUPT."""
import numpy as np
import pytest

from paper_2204_01133_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2204_01133_gb300 import build
    build.build()


CASES = {
    "rns-stage": (lambda: W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=6, dt=0.003), "stage"),
    "rns-persistent": (lambda: W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=6, dt=0.003),
                       "persistent"),
    "rns-tile-fused": (lambda: W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=6, dt=0.003),
                       "fused"),
    "rns-reading-a": (lambda: (lambda pb, u: (dict(pb, history="recompute"), u))(
        *W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=6, dt=0.003)), "auto"),
    "advdiff-cluster": (lambda: W.advdiff(n=2048, pe_size=64, mode="at", k_max=3, seed=6, cfl=0.075), "persistent"),
    "advdiff-fused": (lambda: W.advdiff(n=16384, pe_size=64, mode="at", k_max=3, seed=6, cfl=0.075), "fused"),
    "advdiff-stage-warp": (lambda: W.advdiff(n=16384, pe_size=64, mode="at", k_max=3, seed=6, cfl=0.075), "stage"),
    "detonation-stage": (lambda: W.detonation(n=4096, pe_size=256, mode="at", k_max=4, seed=6), "stage"),
    "detonation-tile-fused": (lambda: W.detonation(n=4096, pe_size=256, mode="at", k_max=4, seed=6), "fused"),
    "weno-interp": (lambda: W.adv_weno(n=256, pe_size=16, mode="at", k_max=2, seed=6, weno="interpolate"), "auto"),
    "prime-window": (lambda: W.entropy_wave(n=1021 * 2, pe_size=1021, mode="at", k_max=3, seed=6), "stage"),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_no_kernel_writes_past_its_slice(name):
    from paper_2204_01133_gb300.api import Solver
    make, path = CASES[name]
    pb, u0 = make()
    s = Solver(pb, u0, path=path)
    s.check_guards()
    s.run(7)
    s.run(13)
    s.check_guards()
    blob = s.checkpoint()
    s.run(5)
    s.restore(blob)
    s.run(3)
    s.check_guards()


def test_arrival_order_and_a_pe_range_keep_the_zones():
    from paper_2204_01133_gb300 import api
    pb, u0 = W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=6, dt=0.003)
    s = api.Solver(pb, u0, path="persistent")
    s.set_option(api.OPT_ARRIVAL, 1)
    s.run(20)
    s.check_guards()
    # a range of PEs of a larger domain, advanced stage by stage with outside windows
    P, B = pb["n"] // pb["pe_size"], pb["pe_size"]
    sub = dict(pb, n=8 * B, pe_base=4, pe_total=P, open_ends=1)
    r = api.Solver(sub, u0[:, 4 * B:12 * B], path="stage")
    H, nv = r.halo, 4
    rng = np.random.default_rng(0)
    for n in range(3):
        for st in range(4):
            for side in (0, 1):
                for lev in range(max(0, n - 4), n + 1):
                    r.put_ext(lev, st, side, 1.0 + 1e-3 * rng.standard_normal((H, nv)))
            r.stage()
    r.check_guards()


def test_an_overwritten_zone_is_reported():
    from paper_2204_01133_gb300 import api
    pb, u0 = W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=6, dt=0.003)
    s = api.Solver(pb, u0)
    s.run(3)
    s.check_guards()
    s.ws.fill_(0)  # a write over the whole workspace reaches every zone
    with pytest.raises(api.AtError) as ei:
        s.check_guards()
    assert ei.value.code == api.AT_ECORRUPT
    assert "canary" in str(ei.value)

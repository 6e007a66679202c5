"""The fixed shock bounds of the GPU parity tests against the conditioning
they stand for (CPU only).

WENO-JS with an absolute eps of 1e-6 is ill-conditioned near shocks: the
oracle drifts from itself when its initial state is perturbed by 1e-15.
Every fixed bound of a detonation case must stay between 10 and 40 times
that measured drift, so a bound can neither hide a real discrepancy behind
slack nor sit so close to the round-off level that a correct kernel fails.
The smooth-flow bounds (1e-12 per step, 1e-10 per run) need no such check:
there the drift is at round-off level.
"""
import numpy as np
import pytest

import parity


@pytest.fixture(scope="module")
def drifts():
    return {name: (parity.self_drift(pb, u0, steps, cols=cols), steps)
            for name, pb, u0, steps, cols in parity.shock_cases()}


def test_every_shock_case_has_a_bound(drifts):
    assert set(drifts) == set(parity.DET_RUN)


def test_run_bounds_are_20x_the_measured_drift(drifts):
    for name, ((_, en), steps) in drifts.items():
        ratio = parity.DET_RUN[name] / en.max()
        print("%s: %d steps, drift %.2e, bound %.1e (%.1fx)" % (name, steps, en.max(), parity.DET_RUN[name], ratio))
        assert 10.0 <= ratio <= 40.0, (name, ratio)


def test_step_bounds_are_20x_the_measured_drift(drifts):
    e1 = np.max([d[0][0] for d in drifts.values()], axis=0)
    ratio = np.asarray(parity.DET_STEP) / e1
    print("one-step drift per variable %s, bounds %s" % (e1, parity.DET_STEP))
    assert np.all((ratio >= 10.0) & (ratio <= 40.0)), ratio


def test_smooth_cases_drift_at_round_off():
    """The reacting flame and advection-diffusion drift at round-off level,
    so the plain 1e-12 / 1e-10 bounds hold with orders of magnitude to spare."""
    from paper_2204_01133_gb300 import workloads as W
    for pb, u0, steps in [
            W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003) + (100,),
            W.advdiff(n=2048, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075) + (500,)]:
        e1, en = parity.self_drift(pb, u0, steps)
        assert e1.max() < 1e-14 and en.max() < 1e-12, (pb["pde"], e1, en)


def test_momentum_scale_has_the_sound_speed_floor():
    """At rest (rho u = 0 everywhere) the momentum scale is max rho c."""
    from paper_2204_01133_gb300 import workloads as W
    pb, u0 = W.rns(case="ignition", n=256, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
    sc = parity.scales(pb, u0)
    rho, p = u0[0], u0[0] * 3.0 * (1.0 + 0.01 * np.exp(-((np.arange(256) - 128.0) / 12.8) ** 2))
    assert np.isclose(sc[1], np.sqrt(1.4 * p * rho).max(), rtol=1e-12)
    assert sc[0] == np.abs(u0[0]).max() and sc[2] == np.abs(u0[2]).max()

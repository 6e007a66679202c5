"""Checkpoint / resume (at_checkpoint_bytes, at_save, at_restore): a blob
taken between two steps, loaded into a new context with the same problem
and delay model, continues exactly as the run that saved it, bit for bit
(state and delay log), on every path and with reading A of the stage
history; a context can also be rewound to an earlier blob.  Blobs of
another problem, another delay model or other history options, truncated
blobs and foreign bytes are refused with AT_EINVAL and change nothing."""
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


def _case(name):
    if name == "rns":
        return W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=4, dt=0.003)
    if name == "rns-reading-a":
        pb, u0 = W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=4, dt=0.003)
        return dict(pb, history="recompute"), u0
    if name == "advdiff":
        return W.advdiff(n=8192, pe_size=64, mode="at", k_max=3, seed=4, cfl=0.075)
    return W.detonation(n=4096, pe_size=256, mode="at", k_max=4, seed=4)


@pytest.mark.parametrize("name,path", [("rns", "stage"), ("rns", "persistent"), ("rns", "fused"),
                                       ("advdiff", "fused"), ("advdiff", "persistent"), ("detonation", "stage"),
                                       ("detonation", "fused"), ("rns-reading-a", "auto")])
@pytest.mark.parametrize("device_blob", [False, True])
def test_resume_continues_bit_for_bit(name, path, device_blob):
    from paper_2204_01133_gb300.api import Solver
    pb, u0 = _case(name)
    a = Solver(pb, u0, path=path)
    a.run(17)
    blob = a.checkpoint(device=device_blob)
    a.run(23)
    ref_state, ref_delays = a.read_state(), a.read_delays()
    b = Solver(pb, u0, path=path)  # a fresh context at level 0
    b.run(3)
    b.restore(blob)
    assert b.stats().level == 17
    b.run(23)
    assert np.array_equal(b.read_state(), ref_state)
    assert np.array_equal(b.read_delays(), ref_delays)
    # rewinding the first context to the blob replays the same steps
    a.restore(blob)
    a.run(23)
    assert np.array_equal(a.read_state(), ref_state)


def test_resume_on_another_path():
    """The blob is path-independent: saved on the persistent path, resumed on
    the per-stage path (all paths compute the same values)."""
    from paper_2204_01133_gb300.api import Solver
    pb, u0 = _case("rns")
    a = Solver(pb, u0, path="persistent")
    a.run(11)
    blob = a.checkpoint()
    a.run(9)
    b = Solver(pb, u0, path="stage")
    b.restore(blob)
    b.run(9)
    assert np.array_equal(b.read_state(), a.read_state())


def test_foreign_blobs_are_refused():
    from paper_2204_01133_gb300 import api
    pb, u0 = _case("rns")
    a = api.Solver(pb, u0)
    a.run(5)
    blob = a.checkpoint()
    st = a.read_state()
    for bad in (dict(pb, seed=pb["seed"] + 1), dict(pb, dt=pb["dt"] * 1.5), dict(pb, k_max=3),
                dict(pb, history="recompute")):
        b = api.Solver(bad, u0)
        b.run(2)
        before = b.read_state()
        with pytest.raises(api.AtError) as ei:
            b.restore(blob)
        assert ei.value.code == api.AT_EINVAL, bad
        assert np.array_equal(b.read_state(), before)
    with pytest.raises(api.AtError) as ei:
        a.restore(blob[:-8])
    assert ei.value.code == api.AT_EINVAL
    junk = blob.copy()
    junk[:8] = 0
    with pytest.raises(api.AtError) as ei:
        a.restore(junk)
    assert ei.value.code == api.AT_EINVAL
    assert np.array_equal(a.read_state(), st)

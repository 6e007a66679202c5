"""The allocation-free entry point at_run_noalloc, through the C ABI.

It serves callers that cannot allocate device memory while they run (a host
that hands out a fixed device-memory budget at startup, or a path where
cudaMalloc's implicit synchronisation or late failure is not acceptable):
its workspace is the library's fixed device scratch array.  It runs the same
kernels on the same delay stream as the regular context path (at_set_problem
+ at_set_delays + at_run with a caller workspace), so its result must equal
that path's bit for bit, on calls in a row that reuse the shared array (a
stale ring, delay log or status word left by the previous call would show),
and oversized problems must be refused before anything runs.  It is also
checked against the oracle directly.  This file is collected last on
purpose.
"""
import numpy as np
import pytest

from paper_2204_01133_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2204_01133_gb300 import build
    build.build()
    return torch


def _regular(pb, init, steps):
    from paper_2204_01133_gb300.api import Solver
    s = Solver(pb, init)
    s.run(steps)
    return s.read_state()


def _noalloc(torch, pb, init, steps):
    from paper_2204_01133_gb300 import api
    state = torch.from_numpy(np.ascontiguousarray(init)).to("cuda")
    api.run_noalloc(pb, state, steps)
    torch.cuda.synchronize()
    return state.cpu().numpy()


def test_noalloc_matches_context_path_on_calls_in_a_row(torch_cuda):
    from paper_2204_01133_gb300 import api
    cases = [
        W.rns(case="flame", n=16384, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003) + (60,),
        W.rns(case="flame", n=16384, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003) + (60,),
        W.advdiff(n=2048, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075) + (500,),
    ]
    for pb, init, steps in cases:
        assert api.workspace_bytes(pb) <= api.NOALLOC_SCRATCH_BYTES
        ref = _regular(pb, init, steps)
        got = _noalloc(torch_cuda, pb, init, steps)
        assert np.array_equal(got, ref), (pb["pde"], np.abs(got - ref).max())


def test_noalloc_refuses_problems_above_its_scratch(torch_cuda):
    from paper_2204_01133_gb300 import api
    pb, init = W.rns(case="flame", n=1 << 18, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003)
    assert api.workspace_bytes(pb) > api.NOALLOC_SCRATCH_BYTES
    state = torch_cuda.from_numpy(np.ascontiguousarray(init)).to("cuda")
    before = state.clone()
    with pytest.raises(api.AtError) as ei:
        api.run_noalloc(pb, state, 1)
    assert ei.value.code == api.AT_ENOMEM
    assert "workspace" in str(ei.value)
    torch_cuda.cuda.synchronize()
    assert torch_cuda.equal(state, before)  # nothing ran


def test_noalloc_matches_the_oracle(torch_cuda):
    """The allocation-free run against the oracle itself, at the per-variable
    bounds of the parity tests (1e-10 after the run)."""
    import oracle
    from parity import TOL_RUN, check
    for pb, init, steps in [W.advdiff(n=2048, pe_size=64, mode="at", k_max=3, seed=5, cfl=0.075) + (400,),
                            W.rns(case="flame", n=2048, pe_size=64, mode="at", k_max=4, seed=5, dt=0.003) + (60,)]:
        got = _noalloc(torch_cuda, pb, init, steps)
        o = oracle.Oracle(pb, init)
        assert o.run(steps) == 0
        check(pb, got, o.state(), TOL_RUN, "noalloc %s step %d" % (pb["pde"], steps))

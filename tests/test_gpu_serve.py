"""Serving: continuous batching admits requests as they arrive, within a
device-memory budget, overlaps their work on the device, and every result
is bit-for-bit the one the request gets when solved alone; one request of
each problem type, served in the mix, is checked against the CPU oracle."""
import numpy as np
import pytest

import oracle
from parity import DET_RUN, SERVE_DET, TOL_RUN, check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2204_01133_gb300 import build
    build.build()


def small_stream(n=14, seed=5, rate=60.0):
    from paper_2204_01133_gb300 import workloads as W
    s = W.serving_stream(rate=rate, duration=10.0, seed=seed, n_min=600, n_max=6000, steps_min=20, steps_max=90,
                         max_requests=n)
    return s


def alone(r):
    from paper_2204_01133_gb300 import workloads as W
    from paper_2204_01133_gb300.api import Solver
    pb, init = W.serving_request(r.kind, r.n, r.seed, instance=r.id)
    s = Solver(pb, init, path="stage")
    s.run(r.steps)
    return s.read_state()


@pytest.mark.parametrize("budget_mb,mode,big", [(4096, 1, None), (4096, 0, 2048), (3, 1, 2048)])
def test_served_results_equal_alone(budget_mb, mode, big):
    """All requests as slots of a flat-mode batch; or big requests (above
    2,048 points) on their own context on a side stream and the others as
    slots.  With a 3 MB budget only a few requests fit at once, so most wait
    for memory to free up."""
    from paper_2204_01133_gb300.serve import Server, summarize
    srv = Server(mem_budget=budget_mb << 20, capacity=8, chunk=13, big_points=big, keep_states=True, mode=mode)
    peak = []
    orig_admit = srv._admit

    def admit(r, now):
        orig_admit(r, now)
        peak.append(srv.used)
    srv._admit = admit
    done, elapsed = srv.run(small_stream(rate=2000.0 if budget_mb < 10 else 60.0))
    assert len(done) == 14 and srv.pending_left == 0
    assert max(peak) <= srv.budget
    kinds = {(r.n > 2048) for r in done}
    assert kinds == {True, False}       # both sizes were served
    for r in done:
        assert r.finish >= r.admit >= r.arrival
        assert np.array_equal(np.asarray(r.state), alone(r)), (r.id, r.kind, r.n)
    s = summarize(done, elapsed)
    assert s["completed"] == 14 and s["latency_p99_s"] >= s["latency_p50_s"] > 0
    if budget_mb < 10:
        assert any(r.admit - r.arrival > 0.01 for r in done)  # memory made some wait


def test_plain_path_matches_too():
    from paper_2204_01133_gb300.serve import serve_plain
    done, _ = serve_plain(small_stream(n=5, seed=9), keep_states=True)
    for r in done:
        assert np.array_equal(np.asarray(r.state), alone(r))


@pytest.mark.parametrize("mode,big", [(1, None), (0, 2600)])
def test_served_requests_match_the_oracle(mode, big):
    """One request of each type at its rounded size (advection-diffusion
    2,944 points, reacting flame 2,496, detonation 2,560), arriving together:
    all as slots of the flat batch, or the two larger ones on contexts of
    their own beside the batch.  Each result against the oracle run of the
    same request; the detonation takes its fixed shock bound."""
    from paper_2204_01133_gb300 import workloads as W
    from paper_2204_01133_gb300.serve import Server
    stream = SERVE_ORACLE_STREAM
    srv = Server(mem_budget=1 << 30, capacity=4, chunk=17, big_points=big, keep_states=True, mode=mode)
    done, _ = srv.run([dict(d) for d in stream])
    assert len(done) == 3
    for r in done:
        pb, init = W.serving_request(r.kind, r.n, r.seed, instance=r.id)
        o = oracle.Oracle(pb, init)
        assert o.run(r.steps) == 0
        tol = DET_RUN["serve"] if r.kind == "detonation" else TOL_RUN
        check(pb, np.asarray(r.state), o.state(), tol, "served %s n=%d" % (r.kind, r.n))


SERVE_ORACLE_STREAM = [
    {"id": 0, "arrival": 0.0, "kind": "advdiff", "n": 3000, "steps": 60, "seed": 11},
    {"id": 1, "arrival": 0.0005, "kind": "rns", "n": 2500, "steps": 60, "seed": 12},
    {"id": SERVE_DET[2], "arrival": 0.001, "kind": "detonation", "n": SERVE_DET[0], "steps": SERVE_DET[3],
     "seed": SERVE_DET[1]},
]

"""Serving: continuous batching admits requests as they arrive, within a
device-memory budget, overlaps their work on the device, and every result
is bit-for-bit the one the request gets when solved alone."""
import numpy as np
import pytest

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

"""The named benchmark configurations (paper_2204_01133_gb300/configs.json):
each builds, with the sizes its description states, and the single-solve
ones give the same problem and initial state as the bench workload they
name (so a user's config and the measured one are the same thing)."""
import numpy as np
import pytest

from paper_2204_01133_gb300 import workloads as W


def test_every_configuration_is_listed():
    assert W.config_names() == ["config0-advdiff", "config1-flame", "config1-ignition", "config2-batched",
                                "config3-detonation", "config4-serving"]


@pytest.mark.parametrize("name,n,pes,steps", [("config0-advdiff", 2048, 32, 10000), ("config1-flame", 16384, 256, 1000),
                                              ("config1-ignition", 16384, 256, 1000)])
def test_single_solves_match_the_bench_workloads(name, n, pes, steps):
    import bench
    (pb, u0), st = W.config(name)
    assert pb["n"] == n and pb["n"] // pb["pe_size"] == pes and st == steps
    kind, (pb2, u2) = bench.build_workload(W._configs()[name]["bench_workload"])
    assert pb == pb2
    assert np.array_equal(u0, u2)


def test_detonation_configuration():
    c = W._configs()["config3-detonation"]
    assert c["kwargs"]["n"] == 1 << 24 and c["kwargs"]["pe_size"] == 1024 and c["steps"] == 100
    import bench
    assert bench.WORKLOADS[c["bench_workload"]]["n"] == c["kwargs"]["n"]
    # the builder itself, at a size the CPU makes in an instant
    pb, u0 = W.detonation(**dict(c["kwargs"], n=1 << 14))
    assert pb["pe_size"] == 1024 and u0.shape == (4, 1 << 14) and np.isfinite(u0).all()


def test_batched_and_serving_configurations():
    batch, steps = W.config("config2-batched")
    assert len(batch) == 4096 and steps == 200
    pts = sum(pb["n"] for pb, _, _ in batch)
    assert 8.5e6 < pts < 1.05e7                      # ~9.4 M points
    assert {pb["pe_size"] for pb, _, _ in batch} == {32, 64}
    reqs, steps = W.config("config4-serving")
    assert len(reqs) == 48 and steps is None
    assert {r["kind"] for r in reqs} == {"advdiff", "rns", "detonation"}
    assert all(100 <= r["steps"] <= 5000 and 512 <= r["n"] <= 262144 for r in reqs)

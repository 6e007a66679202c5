"""The stage kernels' own exponential (Tang's table-driven method, 256
entries) and reciprocals (two Newton steps, or one cubic step, from the
hardware approximation), against the host C library and CUDA, through
libat_probe.so."""
import ctypes
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def probe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2204_01133_gb300 import build
    build.build()
    L = ctypes.CDLL(os.path.join(os.path.dirname(build.__file__), "libat_probe.so"))
    L.at_probe_fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
    L.at_probe_fn.restype = ctypes.c_int

    def run(x, which):
        xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to("cuda")
        yd = torch.empty_like(xd)
        assert L.at_probe_fn(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), xd.numel(),
                             which) == 0
        return yd.cpu().numpy()
    return run


def _inputs():
    rng = np.random.default_rng(7)
    ln2_512 = math.log(2.0) / 512.0  # half a table step: where the reduction rounds to a tie
    k = np.arange(-16000, 16001, dtype=np.float64)
    return np.concatenate([
        rng.uniform(-60.0, 0.0, 1 << 20),        # Arrhenius exponents -Ea/T
        rng.uniform(-708.0, 709.0, 1 << 18),     # the whole normal range
        rng.uniform(-1e-3, 1e-3, 1 << 14),
        k * ln2_512, np.nextafter(k * ln2_512, np.inf), np.nextafter(k * ln2_512, -np.inf),  # reduction ties
        [0.0, -0.0, 1e-300, -1e-300, 511.999, -511.999, 512.0, -512.0],
    ])


def test_table_exp_within_two_ulp_of_libm(probe):
    x = _inputs()
    got = probe(x, 0)
    ref = np.array([math.exp(v) for v in x])
    ulps = np.abs(got - ref) / np.spacing(ref)
    assert np.isfinite(got).all()
    assert ulps.max() <= 2.0, (ulps.max(), x[np.argmax(ulps)])


def test_table_exp_matches_cuda_exp_outside_fast_path(probe):
    x = np.array([-746.0, -745.0, -740.0, -720.0, -600.0, -512.0, 512.0, 700.0, 709.7, 710.0,
                  np.inf, -np.inf, np.nan])
    got, cuda = probe(x, 0), probe(x, 1)
    np.testing.assert_array_equal(got, cuda)
    near = probe(_inputs(), 1)
    assert (np.abs(probe(_inputs(), 0) - near) / np.spacing(near)).max() <= 3.0


@pytest.mark.parametrize("which", [2, 4], ids=["two-quadratic-steps", "one-cubic-step"])
def test_newton_reciprocal_within_one_ulp(probe, which):
    rng = np.random.default_rng(3)
    x = np.concatenate([
        np.exp(rng.uniform(np.log(1e-6), np.log(1e6), 1 << 20)),   # densities, pressures, weight sums
        -np.exp(rng.uniform(np.log(1e-3), np.log(1e3), 1 << 16)),
        2.0 ** np.arange(-60, 61), np.nextafter(2.0 ** np.arange(-60, 61), 0.0),
        1.0 + np.arange(1, 4097) * 2.0 ** -52, 2.0 - np.arange(1, 4097) * 2.0 ** -52,
    ])
    x = np.concatenate([x, np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 1 << 18))])  # WENO weight sums
    got = probe(x, which)
    ref = 1.0 / x                      # IEEE division on the host: correctly rounded
    assert np.array_equal(probe(x, 3), ref)
    ulps = np.abs(got - ref) / np.spacing(np.abs(ref))
    assert ulps.max() <= 1.0, (ulps.max(), x[np.argmax(ulps)])

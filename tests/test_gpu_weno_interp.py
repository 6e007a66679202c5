"""The WENO interpolation form on the GPU (at_problem.weno =
AT_WENO_INTERPOLATE): edge values of the split fluxes by the interpolants of
Eq. interpS with ideal weights {1/16, 5/8, 5/16} (Eqs. fullSten, omg),
differenced by the fourth-order staggered formula, halo 4, against the
oracle's interpolation form with the per-variable bounds of
test_gpu_parity (the detonation with its fixed shock bound)."""
import pytest

from paper_2204_01133_gb300 import workloads as W
from parity import DET_CASES, DET_RUN, DET_STEP
from test_gpu_parity import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2204_01133_gb300 import build
    build.build()


@pytest.mark.parametrize("mode", ["sync", "as", "at"])
def test_scalar_advection(mode):
    pb, u0 = W.adv_weno(n=512, pe_size=32, mode=mode, k_max=3, seed=4, dt_coef=2.0, weno="interpolate")
    parity(pb, u0, 100, what="interp adv " + mode)


def test_burgers():
    pb, u0 = W.burgers(n=1024, pe_size=64, mode="at", k_max=3, seed=6, dt_coef=1.0, weno="interpolate")
    parity(pb, u0, 150, what="interp burgers")


@pytest.mark.parametrize("pe_size,n", [(64, 512), (96, 768), (1024, 4096)])
def test_entropy_wave(pe_size, n):
    """Reactive Euler in smooth flow (a density wave at constant u and p);
    PEs of 64, 96 (one window that is not a power of two) and 1024 (four
    windows of 256)."""
    pb, u0 = W.entropy_wave(n=n, pe_size=pe_size, mode="at", k_max=3, seed=2, weno="interpolate")
    parity(pb, u0, 100, what="interp entropy wave B=%d" % pe_size)


def test_detonation():
    kw, steps = DET_CASES["interp"]
    pb, u0 = W.detonation(**kw)
    parity(pb, u0, steps, first_tol=DET_STEP, run_tol=DET_RUN["interp"], what="interp detonation")


def test_interpolation_form_is_refused_in_batches():
    from paper_2204_01133_gb300 import api
    from paper_2204_01133_gb300.batch import Batch
    pb, u0 = W.adv_weno(n=512, pe_size=32, mode="at", k_max=3, seed=4, dt_coef=2.0, weno="interpolate")
    b = Batch(capacity=2)
    with pytest.raises(api.AtError) as ei:
        b.bind(0, pb, u0, 10)
    assert ei.value.code == api.AT_EINVAL

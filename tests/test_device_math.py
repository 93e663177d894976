"""The kernels' table-driven fp64 exp / log (Tang's methods) against the CUDA library
and the host's libm, on the GPU through chem_diag_math: at most 2 ulp apart over the
argument ranges the integrator uses."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def ulps(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.spacing(np.maximum(np.abs(a), np.abs(b)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_02602_gb300 import build, chem
    build.build()
    return chem


def _dev(x):
    import torch
    return torch.tensor(x, dtype=torch.float64, device="cuda")


def test_exp_matches_library(lib):
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.uniform(-700, 700, 200000), rng.uniform(-5, 5, 200000),
                        np.linspace(-1, 1, 4097), [0.0, 1.0, -1.0, 709.0, -707.0]])
    mine = lib.diag_math(0, _dev(x)).cpu().numpy()
    cuda = lib.diag_math(2, _dev(x)).cpu().numpy()
    assert ulps(mine, cuda).max() <= 2.0
    assert ulps(mine, np.exp(x)).max() <= 2.0
    assert mine[-5] == 1.0


def test_log_matches_library(lib):
    rng = np.random.default_rng(8)
    x = np.concatenate([np.exp(rng.uniform(-700, 700, 200000)), rng.uniform(0.5, 2.0, 200000),
                        rng.uniform(200.0, 6000.0, 100000), 1.0 + np.linspace(-1e-6, 1e-6, 2001),
                        [1.0, 2.0, 0.5, 1500.0]])
    mine = lib.diag_math(1, _dev(x)).cpu().numpy()
    cuda = lib.diag_math(3, _dev(x)).cpu().numpy()
    ref = np.log(x)
    nz = ref != 0.0
    assert ulps(mine[nz], cuda[nz]).max() <= 2.0
    assert ulps(mine[nz], ref[nz]).max() <= 2.0
    assert mine[-4] == 0.0

"""The kernels' device math on the GPU through chem_diag_math: the table-driven fp64
exp / log (Tang's methods) against the CUDA library and the host's libm (at most 2 ulp
apart over the argument ranges the integrator uses); the Newton-Raphson reciprocals
against exact division; the integer-pipe fp32 <-> fp64 conversions and the 2^-12-grid
hi/lo split against their IEEE-754 definitions (numpy's round-to-nearest-even)."""
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


def test_reciprocals(lib):
    """rcp2 within 2 ulp of the exact 1/x; the hardware approximation within 2^-19
    relative, one Newton-Raphson step (rcp1) within 2^-38: each step squares the error."""
    rng = np.random.default_rng(9)
    x = np.concatenate([np.exp(rng.uniform(-690, 690, 200000)), -np.exp(rng.uniform(-690, 690, 50000)),
                        rng.uniform(150.0, 6500.0, 100000), rng.uniform(1e-3, 1e4, 100000),
                        [1.0, 2.0, 0.5, 3.0, 1500.0, 1e-300, 1e300]])
    exact = 1.0 / x
    r2 = lib.diag_math(5, _dev(x)).cpu().numpy()
    r1 = lib.diag_math(4, _dev(x)).cpu().numpy()
    r0 = lib.diag_math(6, _dev(x)).cpu().numpy()
    assert ulps(r2, exact).max() <= 2.0
    e1 = np.abs(r1 / exact - 1.0).max()
    e0 = np.abs(r0 / exact - 1.0).max()
    assert e0 <= 2.0 ** -19, e0
    assert e1 <= 2.0 ** -38, e1
    assert e1 <= 2.0 * e0 * e0 + 2.0 ** -52


def _f32(x):
    """IEEE round-to-nearest-even fp64 -> fp32 (numpy), with magnitudes below the fp32
    normal range taken to signed zero."""
    with np.errstate(over="ignore"):
        f = np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)
    tiny = np.abs(np.asarray(x)) < 2.0 ** -126
    return np.where(tiny, np.copysign(0.0, x), f)


def test_fp64_to_fp32_conversion(lib):
    rng = np.random.default_rng(10)
    x = np.concatenate([
        rng.standard_normal(100000) * np.exp(rng.uniform(-80, 80, 100000)),
        np.exp(rng.uniform(-100, 100, 50000)) * rng.choice([-1.0, 1.0], 50000),
        # ties and near-ties: fp32 values plus half an fp32 ulp, and a hair either side
        *[(lambda f: f + 0.5 * np.spacing(f.astype(np.float32)).astype(np.float64) * s)(
            rng.uniform(1.0, 2.0, 20000).astype(np.float32).astype(np.float64) * 2.0 ** rng.integers(-120, 120, 20000))
          for s in (1.0, 1.0 + 1e-12, 1.0 - 1e-12)],
        [0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38, 1e39, -1e300,
         2.0 ** -126, 2.0 ** -127, -1e-300, 1.1754942e-38],
    ])
    got = lib.diag_math(7, _dev(x)).cpu().numpy()
    want = _f32(x)
    same = (got == want) & (np.signbit(got) == np.signbit(want))
    assert same.all(), x[~same][:5]
    special = np.array([np.inf, -np.inf, np.nan])
    g = lib.diag_math(7, _dev(special)).cpu().numpy()
    assert g[0] == np.inf and g[1] == -np.inf and np.isnan(g[2])


def test_fp32_to_fp64_conversion(lib):
    rng = np.random.default_rng(11)
    f = np.concatenate([rng.standard_normal(100000) * np.exp(rng.uniform(-80, 80, 100000)),
                        [0.0, -0.0, 1.0, 2.0 ** -126, -(2.0 ** -126), 3.4028234663852886e38, 1e-45]])
    f = f.astype(np.float32).astype(np.float64)       # exact fp32 values
    got = lib.diag_math(8, _dev(f)).cpu().numpy()
    want = np.where(np.abs(f) < 2.0 ** -126, np.copysign(0.0, f), f)
    assert np.array_equal(got, want)
    g = lib.diag_math(8, _dev(np.array([np.inf, -np.inf, np.nan]))).cpu().numpy()
    assert g[0] == np.inf and g[1] == -np.inf and np.isnan(g[2])


def test_hilo_split(lib):
    """hi is x truncated toward zero to a multiple of 2^-12, exactly; hi + lo = x to 2^-37;
    signed sums of a few hi parts are exact in fp32."""
    rng = np.random.default_rng(12)
    x = np.concatenate([rng.uniform(-700.0, 700.0, 200000), rng.uniform(-1e-3, 1e-3, 20000),
                        rng.uniform(-4000.0, 4000.0, 20000), [0.0, 2.0 ** -12, -(2.0 ** -12), 1e-20, 1023.75]])
    hi = lib.diag_math(9, _dev(x)).cpu().numpy()
    lo = lib.diag_math(10, _dev(x)).cpu().numpy()
    assert np.array_equal(hi, np.trunc(x * 4096.0) / 4096.0)
    assert np.abs(hi + lo - x).max() <= 2.0 ** -37
    # the fp32 sum of hi parts of |x| < 1000 equals the exact sum
    h = hi[:200000].reshape(-1, 4)
    s32 = (((h[:, 0].astype(np.float32) - h[:, 1].astype(np.float32)) + h[:, 2].astype(np.float32))
           - h[:, 3].astype(np.float32))
    assert np.array_equal(s32.astype(np.float64), h[:, 0] - h[:, 1] + h[:, 2] - h[:, 3])


def test_fma_probe_is_plausible(lib):
    """chem_diag_fma_peak (the roofline denominators' probe): the fp64 rate is below the
    unit-count peak (152 SMs x 2 DFMA lanes x 2 flops x 2.07 GHz, a probe that did no work
    would exceed it) and above half of it; fp32 runs tens of times faster than fp64."""
    from paper_2506_02602_gb300 import roofline
    f64, _ = lib.fma_peak(0, 152 * 8, 256, 200)
    f32, _ = lib.fma_peak(1, 152 * 8, 256, 4000)
    assert 0.5 * roofline.FP64_PEAK_GFLOPS < f64 <= 1.02 * roofline.FP64_PEAK_GFLOPS, f64
    assert f32 > 20 * f64, (f32, f64)
    with pytest.raises(lib.ChemError):
        lib.fma_peak(2, 1, 32, 1)


def test_gelu_approximation_against_library_erf(lib):
    """The network's GELU and GELU' (erf by Abramowitz & Stegun 7.1.26, error <= 1.5e-7)
    against the same formulas with the CUDA library's erff / expf and against the exact
    values (math.erf, fp64): within 4e-7 absolute plus 4 fp32 ulps of the value, far
    inside the BF16 rounding (2^-8 relative) that follows them; negative tails keep their
    relative accuracy below BF16's (no cancellation of 1 + erf: 0.16 % at x = -5)."""
    import math
    x = np.concatenate([np.linspace(-9.0, 9.0, 200001), [0.0, -0.0, 1e-30, -1e-30]])
    xf = x.astype(np.float32).astype(np.float64)
    g = lib.diag_math(11, _dev(x)).cpu().numpy()
    gd = lib.diag_math(12, _dev(x)).cpu().numpy()
    g_lib = lib.diag_math(13, _dev(x)).cpu().numpy()
    gd_lib = lib.diag_math(14, _dev(x)).cpu().numpy()
    erf = np.vectorize(math.erf)
    Phi = 0.5 * (1.0 + erf(xf / math.sqrt(2.0)))
    g_ex = xf * Phi
    gd_ex = Phi + xf * np.exp(-0.5 * xf * xf) / math.sqrt(2.0 * math.pi)
    tol = lambda v: 4e-7 * np.maximum(1.0, np.abs(xf)) + 4 * np.spacing(np.abs(v).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(g - g_ex) <= tol(g_ex)), np.max(np.abs(g - g_ex))
    assert np.all(np.abs(gd - gd_ex) <= tol(gd_ex)), np.max(np.abs(gd - gd_ex))
    assert np.all(np.abs(g - g_lib) <= tol(g_ex) + np.abs(g_lib - g_ex))
    assert np.all(np.abs(gd - gd_lib) <= tol(gd_ex) + np.abs(gd_lib - gd_ex))
    # the negative tail: relative accuracy of GELU(-5) ~ -1.4e-6 below BF16's 2^-8
    i = np.argmin(np.abs(xf + 5.0))
    assert abs(g[i] - g_ex[i]) <= 2e-3 * abs(g_ex[i])

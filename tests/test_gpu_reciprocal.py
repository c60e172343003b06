"""The inverse density of the FP32 step kernels (lbm_reciprocal_fp32: the
hardware reciprocal approximation refined by one Newton-Raphson step) against
CUDA's correctly rounded 1/x and against its stated bounds,
|y x - 1| <= 2^-24 + 2^-40 for 2^-100 <= |x| <= 2^100 and <= 2^-23 out to
2^+-125, over densities of the paper's runs, log-uniform sweeps of both ranges
and the special values."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BOUND = 2.0 ** -24 + 2.0 ** -40


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _rcp(torch, x):
    from paper_1010_4135_gb300 import _abi as A
    d = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    y = torch.empty_like(d)
    st = torch.cuda.current_stream().cuda_stream
    assert A.lbm_reciprocal_fp32(ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(y.data_ptr()), d.numel(),
                                 ctypes.c_void_p(st)) == A.LBM_OK
    return d, y


@pytest.mark.parametrize("lo,hi,bound", [(0.05, 20.0, BOUND), (2.0 ** -100, 2.0 ** 100, BOUND),
                                         (2.0 ** -125, 2.0 ** 125, 2.0 ** -23)])
def test_within_the_bound_and_mostly_the_correctly_rounded_value(torch, lo, hi, bound):
    rng = np.random.default_rng(3)
    n = 1_000_001  # odd: the padded tail lane
    x = np.exp(rng.uniform(np.log(lo), np.log(hi), n)).astype(np.float32)
    x[::2] *= -1.0
    d, y = _rcp(torch, x)
    ref = (1.0 / d).cpu().numpy()  # CUDA's IEEE division, correctly rounded
    got = y.cpu().numpy()
    err = np.abs(got.astype(np.float64) * x.astype(np.float64) - 1.0)
    assert np.isfinite(got).all() and err.max() <= bound, err.max()
    # never further than the neighbouring float of the correctly rounded result
    ulps = np.abs(got.view(np.int32).astype(np.int64) - ref.view(np.int32).astype(np.int64))
    assert ulps.max() <= 1
    assert (ulps == 0).mean() > 0.99


def test_special_values(torch):
    x = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-40, 2.0 ** 127, 1.0, -4.0], dtype=np.float32)
    _, y = _rcp(torch, x)
    got = y.cpu().numpy()
    assert np.isnan(got[:6]).all()
    assert got[6] == 0.0 and got[7] == 1.0 and got[8] == -0.25


def test_empty_and_invalid_calls(torch):
    from paper_1010_4135_gb300 import _abi as A
    p = ctypes.c_void_p(256)
    assert A.lbm_reciprocal_fp32(None, None, 0, None) == A.LBM_OK
    assert A.lbm_reciprocal_fp32(p, p, -1, None) == A.LBM_EINVAL
    assert A.lbm_reciprocal_fp32(None, p, 4, None) == A.LBM_EINVAL

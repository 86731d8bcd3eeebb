"""The kernels' double-precision exponential (table-driven, after Tang 1989),
used for every Arrhenius factor and equilibrium constant, against the CUDA
math library's exp and the host's libm exp: at most 2 units in the last
place over the arguments the rate expressions produce, and the same
overflow / underflow / NaN behaviour."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2101_01702_gb300 import build
    build.build()
    from paper_2101_01702_gb300 import lbm as L
    return L


def _arguments():
    rng = np.random.default_rng(1989)
    ln2_64 = np.log(2.0) / 64
    k = rng.integers(-65000, 65000, 20000).astype(np.float64)
    parts = [
        rng.uniform(-706.0, 706.0, 400000),
        rng.uniform(-60.0, 60.0, 400000),                       # typical g/RT and rate arguments
        rng.uniform(-1e-3, 1e-3, 50000),
        k * ln2_64, np.nextafter(k * ln2_64, np.inf), np.nextafter(k * ln2_64, -np.inf),
        (k + 0.5) * ln2_64,                                      # halfway between table points
        np.array([0.0, -0.0, 1e-300, -1e-300, 5e-324, 1.0, -1.0, 706.99, -706.99, 707.0, -707.0,
                  709.7, -744.0, 710.0, -746.0, 1e4, -1e4]),
    ]
    return np.concatenate(parts)


def _ulps(a, b):
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_exponential_against_cuda_and_libm(lbm):
    import torch
    x = _arguments()
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    yr = torch.empty_like(xd)
    st = lbm.lbm_exp_check(xd.data_ptr(), y.data_ptr(), yr.data_ptr(), x.size,
                           torch.cuda.current_stream().cuda_stream)
    assert st == lbm.LBM_OK
    y, yr = y.cpu().numpy(), yr.cpu().numpy()
    with np.errstate(over="ignore"):          # exp(>709.8) is inf, as intended
        host = np.exp(x)
    finite = np.isfinite(host) & (host > 0)
    assert _ulps(y[finite], yr[finite]).max() <= 2.0
    assert _ulps(y[finite], host[finite]).max() <= 2.0
    # overflow, underflow and exact zero behave as the library's
    assert np.array_equal(np.isinf(y), np.isinf(yr))
    assert np.array_equal(y == 0.0, yr == 0.0)
    assert y[x == 0.0].tolist() == [1.0, 1.0]


def test_exponential_propagates_nan(lbm):
    import torch
    x = torch.tensor([float("nan"), 1.0], dtype=torch.float64, device="cuda")
    y, yr = torch.empty_like(x), torch.empty_like(x)
    assert lbm.lbm_exp_check(x.data_ptr(), y.data_ptr(), yr.data_ptr(), 2,
                             torch.cuda.current_stream().cuda_stream) == lbm.LBM_OK
    assert torch.isnan(y[0]).item() and not torch.isnan(y[1]).item()

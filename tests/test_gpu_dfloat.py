"""The FP32 modes' input split (rw_split_double): hi must be the IEEE
round-to-nearest-even float of x and lo the rounded remainder x - hi, checked
against NumPy's conversions on random doubles over the whole float range,
constructed ties, and the special values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2312_07440_gb300 import rwgt  # noqa: E402

DEV = torch.device("cuda", 0)


def split(x):
    dx = torch.from_numpy(np.ascontiguousarray(x, np.float64)).to(DEV)
    hi = torch.empty(dx.shape, dtype=torch.float32, device=DEV)
    lo = torch.empty_like(hi)
    rwgt.split_double(dx, hi, lo, torch.cuda.current_stream(DEV).cuda_stream)
    torch.cuda.synchronize()
    return hi.cpu().numpy(), lo.cpu().numpy()


def test_split_matches_ieee_conversion():
    rng = np.random.default_rng(7)
    n = 1 << 20
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-125, 127, n)
    x = np.ldexp(mant, expo) * rng.choice([-1.0, 1.0], n)
    # ties: a float plus exactly half its ulp, both parities of the kept part
    f = rng.uniform(1.0, 2.0, 4096).astype(np.float32) * np.float32(1000.0)
    ulp = np.spacing(f).astype(np.float64)
    ties = f.astype(np.float64) + 0.5 * ulp
    # momentum-like values: what the kernels actually split
    mom = rng.normal(scale=500.0, size=65536)
    x = np.concatenate([x, ties, -ties, mom])
    hi, lo = split(x)
    assert np.array_equal(hi, x.astype(np.float32))
    rem = (x - hi.astype(np.float64)).astype(np.float32)   # x - hi is exact in FP64
    big = np.abs(x) >= 2.0 ** -74
    assert np.array_equal(lo[big], rem[big])
    err = np.abs(hi.astype(np.float64) + lo.astype(np.float64) - x)
    assert np.all(err[big] <= 2.0 ** -48 * np.abs(x[big]))


def test_split_special_values():
    tiny = 2.0 ** -130
    x = np.array([0.0, -0.0, tiny, -tiny, 2.0 ** 130, -(2.0 ** 130), np.inf, -np.inf, np.nan,
                  float(np.finfo(np.float32).max), 2.0 ** -126, 1.0 + 2.0 ** -40])
    hi, lo = split(x)
    assert hi[0] == 0 and not np.signbit(hi[0]) and np.signbit(hi[1])
    assert hi[2] == 0 and hi[3] == 0 and np.signbit(hi[3])
    assert np.isposinf(hi[4]) and np.isneginf(hi[5]) and np.isposinf(hi[6]) and np.isneginf(hi[7])
    assert np.isnan(hi[8])
    assert hi[9] == np.finfo(np.float32).max and lo[9] == 0
    assert hi[10] == np.float32(2.0 ** -126) and lo[10] == 0
    assert hi[11] == 1.0 and lo[11] == np.float32(2.0 ** -40)
    assert np.all(lo[:9] == 0)


def test_split_rejects_bad_arguments():
    lib = rwgt.load()
    assert lib.rw_split_double(None, 4, None, None, None) == -1  # RW_ERR_NULL
    assert lib.rw_split_double(None, -1, None, None, None) == -2  # RW_ERR_ARG
    assert lib.rw_split_double(None, 0, None, None, None) == 0

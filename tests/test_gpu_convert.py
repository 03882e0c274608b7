"""The integer-pipe binary64 <-> binary32 conversions that the FP32 kernels use
between the FP64 state and FP32 arithmetic, checked bit for bit against the
GPU's own conversions (round to nearest, ties to even).  The one documented
difference: magnitudes below the binary32 normal range (2^-126) become signed
zero instead of a subnormal."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def api(torch):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_1889_gb300 import api as a
    return a


def _doubles(n, seed=11):
    rng = np.random.default_rng(seed)
    sign = rng.choice([-1.0, 1.0], n)
    x = sign * (1.0 + rng.random(n)) * np.exp2(rng.integers(-140, 130, n).astype(np.float64))
    # exact binary32 ties (the 29 dropped bits = 1 followed by zeros), even and odd kept parts,
    # and their neighbours one binary64 ulp either side
    f = (rng.random(4096).astype(np.float32) + np.float32(1)) * np.exp2(rng.integers(-120, 120, 4096)).astype(np.float32)
    tie = (f.astype(np.float64).view(np.uint64) | np.uint64(1 << 28)).view(np.float64)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028235677973366e38, 3.4028235677973362e38,
                        3.5e38, -1e300, 1e-300, 1.1754943508222875e-38, 1.1754942e-38, 5e-324, 1.0, -2.5])
    return np.concatenate([x, tie, np.nextafter(tie, np.inf), np.nextafter(tie, -np.inf), special])


def test_binary64_to_binary32_matches_the_gpu(api, torch):
    x = torch.tensor(_doubles(1 << 20), device="cuda")
    y = torch.zeros(x.numel(), dtype=torch.float32, device="cuda")
    got, _ = api.diag_convert(x, y)
    ref = x.to(torch.float32)                              # the hardware conversion
    g = got.view(torch.int32).cpu().numpy(); r = ref.view(torch.int32).cpu().numpy()
    rf = ref.cpu().numpy()
    nan = np.isnan(rf)
    assert np.array_equal(np.isnan(got.cpu().numpy()), nan)
    sub = (rf != 0) & (np.abs(rf) < np.float32(2.0 ** -126))
    # below the normal range: signed zero
    assert np.array_equal(g[sub], (r[sub].astype(np.uint32) & np.uint32(0x80000000)).astype(np.int32))
    keep = ~nan & ~sub
    assert np.array_equal(g[keep], r[keep])
    assert keep.sum() > 1_000_000


def test_binary32_to_binary64_matches_the_gpu(api, torch):
    rng = np.random.default_rng(12)
    bits = rng.integers(0, 2 ** 32, 1 << 20, dtype=np.uint64).astype(np.uint32)
    y = torch.tensor(bits.view(np.float32), device="cuda")
    x = torch.zeros(y.numel(), dtype=torch.float64, device="cuda")
    _, got = api.diag_convert(x, y)
    ref = y.to(torch.float64)
    g = got.view(torch.int64).cpu().numpy(); r = ref.view(torch.int64).cpu().numpy()
    yf = y.cpu().numpy()
    nan = np.isnan(yf)
    assert np.array_equal(np.isnan(got.cpu().numpy()), nan)
    sub = (yf != 0) & (np.abs(yf) < np.float32(2.0 ** -126))
    assert np.all(got.cpu().numpy()[sub] == 0.0)
    keep = ~nan & ~sub
    assert np.array_equal(g[keep], r[keep])


def test_diag_convert_rejects_host_arrays(api, torch):
    x = torch.zeros(4, dtype=torch.float64); y = torch.zeros(4, dtype=torch.float32)
    rc = api.lib().msm_diag_convert(4, x.data_ptr(), y.data_ptr(), y.data_ptr(), x.data_ptr(), None)
    assert rc == -1                                        # MSM_EINVAL

"""Device building blocks checked against independent references."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2402_05193_gb300 as jxf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


def _ulps(x, ref):
    """Distance in units in the last place of ref."""
    return np.abs(x - ref) / np.spacing(np.abs(ref))


def test_double_division_within_one_ulp_of_ieee():
    rng = np.random.default_rng(0)
    n = 1 << 20
    a = rng.uniform(-1, 1, n) * 10.0 ** rng.uniform(-150, 150, n)
    b = rng.uniform(-1, 1, n) * 10.0 ** rng.uniform(-150, 150, n)
    b[np.abs(b) < 1e-300] = 1.0
    a[:4] = [1.0, 3.0, -7.0, 1e-300]
    b[:4] = [3.0, 3.0, 0.1, 7.0]
    ad, bd = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    qd = torch.empty_like(ad)
    L = jxf.lib()
    L.jxf_selftest_div.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_longlong]
    L.jxf_selftest_div.restype = ctypes.c_int
    assert L.jxf_selftest_div(ad.data_ptr(), bd.data_ptr(), qd.data_ptr(), n) == 0
    q = qd.cpu().numpy()
    ref = a / b
    ok = np.isfinite(ref) & (np.abs(ref) > 1e-300) & (np.abs(ref) < 1e300)
    u = _ulps(q[ok], ref[ok])
    print("max ulp %.3f, fraction exactly rounded %.4f" % (u.max(), np.mean(u == 0)))
    assert u.max() <= 1.0
    assert q[1] == 1.0  # exact quotients stay exact

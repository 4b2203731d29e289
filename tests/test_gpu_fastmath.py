"""The kernels' double-precision reciprocal, square root and reciprocal cube
root (hardware seed + one cubic correction) against CUDA's own functions, and
the integer-only float -> double widening against the hardware conversion."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2403_08777_gb300 import _abi, build

pytestmark = pytest.mark.gpu

ULP = 2.0 ** -52


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return _abi.load()


def run(lib, which, x):
    xd = torch.from_numpy(x).cuda()
    ours, ref = torch.empty_like(xd), torch.empty_like(xd)
    assert lib.nsrhs_probe_special(which, xd.numel(), ctypes.c_void_p(xd.data_ptr()),
                                   ctypes.c_void_p(ours.data_ptr()),
                                   ctypes.c_void_p(ref.data_ptr()), None) == 0
    torch.cuda.synchronize()
    return ours.cpu().numpy(), ref.cpu().numpy()


def samples(lo, hi, n=1 << 20, seed=0):
    rng = np.random.default_rng(seed)
    x = np.exp(rng.uniform(np.log(lo), np.log(hi), n))
    # exact powers of two, values next to them, and the geometry range of the meshes
    p2 = 2.0 ** np.arange(int(np.log2(lo)) + 1, int(np.log2(hi)))
    return np.concatenate([x, p2, np.nextafter(p2, 0), np.nextafter(p2, np.inf),
                           rng.uniform(1e-9, 1e-6, 1000)])


@pytest.mark.parametrize("which,lo,hi", [(0, 1e-250, 1e250), (1, 1e-300, 1e300),
                                         (2, 1e-300, 1e300)])
def test_special_functions_within_two_ulp(lib, which, lo, hi):
    x = samples(lo, hi)
    ours, ref = run(lib, which, x)
    rel = np.abs(ours - ref) / np.abs(ref)
    assert np.all(np.isfinite(ours))
    assert rel.max() <= 2 * ULP, (which, rel.max() / ULP)


def test_sqrt_of_zero_and_subnormals(lib):
    x = np.array([0.0, 5e-324, 1e-310, 2.2250738585072014e-308, 1.0])
    ours, ref = run(lib, 1, x)
    assert ours[0] == 0.0 and ours[1] == 0.0 and ours[2] == 0.0
    assert abs(ours[3] - ref[3]) <= 2 * ULP * ref[3] and ours[4] == 1.0


def test_widening_is_exact(lib):
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=100000) * 10.0 ** rng.integers(-30, 30, 100000),
                        [0.0, -0.0, 1.0, -2.5, 3.4e38, 1.2e-38]])
    ours, ref = run(lib, 3, x)
    assert np.array_equal(ours.view(np.int64), ref.view(np.int64))

"""nsrhs_mesh_check_noalloc: the mesh check for callers that cannot allocate
device memory (a fixed arena owned by the caller, or a host framework that
forbids cudaMalloc). It must report exactly what nsrhs_mesh_create finds on
the same arrays, call after call, using only its static scratch array.

Collected last (file name) so that a run stopping at its first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import meshgen as mg
from paper_2403_08777_gb300 import _abi, build

pytestmark = pytest.mark.gpu

REL = 1e-12  # the FP64 tolerance of the parity tests


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return _abi.load()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def check_noalloc(lib, coords, conn, thr=10.0):
    """Two calls in a row through the C ABI; returns both results."""
    out = []
    stream = torch.cuda.current_stream()
    for _ in range(2):
        res = torch.full((5,), -7.0, dtype=torch.float64, device=coords.device)  # poison
        st = lib.nsrhs_mesh_check_noalloc(coords.shape[1], conn.shape[1], _ptr(coords), _ptr(conn),
                                          thr, ctypes.c_void_p(stream.cuda_stream), _ptr(res))
        assert st == _abi.OK
        torch.cuda.synchronize()
        raw = res.cpu().numpy()
        ints = raw[:3].view(np.int64)
        out.append({"bad_index": int(ints[0]), "bad_det": int(ints[1]), "n_high_ar": int(ints[2]),
                    "min_detj": float(raw[3]), "max_ar": float(raw[4])})
    return out


def create_status(lib, coords, conn, thr=10.0):
    """The existing entry point on the same arrays: status and mesh info."""
    h = ctypes.c_void_p()
    opts = _abi.MeshOpts(thr)
    st = lib.nsrhs_mesh_create(coords.shape[1], conn.shape[1], _ptr(coords), _ptr(conn),
                               ctypes.byref(opts), None, ctypes.byref(h))
    info = None
    if st == _abi.OK:
        inf = _abi.MeshInfo()
        assert lib.nsrhs_mesh_get_info(h, ctypes.byref(inf)) == _abi.OK
        info = inf
        lib.nsrhs_destroy(h)
    return st, info


def to_dev(*arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def test_valid_mesh_matches_mesh_create(lib):
    for n, jitter in ((40, 0.3), (5, 0.1)):   # large then small: no state carried over
        c, conn, _, _ = mg.box_mesh(n, jitter)
        coords, conn_d = to_dev(c, conn)
        st, info = create_status(lib, coords, conn_d)
        assert st == _abi.OK
        for r in check_noalloc(lib, coords, conn_d):
            assert r["bad_index"] == 0 and r["bad_det"] == 0
            assert r["n_high_ar"] == info.n_high_ar
            assert abs(r["min_detj"] - info.min_detj) <= REL * info.min_detj
            assert abs(r["max_ar"] - info.max_ar) <= REL * info.max_ar
        if jitter == 0.3:
            assert info.n_high_ar > 0


def test_invalid_meshes_match_mesh_create(lib):
    c, conn, _, _ = mg.box_mesh(6, 0.1)
    N = c.shape[1]
    bad = conn.copy()
    bad[1, [3, 50, 700]] = N          # three out-of-range indices
    bad[2, 9] = -4                    # and a negative one
    inv = conn.copy()
    inv[[1, 2], 11] = inv[[2, 1], 11]  # two inverted elements
    inv[[1, 2], 200] = inv[[2, 1], 200]
    for arr, n_idx, n_det in ((bad, 4, 0), (inv, 0, 2)):
        coords, conn_d = to_dev(c, arr)
        st, _ = create_status(lib, coords, conn_d)
        assert st == _abi.EMESH
        for r in check_noalloc(lib, coords, conn_d):
            assert r["bad_index"] == n_idx and r["bad_det"] == n_det


def test_rejects_bad_sizes(lib):
    c, conn, _, _ = mg.box_mesh(2, 0.0)
    coords, conn_d = to_dev(c, conn)
    res = torch.zeros(5, dtype=torch.float64, device="cuda")
    for nn, ne, thr in ((0, 48, 10.0), (27, 0, 10.0), (2**31, 48, 10.0), (27, 2**31, 10.0),
                        (27, 48, 0.0)):
        assert lib.nsrhs_mesh_check_noalloc(nn, ne, _ptr(coords), _ptr(conn_d), thr, None,
                                            _ptr(res)) == _abi.EINVAL
    assert lib.nsrhs_mesh_check_noalloc(27, 48, _ptr(coords), _ptr(conn_d), 10.0, None,
                                        None) == _abi.EINVAL

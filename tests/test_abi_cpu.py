"""The C-ABI library builds, loads and exports every declared symbol; host-side
argument checking (no GPU needed: these calls return before touching CUDA)."""
import ctypes
import os
import re

import pytest

from paper_2403_08777_gb300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.load()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(nsrhs_\w+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert set(_abi.EXPORTED) <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_defaults(lib):
    for s in range(6):
        assert lib.nsrhs_status_string(s)
    assert b"unknown" in lib.nsrhs_status_string(99)
    p = _abi.Params()
    lib.nsrhs_params_default(ctypes.byref(p))
    assert (p.rho, p.mu, p.c_vreman, p.c1, p.c2, p.precision, p.scatter, p.convection,
            p.tau_mode, p.geometry, p.reserved) == (1.0, 1e-2, 0.0, 4.0, 2.0, 0, 0, 0, 0, 0, 0)
    o = _abi.MeshOpts()
    lib.nsrhs_mesh_opts_default(ctypes.byref(o))
    assert (o.ar_threshold, o.colour, o.reserved) == (10.0, 0, 0)
    assert ctypes.sizeof(_abi.Params) == 64 and ctypes.sizeof(_abi.MeshInfo) == 80
    assert ctypes.sizeof(_abi.MeshOpts) == 16


def test_argument_errors_without_gpu(lib):
    P = ctypes.c_void_p
    out = P(1234)
    fake = P(0x1000)
    # NULL output handle / NULL arrays / bad sizes -> EINVAL, *out cleared
    assert lib.nsrhs_mesh_create(10, 10, fake, fake, None, None, None) == _abi.EINVAL
    assert lib.nsrhs_mesh_create(10, 10, None, fake, None, None, ctypes.byref(out)) == _abi.EINVAL
    assert out.value is None
    assert lib.nsrhs_mesh_create(0, 10, fake, fake, None, None, ctypes.byref(out)) == _abi.EINVAL
    assert lib.nsrhs_mesh_create(10, -1, fake, fake, None, None, ctypes.byref(out)) == _abi.EINVAL
    assert lib.nsrhs_mesh_create(2**31, 1, fake, fake, None, None,
                                 ctypes.byref(out)) == _abi.EINVAL
    for bad in (_abi.MeshOpts(-1.0, 0, 0), _abi.MeshOpts(10.0, 2, 0), _abi.MeshOpts(10.0, 1, 7)):
        assert lib.nsrhs_mesh_create(10, 10, fake, fake, ctypes.byref(bad), None,
                                     ctypes.byref(out)) == _abi.EINVAL
    # unknown / destroyed mesh handles are rejected, destroy is NULL-safe
    p = _abi.Params()
    lib.nsrhs_params_default(ctypes.byref(p))
    assert lib.nsrhs_assemble(fake, ctypes.byref(p), fake, fake, None) == _abi.EINVAL
    assert lib.nsrhs_assemble(None, ctypes.byref(p), fake, fake, None) == _abi.EINVAL
    assert lib.nsrhs_assemble_vjp(fake, ctypes.byref(p), fake, fake, fake, None) == _abi.EINVAL
    info = _abi.MeshInfo()
    assert lib.nsrhs_mesh_get_info(fake, ctypes.byref(info)) == _abi.EINVAL
    assert lib.nsrhs_mesh_element_colours(fake, 0, fake, None) == _abi.EINVAL
    assert lib.nsrhs_assemble_rhs_vjp(fake, ctypes.byref(p), fake, fake, fake, fake,
                                      None) == _abi.EINVAL
    assert lib.nsrhs_assemble_elmat(fake, ctypes.byref(p), fake, fake, None) == _abi.EINVAL
    assert lib.nsrhs_lumped_mass(fake, fake, None) == _abi.EINVAL
    assert lib.nsrhs_explicit_step(fake, ctypes.byref(p), 1e-3, 0, fake, fake, None) == _abi.EINVAL
    # the no-alloc check validates its arguments before touching the device
    res = P(0x2000)
    assert lib.nsrhs_mesh_check_noalloc(0, 10, fake, fake, 10.0, None, res) == _abi.EINVAL
    assert lib.nsrhs_mesh_check_noalloc(10, 10, fake, fake, -1.0, None, res) == _abi.EINVAL
    assert lib.nsrhs_mesh_check_noalloc(10, 10, None, fake, 10.0, None, res) == _abi.EINVAL
    lib.nsrhs_destroy(None)
    lib.nsrhs_destroy(fake)


def test_python_layer_fails_loudly_without_library(tmp_path):
    with pytest.raises(_abi.NativeLibraryMissing):
        saved = _abi._lib
        try:
            _abi._lib = None
            _abi.load(str(tmp_path / "missing.so"))
        finally:
            _abi._lib = saved

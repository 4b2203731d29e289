"""CPU oracle for the tetrahedral Navier-Stokes RHS assembly.

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline use this package. The library (the CUDA path) never imports it, and
it imports nothing from the library.

The arithmetic is in ``nsrhs_oracle.cpp`` (plain serial double precision,
complex instantiation for complex-step derivatives); this file only builds
that file with g++ and marshals numpy arrays to it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nsrhs_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libnsrhs_oracle.so")
_lib = None

# Term selection bits of or_element_f64 / or_assemble_f64.
T_CONV, T_VISC, T_PRES, T_SUPG, T_CONT, T_PSPG = 1, 2, 4, 8, 16, 32
T_ALL = 63

# Constants of the tau definition used by the library (c1 = 4, c2 = 2).
C1, C2 = 4.0, 2.0


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I64, U = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint
        lib.or_element_f64.argtypes = [P, P, P, U, P]
        lib.or_element_c128.argtypes = [P, P, P, P, U, P, P]
        lib.or_assemble_f64.argtypes = [I64, I64, P, P, P, P, U, I64, I64, P]
        lib.or_assemble_c128.argtypes = [I64, I64, P, P, P, P, P, U, P, P]
        lib.or_vjp_f64.argtypes = [I64, I64, P, P, P, P, P, P]
        lib.or_detj.argtypes = [I64, I64, P, P, P]
        for f in ("or_element_f64", "or_element_c128", "or_assemble_f64", "or_assemble_c128",
                  "or_vjp_f64", "or_detj"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def _params(rho, mu, c_vreman=0.0, c1=C1, c2=C2, skew=False, tau_elem=False):
    return np.array([rho, mu, c_vreman, c1, c2, float(skew), float(tau_elem)], np.float64)


def _check(r, what):
    if r != 0:
        raise ValueError(f"{what}: oracle status {r} ({'bad arguments' if r == 1 else 'bad mesh'})")


def element(X, U, rho, mu, c_vreman=0.0, terms=T_ALL, c1=C1, c2=C2, skew=False, tau_elem=False):
    """Element RHS F [4][4] (local node, (mom x, y, z, continuity)) of one tet.
    X [4][3] node coordinates, U [4][4] nodal (u, v, w, p)."""
    X = np.ascontiguousarray(X, np.float64)
    U = np.ascontiguousarray(U, np.float64)
    F = np.empty((4, 4), np.float64)
    pr = _params(rho, mu, c_vreman, c1, c2, skew, tau_elem)
    _check(_load().or_element_f64(_p(X), _p(U), _p(pr), terms, _p(F)), "element")
    return F


def element_complex(X, U, rho, mu, c_vreman=0.0, terms=T_ALL, c1=C1, c2=C2, skew=False,
                    tau_elem=False):
    X = np.ascontiguousarray(X, np.float64)
    U = np.asarray(U, np.complex128)
    ur, ui = np.ascontiguousarray(U.real), np.ascontiguousarray(U.imag)
    Fr, Fi = np.empty((4, 4)), np.empty((4, 4))
    pr = _params(rho, mu, c_vreman, c1, c2, skew, tau_elem)
    _check(_load().or_element_c128(_p(X), _p(ur), _p(ui), _p(pr), terms, _p(Fr), _p(Fi)),
           "element_complex")
    return Fr + 1j * Fi


def assemble(coords, conn, up, rho, mu, c_vreman=0.0, terms=T_ALL, e0=0, e1=None,
             c1=C1, c2=C2, skew=False, tau_elem=False):
    """Global RHS [4][N] (float64) over elements [e0, e1)."""
    coords = np.ascontiguousarray(coords, np.float64)
    conn = np.ascontiguousarray(conn, np.int32)
    up = np.ascontiguousarray(up, np.float64)
    N, E = coords.shape[1], conn.shape[1]
    e1 = E if e1 is None else e1
    rhs = np.empty((4, N), np.float64)
    pr = _params(rho, mu, c_vreman, c1, c2, skew, tau_elem)
    _check(_load().or_assemble_f64(N, E, _p(coords), _p(conn), _p(up), _p(pr), terms, e0, e1,
                                   _p(rhs)), "assemble")
    return rhs


def assemble_complex(coords, conn, up, rho, mu, c_vreman=0.0, terms=T_ALL, c1=C1, c2=C2,
                     skew=False, tau_elem=False):
    coords = np.ascontiguousarray(coords, np.float64)
    conn = np.ascontiguousarray(conn, np.int32)
    up = np.asarray(up, np.complex128)
    ur, ui = np.ascontiguousarray(up.real), np.ascontiguousarray(up.imag)
    N, E = coords.shape[1], conn.shape[1]
    rr, ri = np.empty((4, N)), np.empty((4, N))
    pr = _params(rho, mu, c_vreman, c1, c2, skew, tau_elem)
    _check(_load().or_assemble_c128(N, E, _p(coords), _p(conn), _p(ur), _p(ui), _p(pr), terms,
                                    _p(rr), _p(ri)), "assemble_complex")
    return rr + 1j * ri


def vjp(coords, conn, up, w, rho, mu, c_vreman=0.0, c1=C1, c2=C2, skew=False, tau_elem=False):
    """(dRHS/dup)^T w as [4][N], element Jacobians by complex step."""
    coords = np.ascontiguousarray(coords, np.float64)
    conn = np.ascontiguousarray(conn, np.int32)
    up = np.ascontiguousarray(up, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    N, E = coords.shape[1], conn.shape[1]
    g = np.empty((4, N), np.float64)
    pr = _params(rho, mu, c_vreman, c1, c2, skew, tau_elem)
    _check(_load().or_vjp_f64(N, E, _p(coords), _p(conn), _p(up), _p(w), _p(pr), _p(g)), "vjp")
    return g


def detj(coords, conn):
    coords = np.ascontiguousarray(coords, np.float64)
    conn = np.ascontiguousarray(conn, np.int32)
    d = np.empty(conn.shape[1], np.float64)
    _check(_load().or_detj(coords.shape[1], conn.shape[1], _p(coords), _p(conn), _p(d)), "detj")
    return d


def submesh_for_nodes(conn, nodes):
    """Elements incident to any of `nodes`: the oracle's RHS at those nodes
    over this sub-mesh equals its RHS over the full mesh (sampled parity at
    sizes where the full oracle would be slow). Returns conn_sub [4][E_sub]."""
    conn = np.asarray(conn)
    mark = np.zeros(int(conn.max()) + 1, bool)
    mark[np.asarray(nodes)] = True
    mask = mark[conn].any(axis=0)
    return np.ascontiguousarray(conn[:, mask])


# ---- explicit time stepping of the momentum equation (numpy composition) ----

def lumped_mass(coords, conn):
    """Row-sum lumped P1 mass: m_a = sum over elements containing a of V_e/4."""
    conn = np.asarray(conn)
    v4 = detj(coords, conn) / 24.0
    m = np.zeros(np.asarray(coords).shape[1])
    for a in range(4):
        np.add.at(m, conn[a], v4)
    return m


def euler(u, L, dt):
    """u' = u + dt L(u)."""
    return u + dt * L(u)


def ssprk3(u, L, dt):
    """Shu-Osher three-stage strong-stability-preserving Runge-Kutta."""
    u1 = u + dt * L(u)
    u2 = 0.75 * u + 0.25 * (u1 + dt * L(u1))
    return u / 3.0 + 2.0 / 3.0 * (u2 + dt * L(u2))


def explicit_step(coords, conn, up, rho, mu, dt, scheme="ssprk3", **kw):
    """One step of rho m du/dt = F(u, p) (momentum rows, pressure fixed)."""
    m = lumped_mass(coords, conn)
    p = np.asarray(up)[3].copy()

    def L(u):
        full = np.vstack([u, p[None, :]])
        return assemble(coords, conn, full, rho, mu, **kw)[:3] / (rho * m[None, :])

    stepper = {"euler": euler, "ssprk3": ssprk3}[scheme]
    return np.vstack([stepper(np.asarray(up)[:3].copy(), L, dt), p[None, :]])

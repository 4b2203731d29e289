"""Seeded synthetic inputs: jittered Kuhn tet meshes, nodal fields, renumberings.

This module generates inputs only and holds none of the assembly arithmetic.
The CPU oracle and the CUDA path both consume its arrays; it imports neither.

The paper measures on a 5.6M-node / 32M-tet LES mesh of the Bolund cliff
(Sec. III-A), which is not available. These meshes of linear tetrahedra
(Sec. II restricts the study to tets) stand in for it: a unit cube of n^3
hexes, each split into 6 Kuhn tets sharing the hex diagonal, with interior
nodes jittered, and node numbering lexicographic, random or reverse
Cuthill-McKee (RCM) to expose gather/scatter locality.

Layouts (structure of arrays): coords [3][N] float64, conn [4][E] int32
(element index fastest), nodal fields up [4][N] float64 = (u, v, w, p).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "meshgen.cpp")
_LIB = os.path.join(_HERE, "_build", "libmeshgen.so")
_lib = None

# Seeds of the independent random streams (one per kind of input).
SEED_MESH, SEED_FIELDS, SEED_PERM, SEED_COT, SEED_DIRS = 1, 2, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile the host-side generator (g++, portable C++17, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.mg_box_mesh.restype = ctypes.c_int64
        lib.mg_box_mesh.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                                    ctypes.c_double, P, P, P]
        lib.mg_fields.restype = None
        lib.mg_fields.argtypes = [ctypes.c_int64, P, ctypes.c_uint64, ctypes.c_double,
                                  ctypes.c_double, P]
        lib.mg_normal.restype = None
        lib.mg_normal.argtypes = [ctypes.c_int64, ctypes.c_uint64, P]
        lib.mg_random_order.restype = None
        lib.mg_random_order.argtypes = [ctypes.c_int64, ctypes.c_uint64, P]
        lib.mg_rcm_order.restype = ctypes.c_int
        lib.mg_rcm_order.argtypes = [ctypes.c_int64, ctypes.c_int64, P, P]
        lib.mg_bandwidth.restype = ctypes.c_int64
        lib.mg_bandwidth.argtypes = [ctypes.c_int64, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def box_mesh(n: int, jitter: float = 0.1, seed: int = SEED_MESH, min_det_frac: float = 0.05):
    """Kuhn mesh of the unit cube: returns (coords [3][N] f64, conn [4][E] i32,
    hex_colour [n^3] i8, n_reduced).

    Hex (i,j,k) -> elements 6*hex..6*hex+5 (so the 6 tets of a hex are
    consecutive), node (i,j,k) -> i + (n+1)(j + (n+1)k). Tets with
    detJ < min_det_frac*h^3 after jitter get their nodes' jitter halved until
    none remain; n_reduced counts the nodes so treated.
    """
    n1 = n + 1
    N, E = n1 ** 3, 6 * n ** 3
    coords = np.empty((3, N), np.float64)
    conn = np.empty((4, E), np.int32)
    colour = np.empty(n ** 3, np.int8)
    r = _load().mg_box_mesh(n, float(jitter), seed, float(min_det_frac), _p(coords), _p(conn),
                            _p(colour))
    if r < 0:
        raise RuntimeError(f"mg_box_mesh failed ({r})")
    return coords, conn, colour, int(r)


def fields(coords: np.ndarray, seed: int = SEED_FIELDS, noise_sigma: float = 1e-2,
           mag_max: float = 0.0) -> np.ndarray:
    """Nodal (u,v,w,p) [4][N]: Taylor-Green velocity at 2*pi periodicity
    + N(0, noise_sigma^2) noise (+ m*d, m~U(0,mag_max), d uniform on the
    sphere, if mag_max > 0); pressure ~ U(-1, 1)."""
    coords = np.ascontiguousarray(coords, np.float64)
    N = coords.shape[1]
    up = np.empty((4, N), np.float64)
    _load().mg_fields(N, _p(coords), seed, float(noise_sigma), float(mag_max), _p(up))
    return up


def normal(shape, seed: int) -> np.ndarray:
    """Counter-based N(0,1) samples."""
    n = int(np.prod(shape))
    out = np.empty(n, np.float64)
    _load().mg_normal(n, seed, _p(out))
    return out.reshape(shape)


def random_order(N: int, seed: int = SEED_PERM) -> np.ndarray:
    order = np.empty(N, np.int64)
    _load().mg_random_order(N, seed, _p(order))
    return order


def rcm_order(conn: np.ndarray, N: int) -> np.ndarray:
    conn = np.ascontiguousarray(conn, np.int32)
    order = np.empty(N, np.int64)
    r = _load().mg_rcm_order(N, conn.shape[1], _p(conn), _p(order))
    if r != 0:
        raise RuntimeError("mg_rcm_order failed")
    return order


def bandwidth(conn: np.ndarray) -> int:
    conn = np.ascontiguousarray(conn, np.int32)
    return int(_load().mg_bandwidth(conn.shape[1], _p(conn)))


def renumber(order: np.ndarray, coords: np.ndarray, conn: np.ndarray, *nodal):
    """Apply a node order (order[new] = old) to coords, conn and [k][N] arrays."""
    N = coords.shape[1]
    rank = np.empty(N, np.int64)
    rank[order] = np.arange(N, dtype=np.int64)
    new_coords = np.ascontiguousarray(coords[:, order])
    new_conn = rank[conn].astype(np.int32)
    return (new_coords, new_conn) + tuple(np.ascontiguousarray(a[:, order]) for a in nodal)


def delaunay_mesh(n: int, jitter: float = 0.3, seed: int = SEED_MESH):
    """Unstructured tet mesh of the unit cube: Delaunay tetrahedralisation
    (scipy / Qhull) of the (n+1)^3 lattice with interior points jittered by
    U(-jitter h, jitter h). Node valences vary and there is no hex-block
    structure. Zero-volume tets that Qhull leaves on the flat cube faces
    (|detJ| < 1e-8 h^3) are dropped (they carry no volume); the others are
    oriented so that detJ > 0. Returns (coords [3][N] f64, conn [4][E] i32)."""
    from scipy.spatial import Delaunay

    n1 = n + 1
    idx = np.arange(n1 ** 3)
    ijk = np.stack([idx % n1, (idx // n1) % n1, idx // (n1 * n1)], axis=1)
    pts = ijk.astype(np.float64) / n
    interior = np.all((ijk > 0) & (ijk < n), axis=1)
    # seeded PCG64 stream (reproducible across machines)
    off = np.random.default_rng(seed).uniform(-1.0, 1.0, (n1 ** 3, 3)) * jitter / n
    pts[interior] += off[interior]
    simp = Delaunay(pts).simplices.astype(np.int64)
    X = pts[simp]
    det = np.linalg.det(X[:, 1:] - X[:, :1])
    keep = np.abs(det) > 1e-8 / n ** 3
    simp, det = simp[keep], det[keep]
    neg = det < 0
    simp[neg, 1], simp[neg, 2] = simp[neg, 2].copy(), simp[neg, 1].copy()
    coords = np.ascontiguousarray(pts.T)
    conn = np.ascontiguousarray(simp.T.astype(np.int32))
    return coords, conn


def write_msh(path: str, coords: np.ndarray, conn: np.ndarray) -> None:
    """Gmsh MSH 2.2 ASCII with 4-node tetrahedra (element type 4)."""
    N, E = coords.shape[1], conn.shape[1]
    with open(path, "w") as f:
        f.write("$MeshFormat\n2.2 0 8\n$EndMeshFormat\n$Nodes\n%d\n" % N)
        for i in range(N):
            f.write("%d %.17g %.17g %.17g\n" % (i + 1, coords[0, i], coords[1, i], coords[2, i]))
        f.write("$EndNodes\n$Elements\n%d\n" % E)
        for e in range(E):
            a = conn[:, e] + 1
            f.write("%d 4 2 0 1 %d %d %d %d\n" % (e + 1, a[0], a[1], a[2], a[3]))
        f.write("$EndElements\n")


def read_msh(path: str):
    """Read the nodes and the 4-node tetrahedra (type 4) of a Gmsh MSH 2.2
    ASCII file; other element types are skipped. Node tags are mapped to
    0-based indices in file order. Returns (coords [3][N] f64, conn [4][E] i32)."""
    with open(path) as f:
        lines = [ln.strip() for ln in f]
    i = lines.index("$MeshFormat")
    version = lines[i + 1].split()
    if not version[0].startswith("2") or version[1] != "0":
        raise ValueError("only MSH 2.x ASCII is supported")
    i = lines.index("$Nodes")
    n_nodes = int(lines[i + 1])
    tags = np.empty(n_nodes, np.int64)
    xyz = np.empty((n_nodes, 3))
    for k in range(n_nodes):
        parts = lines[i + 2 + k].split()
        tags[k] = int(parts[0])
        xyz[k] = [float(v) for v in parts[1:4]]
    pos = {int(t): k for k, t in enumerate(tags)}
    i = lines.index("$Elements")
    n_el = int(lines[i + 1])
    tets = []
    for k in range(n_el):
        parts = lines[i + 2 + k].split()
        if int(parts[1]) != 4:
            continue
        n_tags = int(parts[2])
        tets.append([pos[int(v)] for v in parts[3 + n_tags:7 + n_tags]])
    coords = np.ascontiguousarray(xyz.T)
    conn = np.ascontiguousarray(np.asarray(tets, np.int32).reshape(-1, 4).T)
    return coords, conn


def make_unstructured(n: int, *, jitter: float = 0.3, order: str = "rcm", rho: float = 1.0,
                      mu: float = 1e-2, mag_max: float = 0.0, c_vreman: float = 0.0,
                      noise_sigma: float = 1e-2) -> "Workload":
    """Workload on the Delaunay mesh of an (n+1)^3 jittered lattice."""
    coords, conn = delaunay_mesh(n, jitter)
    up = fields(coords, noise_sigma=noise_sigma, mag_max=mag_max)
    if order == "random":
        coords, conn, up = renumber(random_order(coords.shape[1]), coords, conn, up)
    elif order == "rcm":
        coords, conn, up = renumber(rcm_order(conn, coords.shape[1]), coords, conn, up)
    return Workload(f"delaunay{n}^3-{order}", n, coords, conn, up, rho, mu, c_vreman, order,
                    jitter)


@dataclass
class Workload:
    """One synthetic assembly problem (host arrays)."""
    name: str
    n: int
    coords: np.ndarray          # [3][N] f64
    conn: np.ndarray            # [4][E] i32
    up: np.ndarray              # [4][N] f64
    rho: float
    mu: float
    c_vreman: float = 0.0
    order: str = "lex"
    jitter: float = 0.1
    n_reduced: int = 0
    hex_colour: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return self.coords.shape[1]

    @property
    def n_elems(self) -> int:
        return self.conn.shape[1]


def make_workload(n: int, *, jitter: float = 0.1, order: str = "lex", rho: float = 1.0,
                  mu: float = 1e-2, mag_max: float = 0.0, c_vreman: float = 0.0,
                  noise_sigma: float = 1e-2, name: str | None = None) -> Workload:
    """Build a workload: Kuhn mesh (seed 1), fields (seed 2), node order
    'lex' | 'random' (seed 3) | 'rcm'."""
    coords, conn, colour, n_red = box_mesh(n, jitter)
    up = fields(coords, noise_sigma=noise_sigma, mag_max=mag_max)
    if order == "random":
        coords, conn, up = renumber(random_order(coords.shape[1]), coords, conn, up)
    elif order == "rcm":
        coords, conn, up = renumber(rcm_order(conn, coords.shape[1]), coords, conn, up)
    elif order != "lex":
        raise ValueError(order)
    return Workload(name or f"kuhn{n}^3-{order}", n, coords, conn, up, rho, mu, c_vreman, order,
                    jitter, n_red, colour)


# The five synthetic problems (sizes and settings of the study; mesh sizes in hexes).
def tiny(**kw) -> Workload:
    """8^3 hexes (3072 tets, 729 nodes), jitter 0.1, lexicographic, rho=1, mu=1e-2."""
    return make_workload(8, name="kuhn8^3-lex", **kw)


def medium(order: str = "rcm", n: int = 128) -> Workload:
    """128^3 hexes (12.58M tets, 2.15M nodes), random or RCM order, mu=1e-2."""
    return make_workload(n, order=order, name=f"kuhn{n}^3-{order}")


def paper_scale(n: int = 256, order: str = "rcm") -> Workload:
    """256^3 hexes (100.7M tets, 16.97M nodes), RCM, rho=1, mu=1e-4,
    velocity = Taylor-Green + m*d with m ~ U(0, 10)."""
    return make_workload(n, order=order, mu=1e-4, mag_max=10.0, name=f"kuhn{n}^3-{order}-re")


def precision_case(n: int = 256, order: str = "rcm") -> Workload:
    """Like paper_scale but with jitter 0.3 h (creates high-aspect-ratio tets)."""
    return make_workload(n, jitter=0.3, order=order, mu=1e-4, mag_max=10.0,
                         name=f"kuhn{n}^3-{order}-j0.3")

"""GPU: the element- and block-colouring scatters (deterministic assembly).

The colourings must be valid (no two elements that share a node have the
same colour; no two blocks that share a node have the same colour; checked on
the host from what the library reports), the coloured forward and adjoint must
match the oracle within the same
tolerances as the atomic path, and repeated calls must give bitwise equal
results (the summation order is fixed by the colour order).
"""
import numpy as np
import pytest
import torch

import meshgen as mg
import oracle
import paper_2403_08777_gb300 as ns
from paper_2403_08777_gb300 import _abi

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12
TOL_MIXED = 1e-5
TOL_VJP_ORACLE = 1e-12
TOL_VJP_FD = 1e-6


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ns.load_library()
    return torch.device("cuda:0")


def relerr(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def on_dev(dev, *arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in arrays]


def check_fp64(x, ref):
    assert relerr(x, ref) <= TOL_FP64, relerr(x, ref)
    assert np.abs(x - ref).max() <= TOL_FP64 * np.abs(ref).max()


def check_colouring(colours, conn, n_nodes, n_colours):
    """Host check: colours in range, every colour used, and each (node,
    colour) pair met at most once (elements sharing a node differ)."""
    E = conn.shape[1]
    assert colours.shape == (E,)
    assert colours.min() >= 0 and colours.max() == n_colours - 1
    assert np.unique(colours).size == n_colours
    pairs = conn.astype(np.int64) * 128 + colours[None, :].astype(np.int64)
    assert np.unique(pairs.ravel()).size == 4 * E
    # a node touched by k elements needs k colours
    assert n_colours >= np.bincount(conn.ravel(), minlength=n_nodes).max()
    assert n_colours <= 128


def check_block_colouring(bcol, block, conn, n_colours, n_blocks):
    """Host check of the block colouring: every block has one colour, and at
    every node the elements of two different blocks never share a colour."""
    E = conn.shape[1]
    assert block.min() == 0 and block.max() == n_blocks - 1
    assert np.bincount(block).max() <= 256
    assert bcol.min() >= 0 and bcol.max() == n_colours - 1
    # one colour per block
    pb = np.unique(np.stack([block, bcol]), axis=1)
    assert pb.shape[1] == n_blocks
    # (node, colour) -> a single block
    rows = np.unique(np.stack([conn.ravel(), np.tile(bcol, 4), np.tile(block, 4)]), axis=1)
    nc = np.unique(rows[:2], axis=1)
    assert nc.shape[1] == rows.shape[1]
    assert E > 0


MESHES = [("kuhn", 8, "lex"), ("kuhn", 13, "random"), ("kuhn", 20, "rcm"),
          ("delaunay", 10, "rcm"), ("delaunay", 14, "random")]


def workload(kind, n, order, **kw):
    if kind == "kuhn":
        return mg.make_workload(n, jitter=0.2, order=order, **kw)
    return mg.make_unstructured(n, order=order, **kw)


@pytest.mark.parametrize("kind,n,order", MESHES)
def test_colouring_is_valid(dev, kind, n, order):
    w = workload(kind, n, order)
    coords, conn = on_dev(dev, w.coords, w.conn)
    m = ns.Mesh(coords, conn, colour=True)
    info = m.info()
    colours = m.element_colours().cpu().numpy()
    check_colouring(colours, w.conn, w.n_nodes, info["n_colours"])
    check_block_colouring(m.element_colours("block_colour").cpu().numpy(),
                          m.element_colours("block").cpu().numpy(), w.conn,
                          info["n_block_colours"], info["n_blocks"])
    # deterministic: the same mesh gets the same colours
    m2 = ns.Mesh(coords, conn, colour=True)
    assert np.array_equal(m2.element_colours().cpu().numpy(), colours)
    plain = ns.Mesh(coords, conn)
    assert plain.info()["n_colours"] == 0 and plain.info()["n_block_colours"] == 0
    # colour-major copy (connectivity, double geometry, 64-byte element
    # records stored in whole blocks of 256), element colours and order;
    # block colours and the per-colour block lists
    assert (info["device_bytes"] - plain.info()["device_bytes"] ==
            (16 + 88 + 1 + 4) * w.n_elems + (64 * 256 + 5) * info["n_blocks"])
    for mm in (m, m2, plain):
        mm.close()


@pytest.mark.parametrize("kind,n,order", MESHES)
def test_colour_scatter_matches_oracle(dev, kind, n, order):
    w = workload(kind, n, order, mu=1e-3, mag_max=3.0)
    coords, conn, up = on_dev(dev, w.coords, w.conn, w.up)
    m = ns.Mesh(coords, conn, colour=True)
    ref = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu)
    for sc in ("colour", "block_colour"):
        check_fp64(m.assemble(up, ns.Params(rho=w.rho, mu=w.mu, scatter=sc)).cpu().numpy(), ref)
        x = m.assemble(up.float(), ns.Params(rho=w.rho, mu=w.mu, scatter=sc,
                                             precision="mixed")).cpu().numpy()
        assert relerr(x, ref) <= TOL_MIXED
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    gref = oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu)
    cot_d = torch.from_numpy(cot).to(dev)
    for sc in ("colour", "block", "block_colour"):
        g = m.assemble_vjp(up, cot_d, ns.Params(rho=w.rho, mu=w.mu, scatter=sc)).cpu().numpy()
        assert relerr(g, gref) <= TOL_VJP_ORACLE, (sc, relerr(g, gref))
        gm = m.assemble_vjp(up.float(), cot_d.float(),
                            ns.Params(rho=w.rho, mu=w.mu, scatter=sc, precision="mixed"))
        assert relerr(gm.cpu().numpy(), gref) <= TOL_VJP_FD, sc
    m.close()


@pytest.mark.parametrize("cv,conv,tau", [(0.07, "convective", "gauss"), (0.0, "skew", "element"),
                                         (0.07, "skew", "gauss")])
def test_colour_scatter_variants(dev, cv, conv, tau):
    w = mg.make_workload(12, jitter=0.2, order="random", mu=1e-3, mag_max=3.0, c_vreman=cv)
    okw = dict(c_vreman=cv, skew=conv == "skew", tau_elem=tau == "element")
    coords, conn, up = on_dev(dev, w.coords, w.conn, w.up)
    m = ns.Mesh(coords, conn, colour=True)
    p = ns.Params(rho=w.rho, mu=w.mu, c_vreman=cv, convection=conv, tau=tau, scatter="colour")
    ref = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu, **okw)
    check_fp64(m.assemble(up, p).cpu().numpy(), ref)
    pb = ns.Params(rho=w.rho, mu=w.mu, c_vreman=cv, convection=conv, tau=tau,
                   scatter="block_colour")
    check_fp64(m.assemble(up, pb).cpu().numpy(), ref)
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    gref = oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu, **okw)
    for pp in (p, pb):
        g = m.assemble_vjp(up, torch.from_numpy(cot).to(dev), pp).cpu().numpy()
        assert relerr(g, gref) <= TOL_VJP_ORACLE
    m.close()


def test_colour_scatter_is_bitwise_reproducible(dev):
    w = mg.make_workload(24, jitter=0.3, order="random", mu=1e-4, mag_max=10.0)
    coords, conn, up = on_dev(dev, w.coords, w.conn, w.up)
    cot = torch.from_numpy(mg.normal((4, w.n_nodes), seed=mg.SEED_COT)).to(dev)
    m = ns.Mesh(coords, conn, colour=True)
    for prec in ("fp64", "mixed"):
        u = up if prec == "fp64" else up.float()
        c = cot if prec == "fp64" else cot.float()
        pa = ns.Params(rho=w.rho, mu=w.mu, scatter="atomic", precision=prec)
        ra = m.assemble(u, pa).cpu().numpy()
        for sc in ("colour", "block_colour"):
            p = ns.Params(rho=w.rho, mu=w.mu, scatter=sc, precision=prec)
            r1, r2 = m.assemble(u, p), m.assemble(u, p)
            assert torch.equal(r1, r2)
            g1, g2 = m.assemble_vjp(u, c, p), m.assemble_vjp(u, c, p)
            assert torch.equal(g1, g2)
            # and the same sums as the atomic scatter up to rounding (the
            # mixed block path sums each node in compensated float first)
            assert relerr(r1.cpu().numpy(), ra) <= (TOL_FP64 if prec == "fp64" else 1e-9)
    # explicit steps through the coloured assembly are reproducible too
    p = ns.Params(rho=w.rho, mu=w.mu, scatter="colour")
    a, b = up.clone(), up.clone()
    for _ in range(2):
        m.explicit_step(a, 1e-4, "ssprk3", p)
        m.explicit_step(b, 1e-4, "ssprk3", p)
    assert torch.equal(a, b)
    m.close()


def test_colour_scatter_ragged_element_counts(dev):
    w = mg.make_workload(6, jitter=0.2, order="random")
    for E in (1, 2, 31, 129, 257, 1000):
        conn = np.ascontiguousarray(w.conn[:, :E])
        ref = oracle.assemble(w.coords, conn, w.up, 1.0, 1e-2)
        coords, conn_d, up = on_dev(dev, w.coords, conn, w.up)
        m = ns.Mesh(coords, conn_d, colour=True)
        info = m.info()
        check_colouring(m.element_colours().cpu().numpy(), conn, w.n_nodes, info["n_colours"])
        check_block_colouring(m.element_colours("block_colour").cpu().numpy(),
                              m.element_colours("block").cpu().numpy(), conn,
                              info["n_block_colours"], info["n_blocks"])
        cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
        gref = oracle.vjp(w.coords, conn, w.up, cot, 1.0, 1e-2)
        cot_d = torch.from_numpy(cot).to(dev)
        for sc in ("colour", "block_colour"):
            check_fp64(m.assemble(up, ns.Params(rho=1.0, mu=1e-2, scatter=sc)).cpu().numpy(), ref)
        for sc in ("colour", "block", "block_colour"):
            g = m.assemble_vjp(up, cot_d, ns.Params(rho=1.0, mu=1e-2, scatter=sc)).cpu().numpy()
            assert relerr(g, gref) <= TOL_VJP_ORACLE, (E, sc)
        m.close()


def test_colour_scatter_needs_a_coloured_mesh(dev):
    w = mg.make_workload(4)
    coords, conn, up = on_dev(dev, w.coords, w.conn, w.up)
    m = ns.Mesh(coords, conn)
    for sc in ("colour", "block_colour"):
        with pytest.raises(ns.NSRHSError) as ei:
            m.assemble(up, ns.Params(scatter=sc))
        assert ei.value.status == _abi.EUNSUPPORTED
    with pytest.raises(ns.NSRHSError) as ei:
        m.assemble_vjp(up, up, ns.Params(scatter="colour"))
    assert ei.value.status == _abi.EUNSUPPORTED
    with pytest.raises(ns.NSRHSError) as ei:
        m.element_colours()
    assert ei.value.status == _abi.EUNSUPPORTED
    m.close()


def fan_mesh(k):
    """k tetrahedra sharing only node 0 (the origin); tet j spans the scaled
    unit axes: every element needs its own colour."""
    coords = [(0.0, 0.0, 0.0)]
    conn = []
    for j in range(k):
        s = 1.0 + j
        base = len(coords)
        coords += [(s, 0.0, 0.0), (0.0, s, 0.0), (0.0, 0.0, s)]
        conn.append((0, base, base + 1, base + 2))
    return (np.ascontiguousarray(np.array(coords).T),
            np.ascontiguousarray(np.array(conn, dtype=np.int32).T))


def test_colouring_limit(dev):
    """128 elements around one node take the 128 colours there are; 129
    cannot be coloured and mesh creation reports it."""
    coords, conn = fan_mesh(128)
    c_d, n_d = on_dev(dev, coords, conn)
    m = ns.Mesh(c_d, n_d, colour=True)
    assert m.info()["n_colours"] == 128
    cols = m.element_colours().cpu().numpy()
    assert np.array_equal(np.sort(cols), np.arange(128))
    m.close()
    coords, conn = fan_mesh(129)
    c_d, n_d = on_dev(dev, coords, conn)
    with pytest.raises(ns.NSRHSError) as ei:
        ns.Mesh(c_d, n_d, colour=True)
    assert ei.value.status == _abi.EUNSUPPORTED
    ns.Mesh(c_d, n_d).close()   # without colouring the mesh is fine

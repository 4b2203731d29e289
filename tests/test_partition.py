"""Host logic of a sharded assembly (the paper's Sec. VII: every process
assembles its own elements, one sum over the interface nodes): the slab
partition, the local numbering and the interface exchange, checked against
the oracle's assembly of the whole mesh. No GPU."""
import numpy as np
import pytest
import torch

import meshgen as mg
import oracle
from paper_2403_08777_gb300 import partition as pt


def _mesh(kind):
    if kind == "kuhn":
        return mg.make_workload(6, jitter=0.2, order="random", mu=1e-3, mag_max=2.0)
    m = mg.delaunay_mesh(5)
    w0 = mg.make_workload(5, mu=1e-3, mag_max=2.0)
    coords, conn = m[0], m[1]
    up = mg.normal((4, coords.shape[1]), seed=7)
    return mg.Workload("delaunay5", 5, coords, conn, up, w0.rho, w0.mu)


@pytest.mark.parametrize("kind", ["kuhn", "delaunay"])
@pytest.mark.parametrize("n_parts,axis", [(1, 2), (2, 2), (3, 0), (5, 1)])
def test_partition_invariants(kind, n_parts, axis):
    w = _mesh(kind)
    N, E = w.coords.shape[1], w.conn.shape[1]
    parts = pt.slab_partition(w.coords, w.conn, n_parts, axis=axis)
    assert [p.index for p in parts] == list(range(n_parts))
    # every element in exactly one part, counts within one of each other
    allel = np.concatenate([p.elems for p in parts])
    assert np.array_equal(np.sort(allel), np.arange(E))
    sizes = [p.n_elems for p in parts]
    assert max(sizes) - min(sizes) <= 1
    # slabs: along the axis, a part's centroids do not pass the next part's
    cent = w.coords[axis][w.conn].mean(axis=0)
    for a, b in zip(parts, parts[1:]):
        assert cent[a.elems].max() <= cent[b.elems].min()
    touched = np.zeros((n_parts, N), bool)
    for p in parts:
        # local connectivity maps back to the global one
        assert p.conn.dtype == np.int32 and p.conn.shape == (4, p.n_elems)
        assert np.array_equal(p.nodes[p.conn], w.conn[:, p.elems])
        # local nodes: exactly the touched ones, owned first, each ascending
        tn = np.unique(w.conn[:, p.elems])
        assert np.array_equal(np.sort(p.nodes), tn)
        touched[p.index, tn] = True
        own, gh = p.nodes[:p.n_owned], p.nodes[p.n_owned:]
        assert np.all(np.diff(own) > 0) and np.all(np.diff(gh) > 0)
    count = touched.sum(axis=0)
    owner = np.argmax(touched, axis=0)
    iface = np.flatnonzero(count > 1)
    for p in parts:
        assert np.all(owner[p.nodes[:p.n_owned]] == p.index)
        assert np.all(owner[p.nodes[p.n_owned:]] < p.index)   # owned by a lower part
        assert p.n_iface == iface.size
        assert np.array_equal(p.nodes[p.iface_local], iface[p.iface_slot])
        assert np.array_equal(np.sort(p.nodes[p.iface_local]),
                              np.intersect1d(p.nodes, iface))
    # every touched node has exactly one owner
    assert sum(p.n_owned for p in parts) == int((count > 0).sum())
    if n_parts == 1:
        assert iface.size == 0 and parts[0].n_owned == parts[0].n_nodes


@pytest.mark.parametrize("kind", ["kuhn", "delaunay"])
@pytest.mark.parametrize("n_parts", [2, 4])
def test_local_assembly_and_exchange_give_the_global_rhs(kind, n_parts):
    """Each part assembled alone over its local nodes (the oracle on the
    sub-mesh), the interface buffers summed over the parts, written back:
    every local row, owned or ghost, equals the whole mesh's row; the VJP
    exchanges the same way."""
    w = _mesh(kind)
    full = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu)
    cot = mg.normal((4, w.coords.shape[1]), seed=mg.SEED_COT)
    gfull = oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu)
    parts = pt.slab_partition(w.coords, w.conn, n_parts)
    for ref, fn in ((full, lambda p: oracle.assemble(p.local(w.coords), p.conn, p.local(w.up),
                                                      w.rho, w.mu)),
                    (gfull, lambda p: oracle.vjp(p.local(w.coords), p.conn, p.local(w.up),
                                                 p.local(cot), w.rho, w.mu))):
        loc = [torch.from_numpy(fn(p)) for p in parts]
        # before the exchange an interface row holds only the part's share
        if parts[0].iface_local.size:
            r = loc[0][:, torch.from_numpy(parts[0].iface_local)].numpy()
            assert not np.allclose(r, ref[:, parts[0].nodes[parts[0].iface_local]])
        total = sum(pt.interface_rows(l, p) for l, p in zip(loc, parts))
        scale = np.abs(ref).max()
        for l, p in zip(loc, parts):
            pt.apply_interface(l, p, total)
            assert np.abs(l.numpy() - ref[:, p.nodes]).max() <= 1e-13 * scale


@pytest.mark.parametrize("kind", ["kuhn", "delaunay"])
@pytest.mark.parametrize("n_parts", [2, 3, 5])
def test_neighbour_exchange_gives_the_global_rhs(kind, n_parts):
    """Point-to-point exchange between parts sharing nodes, routed in
    process: the shared lists of two parts name the same nodes in the same
    order, and after the exchange every local row equals the whole mesh's.
    The messages carry the shared rows only: fewer than the all-reduce's
    n_parts copies of the whole interface vector."""
    w = _mesh(kind)
    full = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu)
    parts = pt.slab_partition(w.coords, w.conn, n_parts)
    for a in parts:
        for q, loc in a.shared.items():
            b = parts[q]
            assert np.array_equal(a.nodes[loc], b.nodes[b.shared[a.index]])
            assert np.all(np.diff(a.nodes[loc]) > 0)
    loc = [torch.from_numpy(oracle.assemble(p.local(w.coords), p.conn, p.local(w.up), w.rho, w.mu))
           for p in parts]
    sent = {p.index: {q: loc[p.index][:, torch.from_numpy(i)].clone() for q, i in p.shared.items()}
            for p in parts}
    for p in parts:
        pt.exchange_neighbours(loc[p.index], p, lambda sends, me=p.index: {q: sent[q][me] for q in sends})
    scale = np.abs(full).max()
    for l, p in zip(loc, parts):
        assert np.abs(l.numpy() - full[:, p.nodes]).max() <= 1e-13 * scale
    p2p = sum(len(i) for p in parts for i in p.shared.values())
    assert 0 < p2p <= n_parts * parts[0].n_iface


def test_exchange_with_a_summing_all_reduce():
    """exchange_interface calls the all-reduce once on a [4, n_iface] buffer
    holding only the part's rows."""
    w = _mesh("kuhn")
    parts = pt.slab_partition(w.coords, w.conn, 3)
    p = parts[1]
    loc = torch.arange(4 * p.n_nodes, dtype=torch.float64).reshape(4, p.n_nodes)
    seen = []

    def all_reduce(buf):
        seen.append(buf.clone())
        buf.mul_(3.0)

    before = loc.clone()
    pt.exchange_interface(loc, p, all_reduce)
    assert len(seen) == 1 and seen[0].shape == (4, p.n_iface)
    mask = torch.zeros(p.n_iface, dtype=torch.bool)
    mask[torch.from_numpy(p.iface_slot)] = True
    assert torch.all(seen[0][:, ~mask] == 0)
    il = torch.from_numpy(p.iface_local)
    assert torch.equal(loc[:, il], 3.0 * before[:, il])
    rest = torch.ones(p.n_nodes, dtype=torch.bool)
    rest[il] = False
    assert torch.equal(loc[:, rest], before[:, rest])


def test_partition_argument_errors():
    w = mg.make_workload(2)
    with pytest.raises(ValueError):
        pt.slab_partition(w.coords, w.conn, 0)
    with pytest.raises(ValueError):
        pt.slab_partition(w.coords, w.conn, w.conn.shape[1] + 1)
    with pytest.raises(ValueError):
        pt.slab_partition(w.coords, w.conn, 64)
    with pytest.raises(ValueError):
        pt.slab_partition(w.coords, w.conn, 2, axis=3)
    bad = w.conn.copy()
    bad[0, 0] = w.coords.shape[1]
    with pytest.raises(ValueError):
        pt.slab_partition(w.coords, bad, 2)
    with pytest.raises(ValueError):
        pt.slab_partition(w.coords.T, w.conn, 2)

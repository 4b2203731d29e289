"""Input generator checks (CPU): counts, conformity, orientation, volume,
renumbering validity and locality, determinism of the seeded streams."""
import numpy as np
import pytest

import meshgen as mg
import oracle


def _faces(conn):
    E = conn.shape[1]
    f = np.concatenate([conn[[1, 2, 3]], conn[[0, 2, 3]], conn[[0, 1, 3]], conn[[0, 1, 2]]], axis=1)
    f = np.sort(f.T, axis=1)
    return f


@pytest.mark.parametrize("n,jitter", [(1, 0.0), (3, 0.1), (6, 0.3)])
def test_counts_conformity_orientation(n, jitter):
    coords, conn, colour, _ = mg.box_mesh(n, jitter)
    N, E = (n + 1) ** 3, 6 * n ** 3
    assert coords.shape == (3, N) and conn.shape == (4, E)
    assert conn.min() == 0 and conn.max() == N - 1
    # every node used
    assert np.unique(conn).size == N
    # conforming: each face shared by 1 (boundary) or 2 (interior) tets
    f = _faces(conn)
    _, counts = np.unique(f, axis=0, return_counts=True)
    assert set(counts.tolist()) <= {1, 2}
    n_boundary = int((counts == 1).sum())
    assert n_boundary == 12 * n * n
    # boundary faces lie on the cube surface
    uf, counts = np.unique(f, axis=0, return_counts=True)
    bf = uf[counts == 1]
    xyz = coords[:, bf]  # [3][F][3]
    on_face = np.zeros(bf.shape[0], bool)
    for d in range(3):
        for val in (0.0, 1.0):
            on_face |= np.all(np.abs(xyz[d] - val) < 1e-15, axis=1)
    assert on_face.all()
    # positive orientation, volumes sum to the unit cube
    det = oracle.detj(coords, conn)
    assert (det > 0).all()
    assert abs(det.sum() / 6.0 - 1.0) < 1e-13
    # hex blocks: elements 6h..6h+5 all contain the hex's corner v0 and v7
    c6 = conn.reshape(4, -1, 6)
    assert (c6[0] == c6[0][:, :1]).all() and (c6[3] == c6[3][:, :1]).all()
    assert colour.min() >= 0 and colour.max() <= 7


def test_jitter_bounds_and_boundary_fixed():
    n, j = 8, 0.1
    coords, _, _, _ = mg.box_mesh(n, j)
    n1 = n + 1
    idx = np.arange(n1 ** 3)
    ijk = np.stack([idx % n1, (idx // n1) % n1, idx // (n1 * n1)]).astype(float) / n
    off = coords - ijk
    interior = np.all((ijk > 0) & (ijk < 1), axis=0)
    assert np.all(off[:, ~interior] == 0.0)
    assert np.abs(off[:, interior]).max() <= j / n + 1e-15
    assert np.abs(off[:, interior]).max() > 0.8 * j / n   # jitter actually applied
    # determinism
    c2, _, _, _ = mg.box_mesh(n, j)
    assert np.array_equal(coords, c2)


def test_jitter_03_repairs_flat_tets():
    coords, conn, _, n_red = mg.box_mesh(12, 0.3)
    det = oracle.detj(coords, conn)
    assert det.min() >= 0.05 / 12 ** 3 * (1 - 1e-12)
    assert n_red > 0


def test_fields_statistics():
    coords, conn, _, _ = mg.box_mesh(16, 0.1)
    up = mg.fields(coords, noise_sigma=0.0)
    x, y, z = 2 * np.pi * coords
    assert np.allclose(up[0], np.sin(x) * np.cos(y) * np.cos(z), atol=1e-14)
    assert np.allclose(up[1], -np.cos(x) * np.sin(y) * np.cos(z), atol=1e-14)
    assert np.all(up[2] == 0)
    assert up[3].min() >= -1 and up[3].max() < 1 and abs(up[3].mean()) < 0.05
    noisy = mg.fields(coords, noise_sigma=1e-2)
    d = (noisy - up)[:3].ravel()
    assert abs(d.std() - 1e-2) < 5e-4
    big = mg.fields(coords, noise_sigma=0.0, mag_max=10.0)
    m = np.linalg.norm((big - up)[:3], axis=0)
    assert m.max() <= 10.0 and m.max() > 9.0 and abs(m.mean() - 5.0) < 0.3


def test_renumberings_are_permutations_and_rcm_is_local():
    coords, conn, _, _ = mg.box_mesh(10, 0.1)
    N = coords.shape[1]
    rnd = mg.random_order(N)
    rcm = mg.rcm_order(conn, N)
    for o in (rnd, rcm):
        assert np.array_equal(np.sort(o), np.arange(N))
    _, c_rnd = mg.renumber(rnd, coords, conn)
    _, c_rcm = mg.renumber(rcm, coords, conn)
    assert mg.bandwidth(c_rcm) < mg.bandwidth(c_rnd) / 10
    assert mg.bandwidth(c_rcm) <= mg.bandwidth(conn)
    # renumbering preserves geometry
    c2, cn2 = mg.renumber(rcm, coords, conn)
    assert np.array_equal(c2[:, cn2], coords[:, conn])


def test_rcm_on_disconnected_mesh():
    coords, conn, _, _ = mg.box_mesh(2, 0.0)
    N = coords.shape[1]
    conn2 = np.concatenate([conn, conn + N], axis=1)
    order = mg.rcm_order(conn2, 2 * N)
    assert np.array_equal(np.sort(order), np.arange(2 * N))


def test_normal_stream():
    a = mg.normal(200000, seed=4)
    assert abs(a.mean()) < 0.01 and abs(a.std() - 1) < 0.01
    assert np.array_equal(a, mg.normal(200000, seed=4))
    assert not np.array_equal(a, mg.normal(200000, seed=5))


def test_delaunay_mesh_is_valid_and_unstructured():
    coords, conn = mg.delaunay_mesh(8, 0.3)
    N = coords.shape[1]
    assert np.unique(conn).size == N
    det = oracle.detj(coords, conn)
    assert (det > 0).all()
    assert abs(det.sum() / 6.0 - 1.0) < 1e-13
    f = _faces(conn)
    _, counts = np.unique(f, axis=0, return_counts=True)
    assert set(counts.tolist()) <= {1, 2}
    # valences vary (no hex-block structure)
    val = np.bincount(conn.ravel(), minlength=N)
    assert val.max() - val.min() > 10
    c2, cn2 = mg.delaunay_mesh(8, 0.3)
    assert np.array_equal(conn, cn2) and np.array_equal(coords, c2)


def test_msh_round_trip(tmp_path):
    coords, conn = mg.delaunay_mesh(4, 0.2)
    path = str(tmp_path / "m.msh")
    mg.write_msh(path, coords, conn)
    c2, cn2 = mg.read_msh(path)
    assert np.array_equal(coords, c2) and np.array_equal(conn, cn2)
    # non-tet elements are skipped, node tags need not be 1..N
    with open(path) as f:
        txt = f.read()
    txt = txt.replace("$Elements\n%d\n" % conn.shape[1],
                      "$Elements\n%d\n1 2 2 0 1 1 2 3\n" % (conn.shape[1] + 1))
    with open(path, "w") as f:
        f.write(txt)
    c3, cn3 = mg.read_msh(path)
    assert np.array_equal(cn3, conn)

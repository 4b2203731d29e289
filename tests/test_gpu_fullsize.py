"""Parity at the benchmark's full size, in the launch configuration bench.py
times: the 256^3-hex mesh (100,663,296 tets, 16,974,593 nodes, RCM order,
rho = 1, mu = 1e-4). The oracle cannot assemble 100M tets in seconds, so it
computes sampled outputs exactly: the RHS (or adjoint) at a node depends only
on the elements that contain it, so the oracle runs over those elements and
the two results are compared at the sampled nodes.
"""
import numpy as np
import pytest
import torch

import meshgen as mg
import oracle
import paper_2403_08777_gb300 as ns

pytestmark = pytest.mark.gpu

N_SAMPLES = 256


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ns.load_library()
    return torch.device("cuda:0")


def sampled(w, seed):
    rng = np.random.default_rng(seed)
    nodes = np.unique(rng.integers(0, w.n_nodes, N_SAMPLES))
    return nodes, oracle.submesh_for_nodes(w.conn, nodes)


def test_fullsize_fp64_forward_and_adjoint(dev):
    w = mg.paper_scale(n=256, order="rcm")
    assert w.n_elems == 100_663_296 and w.n_nodes == 16_974_593
    nodes, sub = sampled(w, 11)
    m = ns.Mesh(torch.from_numpy(w.coords).to(dev), torch.from_numpy(w.conn).to(dev))
    up = torch.from_numpy(w.up).to(dev)
    p = ns.Params(rho=w.rho, mu=w.mu)
    rhs = m.assemble(up, p)[:, torch.from_numpy(nodes).to(dev)].cpu().numpy()
    ref = oracle.assemble(w.coords, sub, w.up, w.rho, w.mu)[:, nodes]
    err = np.linalg.norm(rhs - ref) / np.linalg.norm(ref)
    assert err <= 1e-12, err
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    g = m.assemble_vjp(up, torch.from_numpy(cot).to(dev), p)
    g = g[:, torch.from_numpy(nodes).to(dev)].cpu().numpy()
    gref = oracle.vjp(w.coords, sub, w.up, cot, w.rho, w.mu)[:, nodes]
    gerr = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    assert gerr <= 1e-12, gerr
    # the same with the geometry formed in the call, and with the Vreman model
    idx = torch.from_numpy(nodes).to(dev)
    cot_d = torch.from_numpy(cot).to(dev)
    prc = ns.Params(rho=w.rho, mu=w.mu, geometry="recompute")
    x = m.assemble(up, prc)[:, idx].cpu().numpy()
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-12
    x = m.assemble_vjp(up, cot_d, prc)[:, idx].cpu().numpy()
    assert np.linalg.norm(x - gref) / np.linalg.norm(gref) <= 1e-12
    pv = ns.Params(rho=w.rho, mu=w.mu, c_vreman=0.07)
    refv = oracle.assemble(w.coords, sub, w.up, w.rho, w.mu, c_vreman=0.07)[:, nodes]
    x = m.assemble(up, pv)[:, idx].cpu().numpy()
    assert np.linalg.norm(x - refv) / np.linalg.norm(refv) <= 1e-12
    grefv = oracle.vjp(w.coords, sub, w.up, cot, w.rho, w.mu, c_vreman=0.07)[:, nodes]
    x = m.assemble_vjp(up, cot_d, pv)[:, idx].cpu().numpy()
    assert np.linalg.norm(x - grefv) / np.linalg.norm(grefv) <= 1e-12
    m.close()


def test_fullsize_mixed_precision(dev):
    w = mg.precision_case(n=256, order="rcm")
    nodes, sub = sampled(w, 12)
    m = ns.Mesh(torch.from_numpy(w.coords).to(dev), torch.from_numpy(w.conn).to(dev))
    assert m.info()["n_high_ar"] > 0
    up32 = torch.from_numpy(w.up).to(dev).float()
    x = m.assemble(up32, ns.Params(rho=w.rho, mu=w.mu, precision="mixed"))
    x = x[:, torch.from_numpy(nodes).to(dev)].cpu().numpy()
    ref = oracle.assemble(w.coords, sub, w.up, w.rho, w.mu)[:, nodes]
    err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err
    m.close()


def test_fullsize_one_pass_mixed_adjoint_and_colourings(dev):
    """The one-pass call, the mixed adjoint (block scatter) and the coloured
    scatters at full size, as the benchmark's forms run them."""
    w = mg.paper_scale(n=256, order="rcm")
    nodes, sub = sampled(w, 13)
    idx = torch.from_numpy(nodes).to(dev)
    m = ns.Mesh(torch.from_numpy(w.coords).to(dev), torch.from_numpy(w.conn).to(dev), colour=True)
    up = torch.from_numpy(w.up).to(dev)
    cot_h = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    cot = torch.from_numpy(cot_h).to(dev)
    ref = oracle.assemble(w.coords, sub, w.up, w.rho, w.mu)[:, nodes]
    gref = oracle.vjp(w.coords, sub, w.up, cot_h, w.rho, w.mu)[:, nodes]

    def err(x, r):
        return np.linalg.norm(x[:, idx].cpu().numpy() - r) / np.linalg.norm(r)

    r, g = m.assemble_rhs_vjp(up, cot, ns.Params(rho=w.rho, mu=w.mu))
    assert err(r, ref) <= 1e-12 and err(g, gref) <= 1e-12
    pm = ns.Params(rho=w.rho, mu=w.mu, precision="mixed")
    assert err(m.assemble_vjp(up.float(), cot.float(), pm), gref) <= 1e-6
    r, g = m.assemble_rhs_vjp(up.float(), cot.float(), pm)   # mixed one pass: blocks
    assert err(r, ref) <= 1e-5 and err(g, gref) <= 1e-6
    assert err(m.assemble(up, ns.Params(rho=w.rho, mu=w.mu, scatter="colour")), ref) <= 1e-12
    assert err(m.assemble_vjp(up, cot, ns.Params(rho=w.rho, mu=w.mu, scatter="colour")),
               gref) <= 1e-12
    pbc = ns.Params(rho=w.rho, mu=w.mu, precision="mixed", scatter="block_colour")
    assert err(m.assemble(up.float(), pbc), ref) <= 1e-5
    m.close()

"""Stored expected values (tests/golden/, written by make_golden.py from the
oracle only): the oracle still reproduces them (CPU; up to the rounding
differences between compilers and machines), and the CUDA path matches them
(GPU) within the FP64 tolerance."""
import os

import numpy as np
import pytest

import meshgen as mg
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    return np.loadtxt(os.path.join(GOLDEN, name)).T.copy()


def relerr(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def test_oracle_reproduces_the_stored_values():
    w = mg.tiny()
    rhs, vjp = load("rhs_kuhn8_lex.txt"), load("vjp_kuhn8_lex.txt")
    assert rhs.shape == (4, 729) and vjp.shape == (4, 729)
    assert relerr(oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu), rhs) <= 1e-13
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    assert relerr(oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu), vjp) <= 1e-13


@pytest.mark.gpu
def test_cuda_path_matches_the_stored_values():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_08777_gb300 as ns
    dev = torch.device("cuda:0")
    w = mg.tiny()
    rhs, vjp = load("rhs_kuhn8_lex.txt"), load("vjp_kuhn8_lex.txt")
    m = ns.Mesh(torch.from_numpy(w.coords).to(dev), torch.from_numpy(w.conn).to(dev))
    up = torch.from_numpy(w.up).to(dev)
    cot = torch.from_numpy(mg.normal((4, w.n_nodes), seed=mg.SEED_COT)).to(dev)
    p = ns.Params(rho=w.rho, mu=w.mu)
    x = m.assemble(up, p).cpu().numpy()
    assert relerr(x, rhs) <= 1e-12 and np.abs(x - rhs).max() <= 1e-12 * np.abs(rhs).max()
    assert relerr(m.assemble_vjp(up, cot, p).cpu().numpy(), vjp) <= 1e-12
    pm = ns.Params(rho=w.rho, mu=w.mu, precision="mixed")
    assert relerr(m.assemble(up.float(), pm).cpu().numpy(), rhs) <= 1e-5
    m.close()

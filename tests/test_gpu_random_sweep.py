"""Seeded random sweep of the parameter space, GPU against the oracle.

Each case draws, from its own seed, a mesh size (2..6 hexes a side), a
jitter (0..0.3 h), a node order, rho, mu (1e-4..1e-1, log-uniform), the
Vreman constant (off, or 0.05..0.2), the convective form, the tau mode, an
extra seeded velocity/pressure perturbation and a scatter, and checks the
forward, the adjoint and the one-pass call, FP64 and mixed, against the
oracle on the same inputs. Tolerances as the parity tests: FP64 forward
norm-wise 1e-12 and every entry within 1e-12 max|RHS|, FP64 adjoint 1e-12,
mixed form 1e-5."""
import numpy as np
import pytest
import torch

import meshgen as mg
import oracle
import paper_2403_08777_gb300 as ns

pytestmark = pytest.mark.gpu

N_CASES = 16


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ns.load_library()
    return torch.device("cuda:0")


def relerr(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def draw(k):
    r = np.random.default_rng(7000 + k)
    n = int(r.integers(2, 7))
    kw = dict(jitter=float(r.uniform(0.0, 0.3)), order=("lex", "random", "rcm")[int(r.integers(3))],
              rho=float(r.uniform(0.5, 2.0)), mu=float(10.0 ** r.uniform(-4.0, -1.0)))
    cv = 0.0 if r.integers(2) == 0 else float(r.uniform(0.05, 0.2))
    conv = ("convective", "skew")[int(r.integers(2))]
    tau = ("gauss", "element")[int(r.integers(2))]
    amp = float(r.uniform(0.0, 5.0))
    scatter = ("atomic", "block", "colour", "block_colour")[int(r.integers(4))]
    w = mg.make_workload(n, c_vreman=cv, **kw)
    up = w.up + amp * mg.normal(w.up.shape, seed=8000 + k)
    cot = mg.normal(w.up.shape, seed=9000 + k)
    return w, up, cot, cv, conv, tau, scatter


@pytest.mark.parametrize("k", range(N_CASES))
def test_random_case(dev, k):
    w, up, cot, cv, conv, tau, scatter = draw(k)
    okw = dict(c_vreman=cv, skew=conv == "skew", tau_elem=tau == "element")
    ref = oracle.assemble(w.coords, w.conn, up, w.rho, w.mu, **okw)
    gref = oracle.vjp(w.coords, w.conn, up, cot, w.rho, w.mu, **okw)
    m = ns.Mesh(torch.from_numpy(w.coords).to(dev), torch.from_numpy(w.conn).to(dev), colour=True)
    u = torch.from_numpy(np.ascontiguousarray(up)).to(dev)
    c = torch.from_numpy(cot).to(dev)
    kw = dict(rho=w.rho, mu=w.mu, c_vreman=cv, convection=conv, tau=tau)
    one_pass_scatter = "atomic" if scatter == "colour" else scatter
    # FP64
    p = ns.Params(scatter=scatter, **kw)
    x = m.assemble(u, p).cpu().numpy()
    assert relerr(x, ref) <= 1e-12
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()
    assert relerr(m.assemble_vjp(u, c, p).cpu().numpy(), gref) <= 1e-12
    r1, g1 = m.assemble_rhs_vjp(u, c, ns.Params(scatter=one_pass_scatter, **kw))
    assert relerr(r1.cpu().numpy(), ref) <= 1e-12
    assert relerr(g1.cpu().numpy(), gref) <= 1e-12
    # mixed
    pm = ns.Params(scatter=scatter, precision="mixed", **kw)
    u32, c32 = u.float(), c.float()
    assert relerr(m.assemble(u32, pm).cpu().numpy(), ref) <= 1e-5
    assert relerr(m.assemble_vjp(u32, c32, pm).cpu().numpy(), gref) <= 1e-5
    r2, g2 = m.assemble_rhs_vjp(u32, c32, ns.Params(scatter=one_pass_scatter, precision="mixed",
                                                    **kw))
    assert relerr(r2.cpu().numpy(), ref) <= 1e-5
    assert relerr(g2.cpu().numpy(), gref) <= 1e-5
    m.close()


def test_draws_cover_the_space():
    """The seeded draws reach every scatter, both convective forms, both tau
    modes, Vreman on and off, and every node order."""
    seen = {"scatter": set(), "conv": set(), "tau": set(), "vreman": set(), "order": set()}
    for k in range(N_CASES):
        r = np.random.default_rng(7000 + k)
        r.integers(2, 7)
        r.uniform(0.0, 0.3)
        seen["order"].add(int(r.integers(3)))
        r.uniform(0.5, 2.0)
        r.uniform(-4.0, -1.0)
        v = r.integers(2)
        if v:
            r.uniform(0.05, 0.2)
        seen["vreman"].add(int(v))
        seen["conv"].add(int(r.integers(2)))
        seen["tau"].add(int(r.integers(2)))
        r.uniform(0.0, 5.0)
        seen["scatter"].add(int(r.integers(4)))
    assert seen == {"scatter": {0, 1, 2, 3}, "conv": {0, 1}, "tau": {0, 1}, "vreman": {0, 1},
                    "order": {0, 1, 2}}

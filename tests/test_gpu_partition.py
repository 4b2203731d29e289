"""A sharded assembly's parts through the library on one GPU: each slab of
the package's partition is its own library mesh (local coordinates and
connectivity), assembled alone over its owned and ghost nodes; the parts'
interface buffers are summed (what a multi-process run's all-reduce does)
and written back, or the shared rows exchanged between neighbouring parts. Every local row then matches the oracle's row of the
whole mesh: FP64 RHS and VJP within 1e-12 of max|ref|, the mixed form's
RHS within 1e-5 and its VJP within 1e-6 norm-wise."""
import numpy as np
import pytest
import torch

import meshgen as mg
import oracle
import paper_2403_08777_gb300 as ns
from paper_2403_08777_gb300 import partition as pt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ns.load_library()
    return torch.device("cuda:0")


@pytest.mark.parametrize("n_parts", [2, 4])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_slab_parts_on_one_gpu_match_the_whole_mesh(dev, n_parts, precision):
    w = mg.make_workload(12, jitter=0.2, order="rcm", mu=1e-3, mag_max=2.0)
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    full = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu)
    gfull = oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu)
    parts = pt.slab_partition(w.coords, w.conn, n_parts)
    p = ns.Params(rho=w.rho, mu=w.mu, precision=precision)
    dt = torch.float32 if precision == "mixed" else torch.float64
    rs, gs = [], []
    for part in parts:
        m = ns.Mesh(torch.from_numpy(part.local(w.coords)).to(dev),
                    torch.from_numpy(part.conn).to(dev))
        u = torch.from_numpy(part.local(w.up)).to(dev, dt)
        c = torch.from_numpy(part.local(cot)).to(dev, dt)
        r, g = m.assemble_rhs_vjp(u, c, p)
        rs.append(r)
        gs.append(g)
        m.close()
    for loc, ref, tol in ((rs, full, 1e-5), (gs, gfull, 1e-6)):
        # the point-to-point exchange on copies (messages routed in process)
        loc2 = [l.clone() for l in loc]
        sent = {a.index: {q: loc2[a.index][:, torch.as_tensor(i, device=dev)].clone()
                          for q, i in a.shared.items()} for a in parts}
        for a in parts:
            pt.exchange_neighbours(loc2[a.index], a,
                                   lambda sends, me=a.index: {q: sent[q][me] for q in sends})
        total = sum(pt.interface_rows(l, part) for l, part in zip(loc, parts))
        for l, l2, part in zip(loc, loc2, parts):
            pt.apply_interface(l, part, total)
            rr = ref[:, part.nodes]
            for x in (l.cpu().numpy(), l2.cpu().numpy()):
                if precision == "fp64":
                    assert np.abs(x - rr).max() <= 1e-12 * np.abs(ref).max()
                else:
                    assert np.linalg.norm(x - rr) <= tol * np.linalg.norm(rr)

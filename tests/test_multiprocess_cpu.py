"""Multi-process paths on CPU with the gloo backend (world size 2).

* bench.py's cross-rank reductions: the timed region is the slowest rank's
  and the rate counts the units of every rank.
* The partitioned assembly a multi-GPU run would use (§VII of the paper: the
  assembly is trivially parallel): every rank assembles its own slice of the
  elements and one sum over ranks of the nodal vectors gives the full RHS.
  Checked with the oracle.
* The same with the package's slab partition: every rank assembles its
  sub-mesh over its owned and ghost nodes only, and one all-reduce of the
  interface rows (exchange_interface), or point-to-point messages with the
  ranks it shares nodes with (exchange_neighbours), make every local row
  equal to the whole mesh's, for the RHS and the VJP.
"""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, task, q):
    try:
        sys.path.insert(0, ROOT)
        import torch
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                                world_size=world)
        if task == "bench":
            import bench
            t = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
            rate = bench.whole_job_rate(1000, world, t / 1e3)
            q.put((rank, t, rate))
        elif task in ("slab", "slab_p2p"):
            import meshgen as mg
            import oracle
            from paper_2403_08777_gb300 import partition as pt
            w = mg.make_workload(6, jitter=0.2, order="random", mu=1e-3, mag_max=2.0)
            cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
            part = pt.slab_partition(w.coords, w.conn, world)[rank]
            lc, lu = part.local(w.coords), part.local(w.up)
            r = torch.from_numpy(oracle.assemble(lc, part.conn, lu, w.rho, w.mu))
            g = torch.from_numpy(oracle.vjp(lc, part.conn, lu, part.local(cot), w.rho, w.mu))
            if task == "slab":
                pt.exchange_interface(r, part, dist.all_reduce)
                pt.exchange_interface(g, part, dist.all_reduce)
            else:  # point-to-point between the parts sharing nodes
                pt.exchange_neighbours(r, part, pt.torch_sendrecv())
                pt.exchange_neighbours(g, part, pt.torch_sendrecv())
            full = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu)[:, part.nodes]
            gfull = oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu)[:, part.nodes]
            err = max(float(np.abs(r.numpy() - full).max() / np.abs(full).max()),
                      float(np.abs(g.numpy() - gfull).max() / np.abs(gfull).max()))
            q.put((rank, err, part.n_iface))
        else:
            import meshgen as mg
            import oracle
            w = mg.make_workload(5, jitter=0.2, order="random", mu=1e-3, mag_max=2.0)
            E = w.n_elems
            e0, e1 = rank * E // world, (rank + 1) * E // world
            part = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu, e0=e0, e1=e1)
            t = torch.from_numpy(part)
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            full = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu)
            q.put((rank, float(np.abs(t.numpy() - full).max()), float(np.abs(full).max())))
        dist.destroy_process_group()
    except Exception as exc:  # report to the parent instead of hanging it
        q.put((rank, "error", repr(exc)))


def _run(task, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, task, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    for r in out:
        assert r[1] != "error", r
    return sorted(out)


def test_bench_reductions_gloo():
    out = _run("bench")
    for _, t, rate in out:
        assert t == 15.0                      # the slowest rank's time
        assert rate == pytest.approx(2 * 1000 / 0.015)


def test_partitioned_assembly_interface_sum_gloo():
    for _, err, scale in _run("partition"):
        assert err <= 1e-14 * scale


@pytest.mark.parametrize("task", ["slab", "slab_p2p"])
@pytest.mark.parametrize("world", [2, 3])
def test_slab_partition_exchange_gloo(world, task):
    out = _run(task, world)
    for _, err, n_iface in out:
        assert n_iface > 0
        assert err <= 1e-13

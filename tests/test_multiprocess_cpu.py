"""Multi-process paths on CPU with the gloo backend (world size 2).

* bench.py's cross-rank reductions: the timed region is the slowest rank's
  and the rate counts the units of every rank.
* The partitioned assembly a multi-GPU run would use (§VII of the paper: the
  assembly is trivially parallel): every rank assembles its own slice of the
  elements and one sum over ranks of the nodal vectors (the interface-node
  exchange) gives the full RHS. Checked with the oracle.
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

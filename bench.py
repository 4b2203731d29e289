#!/usr/bin/env python3
"""Benchmark of the tetrahedral Navier-Stokes RHS assembly on one GB300.

One step = one pass of the whole hot path over the workload: the FP64 RHS
assembly (zeroing + gather + element arithmetic + scatter) followed by its
adjoint (vector-Jacobian product) on the same nodal fields.

Workload (stands in for the paper's 32M-tet Bolund LES mesh, Sec. III-A,
which is not available): unit cube of 256^3 hexes split into 6 Kuhn tets
each (100,663,296 tets, 16,974,593 nodes), interior nodes jittered by
+-0.1 h, RCM node order, rho = 1, mu = 1e-4, velocity = Taylor-Green +
N(0, 1e-2) noise + m*d with m ~ U(0, 10) and d uniform on the sphere,
pressure ~ U(-1, 1), seeded and synthetic.

Prints one JSON line (rank 0): `value` from the device-resident step,
`e2e` through StepPipeline from pinned host buffers, `roofline` for the
dominant kernel (the adjoint) against the FP64 pipe rate, `cpu_baseline`
(the oracle on the host cores), sampled clocks, and under `forms` the other
configurations: formulation variants, the one-pass RHS + adjoint, the
element-matrix comparison path, explicit SSP-RK3 steps (and small-mesh steps
from a CUDA graph), the scatter sweep (atomic / block / element colouring /
block colouring), the mixed-precision forward and adjoint with their errors,
the unstructured mesh, random vs RCM node order and the 64^3 adjoint.
--impl reference times the CPU oracle instead (bounded sample, host cores).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import meshgen as mg  # noqa: E402

METRIC = "tets assembled/sec + FP64 TF/s (fraction of roofline), FP32 & adjoint vs plain FP64"
UNIT = "tets/s"

# Algorithmic FP64 operations per tet and call of the kernels' formulation
# (add/sub/mul = 1, fused multiply-add = 2, sqrt/reciprocal/cube root = 1),
# counted by instantiating the element code with a counting scalar
# (tests/test_flop_count.py keeps these numbers in step with the source).
# The element geometry (43 flops per tet) is computed once per mesh and
# cached, so it is not part of a call.
FLOPS_PER_TET = {"fwd": 513, "vjp": 1095, "rhs_vjp": 1385}
FLOPS_PER_TET_VREMAN = {"fwd": 564, "vjp": 1216, "rhs_vjp": 1507}

# The METHOD's own operation count per tet and call (the oracle's definition
# recorded as an expression DAG with constants folded and common
# subexpressions once; the adjoint adds one reverse-mode sweep over it), with
# the geometry nodes (coordinates only) separate: the work the restructured
# kernels replace. tests/test_flop_count.py recomputes these from the oracle.
FLOPS_PER_TET_METHOD = {"fwd": 932, "vjp": 2188, "geometry": 62}
FLOPS_PER_TET_METHOD_VREMAN = {"fwd": 1020, "vjp": 2445, "geometry": 61}

# Forming the element geometry from the node coordinates (edges, cofactors,
# determinant, reciprocal, reciprocal cube root): the same census. The
# default calls read it from the per-mesh cache; geometry="recompute" forms
# it in the call.
FLOPS_GEOMETRY = 43

# DRAM bytes per tet (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of each kernel on the 128^3-hex RCM mesh, scaled to a launch by
# the element count (traffic grows in proportion). None once a kernel has
# changed since its counters were taken.
DRAM_BYTES_PER_TET = {"fwd_fp64": 157.7, "vjp_fp64": 187.9,
                      "fwd_mixed": 92.4, "vjp_mixed": 106.6}

# Algorithmic (compulsory) bytes per tet with ideal node reuse (N/E = 0.1686
# on the Kuhn mesh): connectivity or block map 16, cached geometry 88 (f64) or
# 44 (f32), nodal reads and RHS read-modify-writes per node; see the kernels'
# roofline table in the design notes.
ALG_BYTES_PER_TET = {"fwd_fp64": 120.0, "vjp_fp64": 126.0, "fwd_mixed": 75.0, "vjp_mixed": 78.0}

# FP64 FMA lanes per SM per clock on GB300 (1.25 TF/s nominal at 2.07 GHz).
FP64_LANES_PER_SM = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=256, help="hexes per cube edge")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision lines")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--unstructured", type=int, default=64,
                    help="also time a Delaunay mesh of an (n+1)^3 jittered lattice (0: skip)")
    ap.add_argument("--locality", type=int, default=128,
                    help="also time random vs RCM node order on an n^3-hex mesh (0: skip)")
    ap.add_argument("--sample-fwd", type=int, default=1 << 20,
                    help="oracle forward elements per host process")
    ap.add_argument("--sample-vjp", type=int, default=1 << 16,
                    help="oracle adjoint elements per host process")
    ap.add_argument("--sample-ref", type=int, default=1 << 16,
                    help="--impl reference: elements per host process and step")
    ap.add_argument("--profile", choices=["fp64", "mixed"], default=None,
                    help="for Nsight Compute: only `--steps` forward and adjoint launches of "
                         "that form on the --n mesh (after --warmup), no JSON line")
    return ap.parse_args()


def workload(n: int):
    return mg.paper_scale(n=n, order="rcm")


# ---------------------------------------------------------------------------
# CPU oracle baseline (fork-based pool, started before any CUDA call).

_W = None


def _compact(e0, e1):
    conn = _W.conn[:, e0:e1]
    nodes, inv = np.unique(conn, return_inverse=True)
    return (np.ascontiguousarray(_W.coords[:, nodes]), inv.reshape(conn.shape).astype(np.int32),
            np.ascontiguousarray(_W.up[:, nodes]))


def _oracle_slice(args):
    import oracle
    e0, e1, kind, seed = args
    coords, conn, up = _compact(e0, e1)
    if kind == "fwd":
        t = time.perf_counter()
        oracle.assemble(coords, conn, up, _W.rho, _W.mu, c_vreman=_W.c_vreman)
        return time.perf_counter() - t
    cot = mg.normal(up.shape, seed=seed)
    t = time.perf_counter()
    oracle.vjp(coords, conn, up, cot, _W.rho, _W.mu, c_vreman=_W.c_vreman)
    return time.perf_counter() - t


def cpu_oracle_rates(w, procs: int, n_fwd: int, n_vjp: int, repeats: int = 1):
    """Oracle tets/s for the forward and the adjoint, `procs` processes each
    over its own slice of consecutive elements (nodes compacted per slice).
    Returns (fwd_rate, vjp_rate, step_rate, wall_times)."""
    import oracle
    oracle.build()
    global _W
    _W = w
    E = w.n_elems
    procs = max(1, procs)
    n_fwd = min(n_fwd, E // procs)
    n_vjp = min(n_vjp, E // procs)
    ctx = mp.get_context("fork")
    walls = []
    with ctx.Pool(procs) as pool:
        for _ in range(repeats):
            t0 = time.perf_counter()
            pool.map(_oracle_slice, [(i * n_fwd, (i + 1) * n_fwd, "fwd", 0) for i in range(procs)])
            t1 = time.perf_counter()
            pool.map(_oracle_slice, [(i * n_vjp, (i + 1) * n_vjp, "vjp", mg.SEED_COT)
                                     for i in range(procs)])
            t2 = time.perf_counter()
            walls.append((t1 - t0, t2 - t1))
    tf = statistics.median(x[0] for x in walls)
    tv = statistics.median(x[1] for x in walls)
    fwd_rate = procs * n_fwd / tf
    vjp_rate = procs * n_vjp / tv
    step_rate = 1.0 / (1.0 / fwd_rate + 1.0 / vjp_rate)
    sample = (f"{procs} host processes, each over its own {n_fwd} (forward) and {n_vjp} "
              f"(adjoint) consecutive elements of the {w.name} mesh, nodes compacted per slice; "
              f"rate = elements / wall time, step rate = 1/(1/fwd + 1/adjoint)")
    return fwd_rate, vjp_rate, step_rate, sample, walls


def cpu_oracle_serial(w, n_fwd: int, n_vjp: int):
    """The same oracle on one core (this process): forward and adjoint tets/s
    over the first n_fwd / n_vjp elements of the mesh."""
    global _W
    _W = w
    tf = _oracle_slice((0, min(n_fwd, w.n_elems), "fwd", 0))
    tv = _oracle_slice((0, min(n_vjp, w.n_elems), "vjp", mg.SEED_COT))
    return {"cores": 1, "fwd_tets_per_s": min(n_fwd, w.n_elems) / tf,
            "vjp_tets_per_s": min(n_vjp, w.n_elems) / tv}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# Clock sampling during the timed region.

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", gpu_index], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------

def max_over_ranks(value: float, world: int, device) -> float:
    """Largest value over all ranks (the slowest rank's time); identity for 1 rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Units of all ranks (weak scaling: every rank has the full workload) per second."""
    return world * units_per_rank / seconds


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def l2_note(w):
    """How the step's inputs compare with the 129 MB L2 (no flush is needed
    when they are far larger)."""
    conn, geom, nodal = 16 * w.n_elems, 88 * w.n_elems, 4 * 32 * w.n_nodes
    tot = conn + geom + nodal
    where = "larger than" if tot > 4 * 129e6 else "not larger than"
    return (f"inputs {where} L2 (129 MB): per step {conn / 1e9:.2f} GB connectivity, "
            f"{geom / 1e9:.2f} GB cached geometry, {nodal / 1e9:.2f} GB nodal arrays "
            f"(u, p, cotangent, RHS, gradient)")


def bench_config(w, world: int) -> dict:
    """The workload description both arms print (identical keys and values)."""
    return {"workload": w.name, "n_tets": w.n_elems, "n_nodes": w.n_nodes,
            "rho": w.rho, "mu": w.mu, "jitter": w.jitter, "order": w.order,
            "step": "fp64 forward assembly + fp64 adjoint (VJP)",
            "l2": l2_note(w),
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """The oracle as it stands on the host cores: every step is the FP64
    forward and then the adjoint over the same bounded sample of the
    workload's elements (consecutive slices, one per host process, nodes
    compacted per slice). ms_per_step is the wall time of those steps, so
    steps x ms_per_step is the time actually spent; value = sampled elements
    per step / step time, in the same tets/s of a forward + adjoint step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = workload(args.n)
    import oracle
    oracle.build()
    global _W
    _W = w
    procs = host_cores()
    per = max(1, min(args.sample_ref, w.n_elems // procs))
    n_sample = procs * per
    tasks_f = [(i * per, (i + 1) * per, "fwd", 0) for i in range(procs)]
    tasks_v = [(i * per, (i + 1) * per, "vjp", mg.SEED_COT) for i in range(procs)]
    steps_ms, fwd_s, vjp_s = [], [], []
    with mp.get_context("fork").Pool(procs) as pool:
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_slice, tasks_f)
            t1 = time.perf_counter()
            pool.map(_oracle_slice, tasks_v)
            t2 = time.perf_counter()
            if k >= args.warmup:
                steps_ms.append(1e3 * (t2 - t0))
                fwd_s.append(t1 - t0)
                vjp_s.append(t2 - t1)
    ms = sum(steps_ms) / len(steps_ms)
    value = n_sample / (ms * 1e-3)
    sample = (f"each step: the forward and then the adjoint over the same {n_sample} elements "
              f"({procs} host processes x {per} consecutive elements of the {w.name} mesh, "
              f"nodes compacted per slice); value = {n_sample} tets / mean step wall time")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": bench_config(w, world),
            "sample": {"tets_per_step": n_sample, "fraction_of_workload": n_sample / w.n_elems},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": sample,
                             "fwd_tets_per_s": n_sample / statistics.mean(fwd_s),
                             "vjp_tets_per_s": n_sample / statistics.mean(vjp_s)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    world, rank, local = dist_env()
    w = workload(args.n)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        procs = host_cores()
        fwd, vjp, step, sample, _ = cpu_oracle_rates(w, procs, args.sample_fwd, args.sample_vjp)
        cpu = {"value": step, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample,
               "fwd_tets_per_s": fwd, "vjp_tets_per_s": vjp,
               "serial": cpu_oracle_serial(w, args.sample_fwd, args.sample_vjp)}

    import torch
    import paper_2403_08777_gb300 as ns
    from paper_2403_08777_gb300 import _abi

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    lib = ns.load_library()

    coords = torch.from_numpy(w.coords).to(dev)
    conn = torch.from_numpy(w.conn).to(dev)
    up = torch.from_numpy(w.up).to(dev)
    cot_h = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    cot = torch.from_numpy(cot_h).to(dev)
    t_mesh = time.perf_counter()
    mesh = ns.Mesh(coords, conn, colour=True)
    torch.cuda.synchronize(dev)
    t_mesh = time.perf_counter() - t_mesh
    del coords, conn
    p = ns.Params(rho=w.rho, mu=w.mu, c_vreman=w.c_vreman)
    rhs = torch.empty((4, w.n_nodes), dtype=torch.float64, device=dev)
    grad = torch.empty_like(rhs)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        mesh.assemble(up, p, out=rhs)
        if evs is not None:
            evs[1].record(stream)
        mesh.assemble_vjp(up, cot, p, out=grad)
        if evs is not None:
            evs[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]
    sampler = ClockSampler(gpu_index)
    time.sleep(0.3)
    per = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter()
    start.record(stream)
    for k in range(args.steps):
        step(per[k])
    end.record(stream)
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall
    barrier()
    clocks = sampler.stop()
    ms_total = max_over_ranks(start.elapsed_time(end), world, dev)
    fwd_ms = [e[0].elapsed_time(e[1]) for e in per]
    vjp_ms = [e[1].elapsed_time(e[2]) for e in per]
    ms_step = ms_total / args.steps
    value = whole_job_rate(w.n_elems, world, ms_step * 1e-3)

    # ---- end to end: host buffers, copies inside the timed region ----
    # StepPipeline (public API): every step copies (u, p) and the cotangent in
    # from pinned host memory and the RHS and gradient out; the copies of one
    # step overlap the compute of its neighbours.
    up_h = torch.from_numpy(w.up).pin_memory()
    cot_hp = torch.from_numpy(cot_h).pin_memory()
    rhs_h = [torch.empty((4, w.n_nodes), dtype=torch.float64).pin_memory() for _ in range(2)]
    grad_h = [torch.empty((4, w.n_nodes), dtype=torch.float64).pin_memory() for _ in range(2)]
    pipe = ns.StepPipeline(mesh, p)
    for k in range(args.warmup):
        pipe.submit(k, up_h, cot_hp, rhs_h[k % 2], grad_h[k % 2])
    pipe.synchronize()
    torch.cuda.synchronize(dev)
    barrier()
    t_e2e = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(pipe.s_in)
    for k in range(args.steps):
        pipe.submit(k, up_h, cot_hp, rhs_h[k % 2], grad_h[k % 2])
    pipe.s_out.wait_stream(pipe.s_cmp)
    e1.record(pipe.s_out)
    pipe.synchronize()
    t_e2e = time.perf_counter() - t_e2e
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev) / args.steps
    bytes_nodal = 4 * w.n_nodes * 8
    del pipe

    # ---- FMA peaks (live) ----
    sink = torch.empty(sm_blocks(dev) * 256, dtype=torch.float64, device=dev)

    def probe(fp64: bool, iters: int) -> float:
        blocks = sm_blocks(dev)
        lib.nsrhs_probe_fma(int(fp64), blocks, 1000, _ptr(sink), _stream(stream))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rc = lib.nsrhs_probe_fma(int(fp64), blocks, iters, _ptr(sink), _stream(stream))
        b.record(stream)
        torch.cuda.synchronize(dev)
        assert rc == 0
        return blocks * 256 * 16 * iters * 2 / (a.elapsed_time(b) * 1e-3) / 1e12

    fp64_probe = max(probe(True, 12000) for _ in range(3))
    fp32_probe = max(probe(False, 200000) for _ in range(3))
    # FP64 pipe peak from the hardware rate: 2 FP64 FMA lanes per SM per clock
    # (GB300's nominal 1.25 TF/s at 2.07 GHz on 152 SMs), at the SM clock
    # sampled during the timed region. The FMA-chain probe reaches ~84 % of
    # the pipe (ncu), the element kernels ~89 %, so the probe under-states it.
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = clocks.get("sm_mhz") or 2070.0
    fp64_peak = FP64_LANES_PER_SM * 2 * n_sm * clk_mhz * 1e6 / 1e12

    # ---- mixed precision ----
    forms = {}
    fwd_med, vjp_med = statistics.median(fwd_ms), statistics.median(vjp_ms)
    flops = FLOPS_PER_TET_VREMAN if w.c_vreman else FLOPS_PER_TET
    forms["fwd_fp64"] = {"ms": fwd_med, "tets_per_s": w.n_elems / (fwd_med * 1e-3),
                         "tflops": flops["fwd"] * w.n_elems / (fwd_med * 1e-3) / 1e12}
    forms["vjp_fp64"] = {"ms": vjp_med, "tets_per_s": w.n_elems / (vjp_med * 1e-3),
                         "tflops": flops["vjp"] * w.n_elems / (vjp_med * 1e-3) / 1e12,
                         "vs_fwd_fp64": fwd_med / vjp_med}
    for k in ("fwd_fp64", "vjp_fp64"):
        forms[k]["frac_fp64_pipe"] = forms[k]["tflops"] / fp64_peak
    # the Vreman model switched on (c_v = 0.07; the configurations give only
    # rho and mu, so the headline runs without it), and the element geometry
    # formed from the coordinates in every call instead of read from the cache
    def pipe_line(ms, flops_per_tet, extra=None):
        tf = flops_per_tet * w.n_elems / (ms * 1e-3) / 1e12
        d = {"ms": ms, "tets_per_s": w.n_elems / (ms * 1e-3), "flops_per_tet": flops_per_tet,
             "tflops": tf, "frac_fp64_pipe": tf / fp64_peak}
        d.update(extra or {})
        return d

    pvr = ns.Params(rho=w.rho, mu=w.mu, c_vreman=0.07)
    t = _timed(lambda: mesh.assemble(up, pvr, out=rhs), dev, stream, args)
    forms["fwd_fp64_vreman"] = pipe_line(t, FLOPS_PER_TET_VREMAN["fwd"], {"c_vreman": 0.07})
    t = _timed(lambda: mesh.assemble_vjp(up, cot, pvr, out=grad), dev, stream, args)
    forms["vjp_fp64_vreman"] = pipe_line(t, FLOPS_PER_TET_VREMAN["vjp"], {"c_vreman": 0.07})
    prc = ns.Params(rho=w.rho, mu=w.mu, c_vreman=w.c_vreman, geometry="recompute")
    t = _timed(lambda: mesh.assemble(up, prc, out=rhs), dev, stream, args)
    forms["fwd_fp64_uncached"] = pipe_line(t, flops["fwd"] + FLOPS_GEOMETRY,
                                           {"vs_cached": fwd_med / t})
    t = _timed(lambda: mesh.assemble_vjp(up, cot, prc, out=grad), dev, stream, args)
    forms["vjp_fp64_uncached"] = pipe_line(t, flops["vjp"] + FLOPS_GEOMETRY,
                                           {"vs_cached": vjp_med / t})
    info = mesh.info()
    forms["geometry_cache"] = {
        "bytes_f64": 88 * w.n_elems, "bytes_f32": 44 * w.n_elems,
        "mesh_device_bytes": info["device_bytes"],
        "note": "the mesh here also holds both colourings (colour-major copies)"}
    for name, kw in (("fwd_fp64_skew", {"convection": "skew"}),
                     ("fwd_fp64_tau_element", {"tau": "element"})):
        pv = ns.Params(rho=w.rho, mu=w.mu, c_vreman=w.c_vreman, **kw)
        for _ in range(2):
            mesh.assemble(up, pv, out=rhs)
        va, vb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        va.record(stream)
        for _ in range(max(2, args.steps // 2)):
            mesh.assemble(up, pv, out=rhs)
        vb.record(stream)
        torch.cuda.synchronize(dev)
        vms = va.elapsed_time(vb) / max(2, args.steps // 2)
        forms[name] = {"ms": vms, "tets_per_s": w.n_elems / (vms * 1e-3), "variant": kw}
    # the RHS and the adjoint at the same state in one pass (one-pass call)
    out2 = (rhs, grad)
    op_ms = _timed(lambda: mesh.assemble_rhs_vjp(up, cot, p, out=out2), dev, stream, args)
    forms["rhs_vjp_one_pass"] = {
        "ms": op_ms, "tets_per_s": w.n_elems / (op_ms * 1e-3),
        "tflops": flops["rhs_vjp"] * w.n_elems / (op_ms * 1e-3) / 1e12,
        "vs_separate_calls": (fwd_med + vjp_med) / op_ms}
    # the forward and the adjoint through the differentiable call
    # (NSRHSFunction: forward, then backward with the cotangent)
    upr = up.detach().clone().requires_grad_(True)

    def fwd_bwd():
        upr.grad = None
        ns.assemble(mesh, upr, p).backward(cot)

    ag_ms = _timed(fwd_bwd, dev, stream, args)
    forms["fwd_vjp_autograd"] = {"ms": ag_ms, "tets_per_s": w.n_elems / (ag_ms * 1e-3),
                                 "vs_direct_calls": (fwd_med + vjp_med) / ag_ms}
    del upr
    # mixed-precision adjoint (float sweep, double accumulation)
    up32, cot32 = up.float(), cot.float()
    pmx = ns.Params(rho=w.rho, mu=w.mu, c_vreman=w.c_vreman, precision="mixed")
    for _ in range(2):
        mesh.assemble_vjp(up32, cot32, pmx, out=grad)
    ma, mb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ma.record(stream)
    for _ in range(args.steps):
        mesh.assemble_vjp(up32, cot32, pmx, out=grad)
    mb.record(stream)
    torch.cuda.synchronize(dev)
    mvjp = ma.elapsed_time(mb) / args.steps
    forms["vjp_mixed"] = {"ms": mvjp, "tets_per_s": w.n_elems / (mvjp * 1e-3),
                          "speedup_vs_fp64_vjp": vjp_med / mvjp,
                          "err_vs_oracle_32cube": mixed_vjp_error_32()}
    # the mixed one-pass call (block scatter) against the two mixed calls
    mop = _timed(lambda: mesh.assemble_rhs_vjp(up32, cot32, pmx, out=out2), dev, stream, args)
    mfwd = _timed(lambda: mesh.assemble(up32, pmx, out=rhs), dev, stream, args)
    forms["rhs_vjp_one_pass_mixed"] = {
        "ms": mop, "tets_per_s": w.n_elems / (mop * 1e-3), "kernel": "rhs_vjp_block_kernel<float,0>",
        "separate_ms": {"fwd_mixed": mfwd, "vjp_mixed": mvjp},
        "vs_separate_calls": (mfwd + mvjp) / mop,
        "tflops_fp32": flops["rhs_vjp"] * w.n_elems / (mop * 1e-3) / 1e12,
        "frac_fp32_probe": flops["rhs_vjp"] * w.n_elems / (mop * 1e-3) / 1e12 / fp32_probe}
    del up32, cot32
    # element-matrix comparison path (the pre-restructuring form, Sec. V-A)
    mesh.assemble_elmat(up, p, out=rhs)
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_em = max(2, args.steps // 4)
    ea.record(stream)
    for _ in range(n_em):
        mesh.assemble_elmat(up, p, out=rhs)
    eb.record(stream)
    torch.cuda.synchronize(dev)
    em_ms = ea.elapsed_time(eb) / n_em
    forms["fwd_fp64_element_matrix"] = {"ms": em_ms, "tets_per_s": w.n_elems / (em_ms * 1e-3),
                                        "direct_speedup": em_ms / fwd_med}
    # explicit SSP-RK3 momentum step (3 assemblies + stage updates), in place
    # on a copy of the fields; dt is a CFL-like 0.1 h / max|u|
    u_step = up.clone()
    work = torch.empty((8, w.n_nodes), dtype=torch.float64, device=dev)
    dt = 0.1 / args.n / float(np.abs(w.up[:3]).max())
    mesh.explicit_step(u_step, dt, "ssprk3", p, work=work)
    sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_rk = max(2, args.steps // 4)
    sa.record(stream)
    for _ in range(n_rk):
        mesh.explicit_step(u_step, dt, "ssprk3", p, work=work)
    sb.record(stream)
    torch.cuda.synchronize(dev)
    rk_ms = sa.elapsed_time(sb) / n_rk
    forms["explicit_step_ssprk3"] = {"ms": rk_ms, "assemblies_per_step": 3,
                                     "overhead_vs_3_assemblies": rk_ms / (3 * fwd_med)}
    forms["explicit_step_small_graph"] = time_step_graph(16, dev, stream)
    del u_step, work
    forms["scatter_sweep"] = time_scatter_sweep(mesh, w, up, cot, dev, stream, args, fwd_med,
                                                vjp_med)
    forms["scatter_sweep"]["mesh_setup_s_with_colouring"] = t_mesh
    if not args.no_mixed:
        forms["mixed_same_mesh"] = time_mixed(mesh, w, dev, stream, args, fwd_med)
        mesh.close()
        del mesh
        torch.cuda.empty_cache()
        wj = mg.precision_case(n=args.n, order="rcm")
        cj = torch.from_numpy(wj.coords).to(dev)
        nj = torch.from_numpy(wj.conn).to(dev)
        mj = ns.Mesh(cj, nj)
        del cj, nj
        upj = torch.from_numpy(wj.up).to(dev)
        pj = ns.Params(rho=wj.rho, mu=wj.mu)
        for _ in range(args.warmup):
            mj.assemble(upj, pj)
        fa, fb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fa.record(stream)
        for _ in range(args.steps):
            mj.assemble(upj, pj)
        fb.record(stream)
        torch.cuda.synchronize(dev)
        fp64_j = fa.elapsed_time(fb) / args.steps
        mixed = time_mixed(mj, wj, dev, stream, args, fp64_j)
        mixed["n_high_ar"] = mj.info()["n_high_ar"]
        mixed["err_vs_oracle_64cube"] = mixed_error_64()
        forms["mixed_jitter03"] = mixed
        mj.close()

    if args.unstructured > 0:
        forms["unstructured"] = time_unstructured(args.unstructured, dev, stream, args)
    if args.locality > 0:
        forms["locality"] = time_locality(args.locality, dev, stream, args)
    forms["vjp_64cube"] = time_vjp_64(dev, stream, args)
    if args.locality > 0:
        try:
            forms["partitioned_one_gpu"] = time_partitioned(args.locality, 8, dev, stream, args)
        except Exception as exc:  # an auxiliary form must not cost the bench line
            forms["partitioned_one_gpu"] = {"error": repr(exc)}

    dom = "vjp_fp64" if vjp_med >= fwd_med else "fwd_fp64"
    dom_ms = vjp_med if dom == "vjp_fp64" else fwd_med
    achieved = forms[dom]["tflops"]
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                "traffic": (DRAM_BYTES_PER_TET[dom] * w.n_elems
                            if DRAM_BYTES_PER_TET.get(dom) is not None else None),
                "peak_source": (f"FP64 pipe rate: {FP64_LANES_PER_SM} FMA lanes/SM/clock x 2 flops "
                                f"x {n_sm} SMs x {clk_mhz:.0f} MHz sampled during the timed "
                                f"region (FP64 is not in MEASURED_PEAKS.json); the FMA-chain "
                                f"probe measured {fp64_probe:.3f} TF/s in this run"),
                "flops_per_tet": flops["vjp" if dom == "vjp_fp64" else "fwd"],
                "launch_ms": dom_ms}
    # the same launch counted with the method's own operations (the oracle's
    # definition): what the restructured algebra does in fewer operations
    mflops = FLOPS_PER_TET_METHOD_VREMAN if w.c_vreman else FLOPS_PER_TET_METHOD
    mper = mflops["vjp" if dom == "vjp_fp64" else "fwd"]
    roofline["flops_per_tet_method"] = mper
    roofline["achieved_method"] = mper * w.n_elems / (dom_ms * 1e-3) / 1e12
    roofline["frac_method"] = roofline["achieved_method"] / fp64_peak
    # the mixed-precision kernels against both of their roofs: FP32 FMA (the
    # live probe) and HBM (algorithmic bytes against the measured copy peak)
    roofline_mixed = {}
    mixed_ms = {"fwd_mixed": forms.get("mixed_same_mesh", {}).get("ms"),
                "vjp_mixed": forms["vjp_mixed"]["ms"]}
    for key, ms in mixed_ms.items():
        if ms is not None:
            roofline_mixed[key] = mixed_roofline(key, ms, w.n_elems, fp32_probe, _measured_hbm())
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(w, world),
            "roofline": roofline,
            "roofline_fwd": {"bound": "alu", "achieved": forms["fwd_fp64"]["tflops"],
                             "peak": fp64_peak, "unit": "TFLOP/s",
                             "frac": forms["fwd_fp64"]["tflops"] / fp64_peak,
                             "flops_per_tet": flops["fwd"],
                             "flops_per_tet_method": mflops["fwd"],
                             "achieved_method": mflops["fwd"] * w.n_elems / (fwd_med * 1e-3) / 1e12},
            "roofline_mixed": roofline_mixed,
            "peaks": {"fp64_tflops": fp64_peak, "fp64_probe_tflops": fp64_probe,
                      "fp32_probe_tflops": fp32_probe,
                      "hbm_gbs_measured_peaks_json": _measured_hbm()},
            "forms": forms,
            "e2e": {"value": whole_job_rate(w.n_elems, world, e2e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": 2 * bytes_nodal, "d2h_bytes_per_step": 2 * bytes_nodal,
                    "ms_per_step": e2e_ms, "wall_ms_per_step": 1e3 * t_e2e / args.steps,
                    "overlap": "copies of a step overlap the compute of its neighbours"},
            "gpu_launches": 2 * args.steps,
            "clocks": clocks,
            "wall_s_timed": t_wall}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


MIXED_KERNELS = {"fwd_mixed": "fwd_block_kernel<float,0>", "vjp_mixed": "vjp_block_kernel<float,0>"}
# What ncu shows stopping them (128^3 captures of the current kernels).
MIXED_LIMITER = {
    "fwd_mixed": "issue latency between barrier phases at 4 CTAs/SM (64 registers): "
                 "issue 67 %, L1/TEX 78 % (half of the shared wavefronts bank conflicts), "
                 "FMA 44 %, DRAM 40 %; top stalls barrier, long scoreboard",
    "vjp_mixed": "latency at 3 CTAs/SM (80 registers): issue 59 %, warps active 34 %, "
                 "L1/TEX 71 %, FMA 43 %, DRAM 28 %; top stalls long scoreboard, barrier"}


def mixed_roofline(key, ms, n_elems, fp32_peak, hbm_peak):
    """One mixed-precision kernel on its two roofs. FP32: algorithmic flops
    (the census) per launch / launch time against the FP32 FMA-chain probe.
    HBM: algorithmic bytes per launch / launch time against the measured copy
    bandwidth; the ncu-measured DRAM bytes are `traffic`. `bound` names the
    roof the kernel is closer to."""
    sec = ms * 1e-3
    kind = key.split("_")[0]
    tf = FLOPS_PER_TET[kind] * n_elems / sec / 1e12
    alg = ALG_BYTES_PER_TET[key] * n_elems / sec / 1e9
    meas = DRAM_BYTES_PER_TET.get(key)
    d = {"kernel": MIXED_KERNELS[key], "launch_ms": ms,
         "fp32": {"achieved": tf, "peak": fp32_peak, "unit": "TFLOP/s", "frac": tf / fp32_peak,
                  "peak_source": "FP32 FMA-chain probe, measured in this run"},
         "hbm": {"achieved": alg, "peak": hbm_peak, "unit": "GB/s",
                 "frac": alg / hbm_peak if hbm_peak else None,
                 "bytes_per_tet_algorithmic": ALG_BYTES_PER_TET[key],
                 "measured_dram_gbs": meas * n_elems / sec / 1e9 if meas else None,
                 "peak_source": "hbm_gbs of the driver's measured peaks (copy bandwidth)"},
         "traffic": meas * n_elems if meas else None,
         "limiter_ncu": MIXED_LIMITER[key]}
    fh = d["hbm"]["frac"] or 0.0
    d["bound"] = "hbm" if fh >= d["fp32"]["frac"] else "alu"
    d["frac"] = max(fh, d["fp32"]["frac"])
    return d


def time_mixed(mesh, w, dev, stream, args, fp64_ms):
    import torch
    import paper_2403_08777_gb300 as ns
    up32 = torch.from_numpy(w.up).to(dev).float()
    pm = ns.Params(rho=w.rho, mu=w.mu, c_vreman=w.c_vreman, precision="mixed")
    out = torch.empty((4, w.n_nodes), dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        mesh.assemble(up32, pm, out=out)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        mesh.assemble(up32, pm, out=out)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / args.steps
    return {"ms": ms, "tets_per_s": w.n_elems / (ms * 1e-3), "fp64_ms": fp64_ms,
            "speedup_vs_fp64": fp64_ms / ms, "workload": w.name}


def _timed(fn, dev, stream, args):
    import torch
    for _ in range(args.warmup):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize(dev)
    return a.elapsed_time(b) / args.steps


def time_step_graph(n, dev, stream, steps=50):
    """SSP-RK3 steps on a small n^3-hex mesh, launched one call at a time and
    replayed from one CUDA graph holding the same steps: microseconds per
    step."""
    import torch
    import paper_2403_08777_gb300 as ns
    w = mg.make_workload(n, order="rcm", mu=1e-3, mag_max=2.0)
    m = ns.Mesh(torch.from_numpy(w.coords).to(dev), torch.from_numpy(w.conn).to(dev))
    up = torch.from_numpy(w.up).to(dev)
    p = ns.Params(rho=w.rho, mu=w.mu)
    dt = 0.1 / n / float(np.abs(w.up[:3]).max())
    work = torch.empty((8, w.n_nodes), dtype=torch.float64, device=dev)
    u1 = up.clone()
    for _ in range(3):
        m.explicit_step(u1, dt, "ssprk3", p, work=work)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        m.explicit_step(u1, dt, "ssprk3", p, work=work)
    b.record(stream)
    torch.cuda.synchronize(dev)
    direct = a.elapsed_time(b) * 1e3 / steps
    u2 = up.clone()
    g = ns.StepGraph(m, u2, dt, "ssprk3", p, steps=steps)
    g.replay()
    torch.cuda.synchronize(dev)
    a.record(stream)
    g.replay()
    b.record(stream)
    torch.cuda.synchronize(dev)
    graphed = a.elapsed_time(b) * 1e3 / steps
    m.close()
    return {"workload": w.name, "n_tets": w.n_elems, "us_per_step_direct": direct,
            "us_per_step_graph": graphed, "speedup": direct / graphed}


def time_scatter_sweep(mesh, w, up, cot, dev, stream, args, fwd_ms, vjp_ms):
    """Every scatter on the same mesh: the FP64 and mixed forward with
    atomics, element blocks and element colouring (deterministic), the FP64
    and mixed adjoint with atomics and colouring. Rates in tets/s."""
    import torch
    import paper_2403_08777_gb300 as ns

    def mk(**kw):
        return ns.Params(rho=w.rho, mu=w.mu, c_vreman=w.c_vreman, **kw)

    def rate(ms):
        return w.n_elems / (ms * 1e-3)

    o = torch.empty_like(up)
    up32, cot32 = up.float(), cot.float()
    res = {"n_colours": mesh.info()["n_colours"],
           "fwd_fp64": {"atomic": rate(fwd_ms)}, "fwd_mixed": {},
           "vjp_fp64": {"atomic": rate(vjp_ms)}, "vjp_mixed": {}}
    res["n_block_colours"] = mesh.info()["n_block_colours"]
    for sc in ("block", "colour", "block_colour"):
        res["fwd_fp64"][sc] = rate(_timed(lambda: mesh.assemble(up, mk(scatter=sc), out=o),
                                          dev, stream, args))
    for sc in ("atomic", "block", "colour", "block_colour"):
        res["fwd_mixed"][sc] = rate(_timed(
            lambda: mesh.assemble(up32, mk(scatter=sc, precision="mixed"), out=o),
            dev, stream, args))
    for sc in ("block", "colour", "block_colour"):
        res["vjp_fp64"][sc] = rate(_timed(
            lambda: mesh.assemble_vjp(up, cot, mk(scatter=sc), out=o), dev, stream, args))
    for sc in ("atomic", "block", "colour", "block_colour"):
        res["vjp_mixed"][sc] = rate(_timed(
            lambda: mesh.assemble_vjp(up32, cot32, mk(scatter=sc, precision="mixed"), out=o),
            dev, stream, args))
    # the coloured paths are deterministic: two calls, bitwise equal
    same = True
    for sc in ("colour", "block_colour"):
        for u in (up, up32):
            pr = mk(scatter=sc, precision="fp64" if u is up else "mixed")
            a = mesh.assemble(u, pr).clone()
            same = same and bool(torch.equal(a, mesh.assemble(u, pr)))
    res["colour_bitwise_reproducible"] = same
    return res


def time_locality(n, dev, stream, args):
    """n^3 hexes (rho 1, mu 1e-2, Taylor-Green + noise) with a random and an
    RCM node order: FP64 and mixed forward rates (gather/scatter locality)."""
    import torch
    import paper_2403_08777_gb300 as ns
    out = {}
    for order in ("random", "rcm"):
        w = mg.medium(order=order, n=n)
        m = ns.Mesh(torch.from_numpy(w.coords).to(dev), torch.from_numpy(w.conn).to(dev))
        up = torch.from_numpy(w.up).to(dev)
        up32 = up.float()
        o = torch.empty_like(up)
        p = ns.Params(rho=w.rho, mu=w.mu)
        pm = ns.Params(rho=w.rho, mu=w.mu, precision="mixed")
        f = _timed(lambda: m.assemble(up, p, out=o), dev, stream, args)
        x = _timed(lambda: m.assemble(up32, pm, out=o), dev, stream, args)
        xa = _timed(lambda: m.assemble(up32, ns.Params(rho=w.rho, mu=w.mu, precision="mixed",
                                                       scatter="atomic"), out=o),
                    dev, stream, args)
        out[order] = {"fwd_fp64_tets_per_s": w.n_elems / (f * 1e-3),
                      "mixed_block_tets_per_s": w.n_elems / (x * 1e-3),
                      "mixed_atomic_tets_per_s": w.n_elems / (xa * 1e-3),
                      "bandwidth": mg.bandwidth(w.conn)}
        m.close()
    out["workload"] = f"kuhn{n}^3 (random vs rcm)"
    return out


def time_partitioned(n, n_parts, dev, stream, args):
    """The n^3-hex mesh (paper-scale fields) cut into n_parts z-slabs
    (partition.slab_partition), each part its own library mesh on this GPU:
    the whole mesh's forward against each part's (what one rank of a sharded
    run assembles), the ghost-node overhead, the bytes one rank moves in
    either interface exchange, and the exchanged parts against the whole
    mesh's RHS."""
    import torch
    import paper_2403_08777_gb300 as ns
    from paper_2403_08777_gb300 import partition as pt
    w = mg.paper_scale(n=n, order="rcm")
    p = ns.Params(rho=w.rho, mu=w.mu)
    whole = ns.Mesh(torch.from_numpy(w.coords).to(dev), torch.from_numpy(w.conn).to(dev))
    up = torch.from_numpy(w.up).to(dev)
    o = torch.empty_like(up)
    t_whole = _timed(lambda: whole.assemble(up, p, out=o), dev, stream, args)
    ref = o.clone()
    whole.close()
    parts = pt.slab_partition(w.coords, w.conn, n_parts)
    t_parts, outs = [], []
    for part in parts:
        m = ns.Mesh(torch.from_numpy(part.local(w.coords)).to(dev),
                    torch.from_numpy(part.conn).to(dev))
        u = torch.from_numpy(part.local(w.up)).to(dev)
        op = torch.empty_like(u)
        t_parts.append(_timed(lambda: m.assemble(u, p, out=op), dev, stream, args))
        outs.append(op)
        m.close()
    total = sum(pt.interface_rows(l, q) for l, q in zip(outs, parts))
    err = 0.0
    scale = float(ref.abs().max())
    for l, q in zip(outs, parts):
        pt.apply_interface(l, q, total)
        idx = torch.as_tensor(q.nodes, device=dev)
        err = max(err, float((l - ref[:, idx]).abs().max()) / scale)
    return {"workload": w.name, "n_parts": n_parts, "partition": "z slabs, equal element counts",
            "whole_fwd_ms": t_whole, "part_fwd_ms_max": max(t_parts),
            "part_fwd_ms_sum": sum(t_parts), "per_rank_speedup": t_whole / max(t_parts),
            "ghost_node_overhead": sum(q.n_nodes for q in parts) / w.n_nodes - 1,
            "exchange_bytes_per_rank_allreduce": 4 * 8 * parts[0].n_iface,
            "exchange_bytes_per_rank_p2p_max": max(4 * 8 * sum(len(i) for i in q.shared.values())
                                                   for q in parts),
            "max_rel_diff_vs_whole_mesh": err}


def time_vjp_64(dev, stream, args):
    """Adjoint throughput on the 64^3-hex mesh (1,572,864 tets)."""
    import torch
    import paper_2403_08777_gb300 as ns
    w = mg.paper_scale(n=64, order="rcm")
    m = ns.Mesh(torch.from_numpy(w.coords).to(dev), torch.from_numpy(w.conn).to(dev))
    up = torch.from_numpy(w.up).to(dev)
    cot = torch.from_numpy(mg.normal((4, w.n_nodes), seed=mg.SEED_COT)).to(dev)
    o = torch.empty_like(up)
    p = ns.Params(rho=w.rho, mu=w.mu)
    v = _timed(lambda: m.assemble_vjp(up, cot, p, out=o), dev, stream, args)
    m.close()
    return {"workload": w.name, "n_tets": w.n_elems, "tets_per_s": w.n_elems / (v * 1e-3)}


def time_unstructured(n, dev, stream, args):
    """FP64 forward and adjoint and the mixed forward on the Delaunay mesh of
    an (n+1)^3 jittered lattice (RCM order): irregular valence, no hex blocks."""
    import torch
    import paper_2403_08777_gb300 as ns
    w = mg.make_unstructured(n, order="rcm", mu=1e-4, mag_max=10.0)
    m = ns.Mesh(torch.from_numpy(w.coords).to(dev), torch.from_numpy(w.conn).to(dev))
    up = torch.from_numpy(w.up).to(dev)
    cot = torch.from_numpy(mg.normal((4, w.n_nodes), seed=mg.SEED_COT)).to(dev)
    p = ns.Params(rho=w.rho, mu=w.mu)
    pm = ns.Params(rho=w.rho, mu=w.mu, precision="mixed")
    up32 = up.float()
    out = torch.empty_like(up)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / args.steps

    fwd = timed(lambda: m.assemble(up, p, out=out))
    vjp = timed(lambda: m.assemble_vjp(up, cot, p, out=out))
    mix = timed(lambda: m.assemble(up32, pm, out=out))
    info = m.info()
    m.close()
    return {"workload": w.name, "n_tets": w.n_elems, "n_nodes": w.n_nodes,
            "fwd_fp64_tets_per_s": w.n_elems / (fwd * 1e-3),
            "vjp_fp64_tets_per_s": w.n_elems / (vjp * 1e-3),
            "mixed_tets_per_s": w.n_elems / (mix * 1e-3), "n_high_ar": info["n_high_ar"],
            "max_ar": info["max_ar"]}


def mixed_vjp_error_32() -> float:
    """Norm-wise error of the mixed adjoint against the oracle (complex-step
    element Jacobians) on the 32^3 paper-scale-settings mesh."""
    import torch
    import oracle
    import paper_2403_08777_gb300 as ns
    w = mg.paper_scale(n=32, order="rcm")
    dev = torch.device("cuda", torch.cuda.current_device())
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    m = ns.Mesh(torch.from_numpy(w.coords).to(dev), torch.from_numpy(w.conn).to(dev))
    g = m.assemble_vjp(torch.from_numpy(w.up).to(dev).float(), torch.from_numpy(cot).to(dev).float(),
                       ns.Params(rho=w.rho, mu=w.mu, precision="mixed")).cpu().numpy()
    m.close()
    ref = oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu)
    return float(np.linalg.norm(g - ref) / np.linalg.norm(ref))


def mixed_error_64() -> float:
    """Norm-wise error of the mixed form against the oracle on the 64^3
    jitter-0.3 sub-run (1,572,864 tets)."""
    import torch
    import oracle
    import paper_2403_08777_gb300 as ns
    w = mg.precision_case(n=64, order="rcm")
    dev = torch.device("cuda", torch.cuda.current_device())
    m = ns.Mesh(torch.from_numpy(w.coords).to(dev), torch.from_numpy(w.conn).to(dev))
    x = m.assemble(torch.from_numpy(w.up).to(dev).float(),
                   ns.Params(rho=w.rho, mu=w.mu, precision="mixed")).cpu().numpy()
    m.close()
    ref = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu)
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def sm_blocks(dev) -> int:
    import torch
    return torch.cuda.get_device_properties(dev).multi_processor_count * 8


def _ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


def _stream(s):
    import ctypes
    return ctypes.c_void_p(s.cuda_stream)


def _measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        return None


def run_profile(args):
    """A short launch sequence for a profiler: the forward, the adjoint and
    the one-pass call of one form, --warmup then --steps times each, on the
    --n mesh."""
    import torch
    import paper_2403_08777_gb300 as ns
    w = workload(args.n)
    dev = torch.device("cuda", 0)
    mesh = ns.Mesh(torch.from_numpy(w.coords).to(dev), torch.from_numpy(w.conn).to(dev))
    up = torch.from_numpy(w.up).to(dev)
    cot = torch.from_numpy(mg.normal((4, w.n_nodes), seed=mg.SEED_COT)).to(dev)
    if args.profile == "mixed":
        up, cot = up.float(), cot.float()
    p = ns.Params(rho=w.rho, mu=w.mu, precision=args.profile)
    out = torch.empty((4, w.n_nodes), dtype=torch.float64, device=dev)
    for _ in range(args.warmup + args.steps):
        mesh.assemble(up, p, out=out)
    for _ in range(args.warmup + args.steps):
        mesh.assemble_vjp(up, cot, p, out=out)
    out2 = (out, torch.empty_like(out))
    for _ in range(args.warmup + args.steps):
        mesh.assemble_rhs_vjp(up, cot, p, out=out2)
    torch.cuda.synchronize(dev)
    mesh.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""GB300-native Navier-Stokes RHS assembly on linear tetrahedra (arXiv 2403.08777).

Thin Python binding over the C ABI of ``include/nsrhs.h``: argument
marshalling only. Every step of the assembly runs in the CUDA kernels of
``libnsrhs.so``; PyTorch provides device memory and the current stream.
There is no CPU fallback: if the library has not been built, the calls raise.

    mesh = Mesh(coords_cuda_f64[3, N], conn_cuda_i32[4, E])
    rhs  = mesh.assemble(up_cuda_f64[4, N], rho=1.0, mu=1e-2)        # [4, N] f64
    grad = mesh.assemble_vjp(up, cot)                                 # [4, N] f64
    rhs  = assemble(mesh, up, rho=1.0, mu=1e-2)                      # differentiable in up
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _abi
from ._abi import NSRHSError, NativeLibraryMissing  # noqa: F401

__all__ = ["Mesh", "Params", "assemble", "assemble_host", "StepPipeline", "StepGraph", "NSRHSFunction",
           "NSRHSError", "NativeLibraryMissing", "load_library"]

_PREC = {"fp64": _abi.FP64, "mixed": _abi.MIXED}
_SCAT = {"auto": _abi.SCATTER_AUTO, "atomic": _abi.SCATTER_ATOMIC, "block": _abi.SCATTER_BLOCK,
         "colour": _abi.SCATTER_COLOUR, "block_colour": _abi.SCATTER_BLOCK_COLOUR}
_CONV = {"convective": _abi.CONVECTIVE, "skew": _abi.SKEW}
_TAU = {"gauss": _abi.TAU_GAUSS, "element": _abi.TAU_ELEMENT}
_GEOM = {"cached": _abi.GEOM_CACHED, "recompute": _abi.GEOM_RECOMPUTE}


def load_library():
    return _abi.load()


@dataclass(frozen=True)
class Params:
    rho: float = 1.0
    mu: float = 1e-2
    c_vreman: float = 0.0
    c1: float = 4.0
    c2: float = 2.0
    precision: str = "fp64"
    scatter: str = "auto"
    convection: str = "convective"   # or "skew" (energy-preserving)
    tau: str = "gauss"               # or "element"
    geometry: str = "cached"         # or "recompute" (formed from coordinates in every call)

    def to_c(self) -> _abi.Params:
        if (self.precision not in _PREC or self.scatter not in _SCAT or
                self.convection not in _CONV or self.tau not in _TAU or
                self.geometry not in _GEOM):
            raise ValueError(f"bad option in {self}")
        return _abi.Params(self.rho, self.mu, self.c_vreman, self.c1, self.c2,
                           _PREC[self.precision], _SCAT[self.scatter], _CONV[self.convection],
                           _TAU[self.tau], _GEOM[self.geometry], 0)


def _stream_handle(device: torch.device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _require(t: torch.Tensor, name: str, dtype, shape, device=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, mesh is on {device}")


class Mesh:
    """A tetrahedral mesh resident on one GPU (library-owned device copies)."""

    def __init__(self, coords: torch.Tensor, conn: torch.Tensor, ar_threshold: float = 10.0,
                 colour: bool = False):
        """colour=True also colours the elements for scatter='colour'
        (deterministic, bitwise reproducible assembly)."""
        lib = _abi.load()
        if coords.dim() != 2 or coords.shape[0] != 3 or conn.dim() != 2 or conn.shape[0] != 4:
            raise ValueError("coords must be [3, N] and conn [4, E]")
        _require(coords, "coords", torch.float64, coords.shape)
        _require(conn, "conn", torch.int32, conn.shape, coords.device)
        self.device = coords.device
        self.n_nodes, self.n_elems = int(coords.shape[1]), int(conn.shape[1])
        opts = _abi.MeshOpts(float(ar_threshold), 1 if colour else 0, 0)
        handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = lib.nsrhs_mesh_create(self.n_nodes, self.n_elems, ctypes.c_void_p(coords.data_ptr()),
                                       ctypes.c_void_p(conn.data_ptr()), ctypes.byref(opts),
                                       _stream_handle(self.device), ctypes.byref(handle))
        _abi.check(st, "nsrhs_mesh_create")
        self._h = handle

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("mesh has been closed")
        return self._h

    def info(self) -> dict:
        inf = _abi.MeshInfo()
        _abi.check(_abi.load().nsrhs_mesh_get_info(self.handle, ctypes.byref(inf)),
                   "nsrhs_mesh_get_info")
        return {f: getattr(inf, f) for f, _ in _abi.MeshInfo._fields_}

    def element_colours(self, which: str = "element") -> torch.Tensor:
        """Per element in the caller's element order, [E] int32 (a mesh created
        with colour=True): which='element' its colour (COLOUR scatter),
        'block_colour' its block's colour (BLOCK_COLOUR scatter), 'block' its
        block index."""
        kinds = {"element": _abi.ELEMENT_COLOUR, "block_colour": _abi.ELEMENT_BLOCK_COLOUR,
                 "block": _abi.ELEMENT_BLOCK}
        if which not in kinds:
            raise ValueError(f"which must be one of {sorted(kinds)}")
        out = torch.empty(self.n_elems, dtype=torch.int32, device=self.device)
        with torch.cuda.device(self.device):
            st = _abi.load().nsrhs_mesh_element_colours(self.handle, kinds[which],
                                                         ctypes.c_void_p(out.data_ptr()),
                                                         _stream_handle(self.device))
        _abi.check(st, "nsrhs_mesh_element_colours")
        return out

    def _params(self, params: Params | None, kw) -> Params:
        if params is None:
            params = Params(**kw)
        elif kw:
            raise TypeError("pass either params or keyword parameters")
        return params

    def assemble(self, up: torch.Tensor, params: Params | None = None, *, out=None, **kw):
        """RHS [4, N] float64 of nodal fields up [4, N] (float64, or float32
        with precision='mixed'), on the current stream."""
        p = self._params(params, kw)
        dt = torch.float32 if p.precision == "mixed" else torch.float64
        _require(up, "up", dt, (4, self.n_nodes), self.device)
        if out is None:
            out = torch.empty((4, self.n_nodes), dtype=torch.float64, device=self.device)
        else:
            _require(out, "out", torch.float64, (4, self.n_nodes), self.device)
        cp = p.to_c()
        with torch.cuda.device(self.device):
            st = _abi.load().nsrhs_assemble(self.handle, ctypes.byref(cp),
                                            ctypes.c_void_p(up.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()),
                                            _stream_handle(self.device))
        _abi.check(st, "nsrhs_assemble")
        return out

    def assemble_vjp(self, up: torch.Tensor, cot: torch.Tensor, params: Params | None = None, *,
                     out=None, **kw):
        """(d rhs / d up)^T cot, [4, N] float64; up and cot float64 (fp64) or
        float32 (precision='mixed')."""
        p = self._params(params, kw)
        dt = torch.float32 if p.precision == "mixed" else torch.float64
        _require(up, "up", dt, (4, self.n_nodes), self.device)
        _require(cot, "cot", dt, (4, self.n_nodes), self.device)
        if out is None:
            out = torch.empty((4, self.n_nodes), dtype=torch.float64, device=self.device)
        else:
            _require(out, "out", torch.float64, (4, self.n_nodes), self.device)
        cp = p.to_c()
        with torch.cuda.device(self.device):
            st = _abi.load().nsrhs_assemble_vjp(self.handle, ctypes.byref(cp),
                                                ctypes.c_void_p(up.data_ptr()),
                                                ctypes.c_void_p(cot.data_ptr()),
                                                ctypes.c_void_p(out.data_ptr()),
                                                _stream_handle(self.device))
        _abi.check(st, "nsrhs_assemble_vjp")
        return out

    def assemble_rhs_vjp(self, up: torch.Tensor, cot: torch.Tensor,
                         params: Params | None = None, *, out=None, **kw):
        """(rhs, (d rhs / d up)^T cot) at the same state in one pass; both
        [4, N] float64. out: optional pair of [4, N] float64 tensors."""
        p = self._params(params, kw)
        dt = torch.float32 if p.precision == "mixed" else torch.float64
        _require(up, "up", dt, (4, self.n_nodes), self.device)
        _require(cot, "cot", dt, (4, self.n_nodes), self.device)
        if out is None:
            out = tuple(torch.empty((4, self.n_nodes), dtype=torch.float64, device=self.device)
                        for _ in range(2))
        else:
            for t, name in zip(out, ("out[0]", "out[1]")):
                _require(t, name, torch.float64, (4, self.n_nodes), self.device)
        rhs, grad = out
        cp = p.to_c()
        with torch.cuda.device(self.device):
            st = _abi.load().nsrhs_assemble_rhs_vjp(self.handle, ctypes.byref(cp),
                                                    ctypes.c_void_p(up.data_ptr()),
                                                    ctypes.c_void_p(cot.data_ptr()),
                                                    ctypes.c_void_p(rhs.data_ptr()),
                                                    ctypes.c_void_p(grad.data_ptr()),
                                                    _stream_handle(self.device))
        _abi.check(st, "nsrhs_assemble_rhs_vjp")
        return rhs, grad

    def assemble_elmat(self, up: torch.Tensor, params: Params | None = None, *, out=None, **kw):
        """The FP64 RHS through full 16x16 element matrices (comparison path)."""
        p = self._params(params, kw)
        _require(up, "up", torch.float64, (4, self.n_nodes), self.device)
        if out is None:
            out = torch.empty((4, self.n_nodes), dtype=torch.float64, device=self.device)
        cp = p.to_c()
        with torch.cuda.device(self.device):
            st = _abi.load().nsrhs_assemble_elmat(self.handle, ctypes.byref(cp),
                                                  ctypes.c_void_p(up.data_ptr()),
                                                  ctypes.c_void_p(out.data_ptr()),
                                                  _stream_handle(self.device))
        _abi.check(st, "nsrhs_assemble_elmat")
        return out

    def lumped_mass(self) -> torch.Tensor:
        """Row-sum lumped P1 mass of every node, [N] float64."""
        out = torch.empty(self.n_nodes, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            st = _abi.load().nsrhs_lumped_mass(self.handle, ctypes.c_void_p(out.data_ptr()),
                                               _stream_handle(self.device))
        _abi.check(st, "nsrhs_lumped_mass")
        return out

    def explicit_step(self, up: torch.Tensor, dt: float, scheme: str = "ssprk3",
                      params: Params | None = None, *, work: torch.Tensor | None = None, **kw):
        """Advance the velocity rows of up [4, N] (float64, in place) by one
        explicit step of rho m du/dt = F (pressure row kept); returns up.
        precision='mixed' assembles the stage RHS in the mixed form (the
        state stays float64); work is [8, N] (fp64) or [10, N] (mixed)."""
        p = self._params(params, kw)
        _require(up, "up", torch.float64, (4, self.n_nodes), self.device)
        rows = 10 if p.precision == "mixed" else 8
        if work is None:
            work = torch.empty((rows, self.n_nodes), dtype=torch.float64, device=self.device)
        _require(work, "work", torch.float64, (rows, self.n_nodes), self.device)
        sch = {"euler": _abi.EULER, "ssprk3": _abi.SSPRK3}[scheme]
        cp = p.to_c()
        with torch.cuda.device(self.device):
            st = _abi.load().nsrhs_explicit_step(self.handle, ctypes.byref(cp), float(dt), sch,
                                                 ctypes.c_void_p(up.data_ptr()),
                                                 ctypes.c_void_p(work.data_ptr()),
                                                 _stream_handle(self.device))
        _abi.check(st, "nsrhs_explicit_step")
        return up

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            _abi.load().nsrhs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NSRHSFunction(torch.autograd.Function):
    """rhs = A(up) with the hand-written adjoint kernel as backward.
    Differentiable with respect to up only (mesh and parameters are constants);
    fp64 (up float64) or mixed (up float32; rhs float64, gradient float32)."""

    @staticmethod
    def forward(ctx, up: torch.Tensor, mesh: Mesh, params: Params):
        ctx.mesh, ctx.params = mesh, params
        ctx.save_for_backward(up)
        return mesh.assemble(up.detach().contiguous(), params)

    @staticmethod
    def backward(ctx, grad_rhs: torch.Tensor):
        (up,) = ctx.saved_tensors
        cot = grad_rhs.contiguous()
        if ctx.params.precision == "mixed":
            # float cotangent into the float reverse sweep; the gradient is
            # accumulated in double and returned in up's dtype (float32)
            cot = cot.float()
        g = ctx.mesh.assemble_vjp(up.detach().contiguous(), cot, ctx.params)
        return g.to(up.dtype), None, None


def assemble(mesh: Mesh, up: torch.Tensor, params: Params | None = None, **kw) -> torch.Tensor:
    """Differentiable RHS assembly (fp64, or mixed with float32 up)."""
    p = mesh._params(params, kw)
    return NSRHSFunction.apply(up, mesh, p)


def assemble_host(mesh: Mesh, up_host: torch.Tensor, params: Params | None = None,
                  out_host: torch.Tensor | None = None, **kw) -> torch.Tensor:
    """End-to-end call on host buffers: copy up (pinned host) to the device,
    assemble, copy the RHS back into out_host (pinned host), synchronise."""
    p = mesh._params(params, kw)
    dt = torch.float32 if p.precision == "mixed" else torch.float64
    if up_host.is_cuda or up_host.dtype != dt or tuple(up_host.shape) != (4, mesh.n_nodes):
        raise ValueError("up_host must be a host tensor [4, N] of the precision's dtype")
    up = up_host.to(mesh.device, non_blocking=True)
    rhs = mesh.assemble(up, p)
    if out_host is None:
        out_host = torch.empty((4, mesh.n_nodes), dtype=torch.float64, pin_memory=True)
    out_host.copy_(rhs, non_blocking=True)
    torch.cuda.current_stream(mesh.device).synchronize()
    return out_host


class StepGraph:
    """`steps` explicit time steps of up (in place) captured once in a CUDA
    graph and replayed with one launch: for small meshes, where the steps'
    kernel launches (each Runge-Kutta stage is a memset, an assembly and an
    update) cost more than their work. The library calls allocate nothing and
    never synchronise, so they can be captured; the graph is bound to the
    addresses of `up` and of its own work buffer.

        g = StepGraph(mesh, up, dt, "ssprk3", params, steps=10)
        g.replay()            # ten steps, on the current stream
    """

    def __init__(self, mesh: Mesh, up: torch.Tensor, dt: float, scheme: str = "ssprk3",
                 params: Params | None = None, *, steps: int = 1, **kw):
        if steps < 1:
            raise ValueError("steps must be >= 1")
        p = mesh._params(params, kw)
        _require(up, "up", torch.float64, (4, mesh.n_nodes), mesh.device)
        self.mesh, self.up, self.steps = mesh, up, steps
        rows = 10 if p.precision == "mixed" else 8
        self.work = torch.empty((rows, mesh.n_nodes), dtype=torch.float64, device=mesh.device)
        side = torch.cuda.Stream(mesh.device)
        side.wait_stream(torch.cuda.current_stream(mesh.device))
        with torch.cuda.stream(side):
            # one eager step first (first launches of a kernel may initialise
            # lazily, which capture does not allow), then restore up
            saved = up.clone()
            mesh.explicit_step(up, dt, scheme, p, work=self.work)
            up.copy_(saved)
        torch.cuda.current_stream(mesh.device).wait_stream(side)
        del saved
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.device(mesh.device), torch.cuda.graph(self.graph):
            for _ in range(steps):
                mesh.explicit_step(up, dt, scheme, p, work=self.work)

    def replay(self) -> torch.Tensor:
        self.graph.replay()
        return self.up


class StepPipeline:
    """Repeated steps on HOST buffers — copy (u, p) and the cotangent in,
    assemble, run the adjoint, copy the RHS and the gradient out — with the
    copies of one step overlapped with the compute of its neighbours (two
    device buffer sets, separate copy-in, compute and copy-out streams).

        pipe = StepPipeline(mesh, params)
        for k in range(n):
            pipe.submit(k, up_host, cot_host, rhs_host[k % 2], grad_host[k % 2])
        pipe.synchronize()

    Host tensors should be pinned for the copies to be asynchronous. A host
    output passed to step k may be read after step k + 2 has been submitted
    or after synchronize(). cot_host / grad_host may be None (forward only).
    """

    def __init__(self, mesh: Mesh, params: Params | None = None, **kw):
        self.mesh = mesh
        self.params = mesh._params(params, kw)
        if self.params.precision != "fp64":
            raise ValueError("StepPipeline runs the fp64 forward and adjoint")
        dev = mesh.device
        self.s_in = torch.cuda.Stream(dev)
        self.s_cmp = torch.cuda.Stream(dev)
        self.s_out = torch.cuda.Stream(dev)
        shape = (4, mesh.n_nodes)
        self.sets = []
        for _ in range(2):
            self.sets.append({
                "up": torch.empty(shape, dtype=torch.float64, device=dev),
                "cot": torch.empty(shape, dtype=torch.float64, device=dev),
                "rhs": torch.empty(shape, dtype=torch.float64, device=dev),
                "grad": torch.empty(shape, dtype=torch.float64, device=dev),
                "up_in": torch.cuda.Event(), "cot_in": torch.cuda.Event(),
                "fwd": torch.cuda.Event(), "done": torch.cuda.Event(),
                "free": torch.cuda.Event(), "used": False})

    def submit(self, k: int, up_host: torch.Tensor, cot_host: torch.Tensor | None,
               rhs_host: torch.Tensor, grad_host: torch.Tensor | None) -> None:
        b = self.sets[k % 2]
        with torch.cuda.stream(self.s_in):
            if b["used"]:
                self.s_in.wait_event(b["free"])
            b["up"].copy_(up_host, non_blocking=True)
            b["up_in"].record(self.s_in)
            if cot_host is not None:
                # the cotangent's copy overlaps this step's forward
                b["cot"].copy_(cot_host, non_blocking=True)
            b["cot_in"].record(self.s_in)
        with torch.cuda.stream(self.s_cmp):
            self.s_cmp.wait_event(b["up_in"])
            self.mesh.assemble(b["up"], self.params, out=b["rhs"])
            b["fwd"].record(self.s_cmp)
            if cot_host is not None:
                self.s_cmp.wait_event(b["cot_in"])
                self.mesh.assemble_vjp(b["up"], b["cot"], self.params, out=b["grad"])
            b["done"].record(self.s_cmp)
        with torch.cuda.stream(self.s_out):
            self.s_out.wait_event(b["fwd"])
            rhs_host.copy_(b["rhs"], non_blocking=True)
            self.s_out.wait_event(b["done"])
            if cot_host is not None:
                grad_host.copy_(b["grad"], non_blocking=True)
            b["free"].record(self.s_out)
        b["used"] = True

    def synchronize(self) -> None:
        for st in (self.s_in, self.s_cmp, self.s_out):
            st.synchronize()

"""Element partitions for a sharded assembly.

The paper calls the RHS assembly trivially parallel (Sec. VII): every
process assembles its own elements, and the only exchange is the sum of the
rows of the nodes that elements of several processes share. The library
itself runs one mesh on one GPU per process and holds no collective. A
sharded run creates one library mesh per part from the part's local
coordinates and connectivity, assembles it into a local RHS over the part's
owned and ghost nodes, and sums the interface rows over the parts with one
all-reduce of its own choosing (NCCL, gloo, ...).

This module is that host-side bookkeeping:

* slab_partition: elements split into n_parts slabs of equal element count
  along one axis (by element centroid);
* local node numbering per part: the nodes the part's elements touch, owned
  nodes first (a node is owned by the lowest-numbered part that touches
  it), then ghosts, each in ascending global id;
* the interface: the nodes touched by more than one part, in ascending
  global id; each part knows the local index and the interface slot of its
  interface nodes;
* interface_rows / apply_interface / exchange_interface: gather a local
  RHS's interface rows into a [4, n_iface] buffer, sum the buffers over the
  parts (the caller's all-reduce), and write the sums back. Afterwards every
  local row, owned or ghost, equals the row of the whole mesh's RHS;
* exchange_neighbours: the same result from point-to-point messages between
  the parts that share nodes (for slabs, one face per neighbour), which moves
  the shared rows only.

Host-side numpy for the partition; the exchange helpers are torch indexing
on whatever device the local RHS lives on.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MAX_PARTS = 63   # one bit per part in a 64-bit node mask


@dataclass
class Part:
    index: int
    n_parts: int
    elems: np.ndarray        # [E_p] int64 global element ids, ascending
    nodes: np.ndarray        # [N_p] int64 global node ids: owned, then ghosts
    n_owned: int
    conn: np.ndarray         # [4, E_p] int32 local node ids
    iface_local: np.ndarray  # [I_p] int64 local indices of the part's interface nodes
    iface_slot: np.ndarray   # [I_p] int64 their slots in the interface vector
    n_iface: int             # length of the interface vector (all parts)
    shared: dict             # q -> [S_pq] int64 local indices of the nodes shared with
                             # part q, in ascending global id (aligned on both sides)

    @property
    def n_nodes(self) -> int:
        return int(self.nodes.size)

    @property
    def n_elems(self) -> int:
        return int(self.elems.size)

    def local(self, nodal: np.ndarray) -> np.ndarray:
        """The part's columns of a [k, N] nodal array (coordinates, fields)."""
        return np.ascontiguousarray(nodal[:, self.nodes])


def slab_partition(coords: np.ndarray, conn: np.ndarray, n_parts: int,
                   axis: int = 2) -> list[Part]:
    """Split the elements of (coords [3, N], conn [4, E]) into n_parts slabs
    along `axis` by element centroid, with element counts that differ by at
    most one (ties in the centroid keep the element order)."""
    coords = np.asarray(coords, dtype=np.float64)
    conn = np.asarray(conn)
    if coords.ndim != 2 or coords.shape[0] != 3 or conn.ndim != 2 or conn.shape[0] != 4:
        raise ValueError("coords must be [3, N] and conn [4, E]")
    N, E = coords.shape[1], conn.shape[1]
    if not 1 <= n_parts <= min(MAX_PARTS, max(E, 1)):
        raise ValueError(f"n_parts must be in 1..min({MAX_PARTS}, n_elems)")
    if axis not in (0, 1, 2):
        raise ValueError("axis must be 0, 1 or 2")
    if conn.size and (conn.min() < 0 or conn.max() >= N):
        raise ValueError("conn holds a node index out of range")
    cent = coords[axis][conn].sum(axis=0)            # 4 x the centroid coordinate
    order = np.argsort(cent, kind="stable")
    bounds = [(p * E) // n_parts for p in range(n_parts + 1)]
    part_elems = [np.sort(order[bounds[p]:bounds[p + 1]]).astype(np.int64) for p in range(n_parts)]

    mask = np.zeros(N, dtype=np.uint64)
    for p, el in enumerate(part_elems):
        mask[conn[:, el].ravel()] |= np.uint64(1) << np.uint64(p)
    touched_by = np.zeros(N, dtype=np.int64)
    owner = np.full(N, -1, dtype=np.int64)
    for p in range(n_parts):
        has = ((mask >> np.uint64(p)) & np.uint64(1)) == 1
        touched_by += has
        owner[(owner < 0) & has] = p
    iface = np.flatnonzero(touched_by > 1).astype(np.int64)

    parts = []
    for p, el in enumerate(part_elems):
        has = ((mask >> np.uint64(p)) & np.uint64(1)) == 1
        mine = np.flatnonzero(has & (owner == p))
        ghosts = np.flatnonzero(has & (owner != p))
        nodes = np.concatenate([mine, ghosts]).astype(np.int64)
        g2l = np.full(N, -1, dtype=np.int64)
        g2l[nodes] = np.arange(nodes.size, dtype=np.int64)
        lconn = g2l[conn[:, el]].astype(np.int32)
        ifl = np.flatnonzero(touched_by[nodes] > 1).astype(np.int64)
        slot = np.searchsorted(iface, nodes[ifl]).astype(np.int64)
        shared = {}
        gif = np.sort(nodes[ifl])
        mif = mask[gif]
        for q in range(n_parts):
            if q != p:
                sel = ((mif >> np.uint64(q)) & np.uint64(1)) == 1
                if sel.any():
                    shared[q] = g2l[gif[sel]]
        parts.append(Part(p, n_parts, el, nodes, int(mine.size), np.ascontiguousarray(lconn),
                          ifl, slot, int(iface.size), shared))
    return parts


def _index(part: Part, device):
    import torch
    return (torch.as_tensor(part.iface_local, device=device),
            torch.as_tensor(part.iface_slot, device=device))


def interface_rows(rhs_local, part: Part):
    """[k, n_iface] buffer holding the part's interface rows at their slots
    and zeros elsewhere (rhs_local: [k, N_p] torch tensor)."""
    import torch
    il, sl = _index(part, rhs_local.device)
    buf = torch.zeros((rhs_local.shape[0], part.n_iface), dtype=rhs_local.dtype,
                      device=rhs_local.device)
    buf[:, sl] = rhs_local[:, il]
    return buf


def apply_interface(rhs_local, part: Part, summed):
    """Write the summed interface buffer back into the part's rows."""
    il, sl = _index(part, rhs_local.device)
    rhs_local[:, il] = summed[:, sl]
    return rhs_local


def exchange_interface(rhs_local, part: Part, all_reduce):
    """The one exchange step: interface_rows, the caller's in-place sum over
    the parts (e.g. torch.distributed.all_reduce), apply_interface."""
    buf = interface_rows(rhs_local, part)
    all_reduce(buf)
    return apply_interface(rhs_local, part, buf)


def exchange_neighbours(rhs_local, part: Part, sendrecv):
    """The exchange as point-to-point messages: to every part q it shares
    nodes with, this part sends its own rows of those nodes and receives q's
    ([k, S_pq] each, in ascending global id), then adds what it received.
    sendrecv(sends) takes {q: tensor to send to q} and returns {q: tensor
    received from q} (see torch_sendrecv). The bytes moved are the shared
    faces only, not the whole interface vector."""
    import torch
    idx = {q: torch.as_tensor(loc, device=rhs_local.device) for q, loc in part.shared.items()}
    sends = {q: rhs_local[:, i].contiguous() for q, i in idx.items()}
    recvs = sendrecv(sends)
    for q, i in idx.items():
        rhs_local[:, i] += recvs[q]
    return rhs_local


def torch_sendrecv(group=None):
    """A sendrecv for exchange_neighbours over torch.distributed: every
    message posted as a non-blocking send and receive, then all awaited."""
    import torch
    import torch.distributed as dist

    def run(sends):
        recvs = {q: torch.empty_like(t) for q, t in sends.items()}
        reqs = []
        for q in sorted(sends):
            reqs.append(dist.isend(sends[q], q, group=group))
            reqs.append(dist.irecv(recvs[q], q, group=group))
        for r in reqs:
            r.wait()
        return recvs

    return run

"""Element partitioning and the halo sum of interface-node contributions across ranks.

The paper partitions the mesh into blocks, lets every process form its elements, and only then
calls the assembly, which exchanges the contributions to nodes shared between processes (Section 6:
block partitioning; assembly after all local elements are computed). This module is that exchange
step for one GPU per rank: every rank owns a contiguous block of elements (slabs of the element
ordering), assembles their contributions into the rows of the nodes its elements touch, and
`halo_sum` adds the contributions to nodes owned by other ranks into their owners' rows
(point-to-point messages over torch.distributed: NCCL between GPUs, gloo on CPU). Fine-scale
unknowns are internal to elements and need no exchange (Section 5).

Node ownership: a node belongs to the lowest rank among the ranks whose elements touch it.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Part:
    rank: int
    n_ranks: int
    elems: np.ndarray          # global ids of the elements this rank forms
    nodes: np.ndarray          # global ids of every node its elements touch (sorted)
    owner: np.ndarray          # owner rank of each entry of `nodes`
    local_conn: np.ndarray     # connectivity of `elems` in local node numbering (int32)
    send: dict = field(default_factory=dict)   # rank -> local rows of ghost nodes it owns
    recv: dict = field(default_factory=dict)   # rank -> local rows of owned nodes it also touches

    @property
    def owned(self) -> np.ndarray:
        """Local rows of the nodes this rank owns."""
        return np.nonzero(self.owner == self.rank)[0]


def partition_elements(n_elems: int, n_ranks: int) -> list[np.ndarray]:
    """Contiguous, balanced blocks of the element ordering (slabs of a lattice ordering)."""
    bounds = np.linspace(0, n_elems, n_ranks + 1).round().astype(np.int64)
    return [np.arange(bounds[r], bounds[r + 1]) for r in range(n_ranks)]


def build_parts(conn: np.ndarray, n_nodes: int, n_ranks: int) -> list[Part]:
    """Partition a mesh for n_ranks and compute, for every rank, its touched nodes, their owners
    and the halo lists. Deterministic: every rank can call it and obtain the same result."""
    conn = np.asarray(conn)
    blocks = partition_elements(conn.shape[0], n_ranks)
    node_owner = np.full(n_nodes, n_ranks, dtype=np.int64)
    touched = []
    for r, el in enumerate(blocks):
        nd = np.unique(conn[el].ravel())
        touched.append(nd)
        node_owner[nd] = np.minimum(node_owner[nd], r)
    parts = []
    for r, el in enumerate(blocks):
        nd = touched[r]
        lookup = {int(g): i for i, g in enumerate(nd)}
        local_conn = np.vectorize(lookup.__getitem__, otypes=[np.int64])(conn[el]).astype(np.int32)
        parts.append(Part(rank=r, n_ranks=n_ranks, elems=el, nodes=nd, owner=node_owner[nd],
                          local_conn=local_conn))
    # halo lists: rank r sends its rows of nodes owned by s; owner s receives them in the same
    # (global id) order
    for r, p in enumerate(parts):
        for s in range(n_ranks):
            if s == r:
                continue
            ghost = np.nonzero(p.owner == s)[0]
            if ghost.size:
                p.send[s] = ghost
                q = parts[s]
                pos = np.searchsorted(q.nodes, p.nodes[ghost])
                q.recv[r] = pos
    return parts


def halo_sum(part: Part, local, group=None):
    """Add the contributions this rank holds for nodes owned by other ranks into their owners.

    local: torch tensor (n_touched, k) of this rank's assembled rows (any device the process
    group supports). Returns the same tensor with owned rows complete (ghost rows untouched)."""
    import torch
    import torch.distributed as dist
    reqs = []
    bufs = {}
    for s, rows in sorted(part.recv.items()):
        bufs[s] = torch.empty((rows.size,) + tuple(local.shape[1:]), dtype=local.dtype,
                              device=local.device)
        reqs.append(dist.irecv(bufs[s], src=s, group=group))
    sends = {}
    for s, rows in sorted(part.send.items()):
        idx = torch.as_tensor(rows, device=local.device)
        sends[s] = local.index_select(0, idx).contiguous()
        reqs.append(dist.isend(sends[s], dst=s, group=group))
    for rq in reqs:
        rq.wait()
    for s, rows in bufs.items():
        idx = torch.as_tensor(part.recv[s], device=local.device)
        local.index_add_(0, idx, rows)
    return local


def owned_sum_of_squares(part: Part, local, extra=None, group=None) -> float:
    """Global sum of squares over owned rows (plus `extra`, e.g. the fine-scale residuals of the
    rank's own elements), reduced over ranks."""
    import torch
    import torch.distributed as dist
    own = torch.as_tensor(part.owned, device=local.device)
    s = (local.index_select(0, own) ** 2).sum()
    if extra is not None:
        s = s + (extra ** 2).sum()
    s = s.reshape(1).to(torch.float64)
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    return float(s.item())

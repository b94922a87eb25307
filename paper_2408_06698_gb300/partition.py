"""Element partitions for the partitioned convection apply (host-side set-up).

The HOPU convection operator of Section 3.2 couples an element only to the elements that
share a facet with it (volume term on T, facet terms on the facets of T).  A partition
therefore owns a set of elements and reads one halo layer: the facet neighbours of its
elements that other partitions own.  Each partition is an ordinary context on its local
mesh (owned elements first, then the halo): its owned elements keep every facet with the
same geometry, orientation and sides as in the whole mesh (all of them follow from the
vertices' periodic representatives), so their outputs equal those of the whole mesh once
the halo holds the owners' values; the halo elements' other facets become boundary facets
and only change the halo's own outputs, which are discarded.

One apply = one halo exchange (the owners' L2 blocks of u and of the wind, packed and
unpacked by the library's kernels) + the apply on every partition.  Here the partitions
live on one device and the exchange is a device-to-device copy; the plan (who sends which
element to whom, in which order) is what a multi-device transport would carry, and
``exchange_host`` runs the same plan between CPU ranks of a torch.distributed group.
This module only arranges data; every step of the operator runs in the library.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch


def facet_neighbours(elems: np.ndarray, rep: np.ndarray | None) -> np.ndarray:
    """[E, d+1] element across local facet f (opposite local vertex f), -1 on the boundary.

    Facets are matched by their sorted periodic-representative vertex tuples."""
    elems = np.asarray(elems, dtype=np.int64)
    E, nv = elems.shape
    r = elems if rep is None else np.asarray(rep, dtype=np.int64)[elems]
    keys = np.stack([np.sort(np.delete(r, f, axis=1), axis=1) for f in range(nv)], axis=1)  # [E, d+1, d]
    flat = keys.reshape(E * nv, -1)
    _, inv = np.unique(flat, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    order = np.argsort(inv, kind="stable")
    nb = -np.ones(E * nv, dtype=np.int64)
    srt = inv[order]
    same = srt[1:] == srt[:-1]
    a, b = order[:-1][same], order[1:][same]
    nb[a] = b // nv
    nb[b] = a // nv
    return nb.reshape(E, nv)


@dataclass
class Partition:
    rank: int
    owned: np.ndarray                     # global ids, ascending
    halo: np.ndarray                      # global ids of the halo, ascending by (owner, id)
    halo_owner: np.ndarray                # owning partition of each halo element
    recv: dict = field(default_factory=dict)   # q -> local indices (in this partition) filled from q
    send: dict = field(default_factory=dict)   # q -> local indices (owned) that q needs, in q's recv order

    @property
    def local(self) -> np.ndarray:
        return np.concatenate([self.owned, self.halo])

    @property
    def n_owned(self) -> int:
        return len(self.owned)


def partitions_from_owner(elems, rep, owner: np.ndarray) -> list[Partition]:
    """Partitions (halo and exchange plan) for a given owner partition of every element."""
    owner = np.asarray(owner, dtype=np.int64)
    P = int(owner.max()) + 1
    nb = facet_neighbours(elems, rep)
    parts = []
    for p in range(P):
        owned = np.nonzero(owner == p)[0]
        cand = nb[owned].reshape(-1)
        cand = np.unique(cand[cand >= 0])
        halo = cand[owner[cand] != p]
        ho = owner[halo]
        order = np.lexsort((halo, ho))
        parts.append(Partition(p, owned, halo[order], ho[order]))
    pos = []
    for part in parts:
        m = {int(g): i for i, g in enumerate(part.local)}
        pos.append(m)
    for part in parts:
        for q in range(P):
            sel = np.nonzero(part.halo_owner == q)[0]
            if len(sel) == 0:
                continue
            part.recv[q] = part.n_owned + sel
            parts[q].send[part.rank] = np.array([pos[q][int(g)] for g in part.halo[sel]], dtype=np.int64)
    return parts


def slab_partitions(mesh, P: int) -> list[Partition]:
    """P slabs of a periodic box mesh (workloads.periodic_box_mesh numbering: d! simplices
    per cube, cube index with axis 0 fastest), cut along the last axis."""
    d, n = mesh.dim, mesh.n
    per_cube = 2 if d == 2 else 6
    cube = np.arange(mesh.n_elems) // per_cube
    layer = cube // n ** (d - 1)
    owner = (layer * P) // n
    return partitions_from_owner(mesh.elems, mesh.rep, owner)


def exchange_host(parts_or_part, local: np.ndarray, nloc: int, group=None) -> np.ndarray:
    """The halo exchange between CPU ranks of a torch.distributed group (gloo): this rank's
    partition sends the owned blocks its neighbours need and fills its halo blocks.
    local: [n_local, nloc] array of this rank's local L2 blocks; returns it updated."""
    import torch.distributed as dist
    part = parts_or_part
    reqs = []
    bufs = {}
    for q, idx in sorted(part.send.items()):
        reqs.append(dist.isend(torch.as_tensor(np.ascontiguousarray(local[idx])), q, group=group))
    for q, idx in sorted(part.recv.items()):
        bufs[q] = torch.empty((len(idx), nloc), dtype=torch.as_tensor(local).dtype)
        reqs.append(dist.irecv(bufs[q], q, group=group))
    for r in reqs:
        r.wait()
    for q, idx in part.recv.items():
        local[idx] = bufs[q].numpy()
    return local


class PartitionedHopu:
    """P logical partitions of one mesh on one device: one context per partition on its
    local mesh, the halo exchange by the library's pack / unpack kernels."""

    def __init__(self, coords, elems, rep, parts: list[Partition], device="cuda", **opts):
        from .hopu import Hopu
        self.parts = parts
        self.ctx = [Hopu(coords, np.asarray(elems)[p.local], rep, device=device, **opts) for p in parts]
        self.device = self.ctx[0].device
        self.nloc = self.ctx[0].n_l2 // self.ctx[0].n_elems
        ids = lambda a: torch.as_tensor(np.asarray(a, dtype=np.int32), device=self.device)
        self._plan = [(q, p.rank, ids(self.parts[q].send[p.rank]), ids(idx))
                      for p in parts for q, idx in sorted(p.recv.items())]

    def scatter(self, global_l2: torch.Tensor) -> list[torch.Tensor]:
        """Local L2 vectors of every partition from a global one: owned blocks filled, halo
        blocks zero (the exchange fills them)."""
        g = global_l2.reshape(-1, self.nloc)
        out = []
        for p, c in zip(self.parts, self.ctx):
            v = torch.zeros((len(p.local), self.nloc), dtype=c.dtype, device=self.device)
            v[: p.n_owned] = g[torch.as_tensor(p.owned, device=self.device)].to(c.dtype)
            out.append(v.reshape(-1))
        return out

    def gather(self, local: list[torch.Tensor], out: torch.Tensor) -> torch.Tensor:
        """The owned blocks of every partition into a global L2 vector."""
        o = out.reshape(-1, self.nloc)
        for p, v in zip(self.parts, local):
            o[torch.as_tensor(p.owned, device=self.device)] = v.reshape(-1, self.nloc)[: p.n_owned]
        return out

    def exchange(self, local: list[torch.Tensor]):
        """Fill every partition's halo blocks from their owners (pack on the owner's
        context, unpack on the reader's)."""
        for q, p, send_ids, recv_ids in self._plan:
            buf = self.ctx[q].pack_elements(send_ids, local[q])
            self.ctx[p].unpack_elements(recv_ids, buf, local[p])

    def apply_convection_l2(self, w_local: list[torch.Tensor], u_local: list[torch.Tensor]) -> list[torch.Tensor]:
        """One partitioned apply: the halo exchange of u and w, then every partition's apply.
        The owned blocks of the results are those of the whole mesh."""
        self.exchange(u_local)
        if any(w is not u for w, u in zip(w_local, u_local)):
            self.exchange(w_local)
        return [c.apply_convection_l2(w, u) for c, w, u in zip(self.ctx, w_local, u_local)]

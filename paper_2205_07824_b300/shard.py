"""Element partitions for the sharded LDG operators (Section 3.5: the mesh split over
ranks, one GPU each, with a ghost layer exchanged between them).

This module holds no arithmetic of the method: it decides which elements a rank owns,
which ghost copies of face neighbours it holds, in which order blocks travel between
ranks, and moves them with ``torch.distributed`` (point-to-point sends for the ghosts, a
sum all-reduce for the Krylov dot products). The library computes; see the stage and
sharded calls of ``include/ldg.h``.

Local layout of rank r: its owned elements (a contiguous range of the global numbering)
first, then its ghosts in increasing global number. Every element-major vector of the
rank (u, v, q, J.v, ...) follows that layout; the ghost blocks are refreshed by
:meth:`GhostExchange.exchange` before each stage that reads them.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from .synth import HEX, QUAD, TET, TRI, Mesh

# local vertex lists of the faces of each element type (faces are matched by their
# sorted vertex ids; the order of faces here is irrelevant)
_FACES = {
    TRI: [(0, 1), (1, 2), (2, 0)],
    QUAD: [(0, 2), (1, 3), (0, 1), (2, 3)],
    TET: [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)],
    HEX: [(0, 2, 4, 6), (1, 3, 5, 7), (0, 1, 4, 5), (2, 3, 6, 7), (0, 1, 2, 3), (4, 5, 6, 7)],
}


def face_neighbours(mesh: Mesh) -> np.ndarray:
    """[E][n_faces] global face neighbour of each element (-1 on the boundary), from the
    topological vertex ids (periodic seams share ids)."""
    faces = _FACES[mesh.etype]
    owner = {}
    nb = -np.ones((mesh.n_elem, len(faces)), dtype=np.int64)
    for e in range(mesh.n_elem):
        for f, loc in enumerate(faces):
            key = tuple(sorted(int(mesh.vid[e, i]) for i in loc))
            if key in owner:
                e2, f2 = owner.pop(key)
                nb[e, f], nb[e2, f2] = e2, e
            else:
                owner[key] = (e, f)
    return nb


@dataclass
class Shard:
    """Rank `rank` of `nparts`: owned global elements, ghosts, the local mesh and the
    exchange lists (local element positions, in a canonical order both sides share)."""
    rank: int
    nparts: int
    owned: np.ndarray          # global ids, increasing (a contiguous range)
    ghosts: np.ndarray         # global ids, increasing
    mesh: Mesh                 # owned elements first, then ghosts
    send: dict                 # peer -> local positions of owned elements that peer holds as ghosts
    recv: dict                 # peer -> local positions of ghosts that peer owns

    @property
    def n_owned(self) -> int:
        return int(len(self.owned))

    @property
    def n_local(self) -> int:
        return int(len(self.owned) + len(self.ghosts))

    def owned_of(self, global_vec: np.ndarray, block: int) -> np.ndarray:
        """The owned blocks of a global element-major vector."""
        return global_vec.reshape(-1, block)[self.owned].ravel()


def ranges(n_elem: int, nparts: int) -> list:
    """Balanced contiguous element ranges [lo, hi) of the ranks."""
    cut = [round(i * n_elem / nparts) for i in range(nparts + 1)]
    return [(cut[i], cut[i + 1]) for i in range(nparts)]


def partition(mesh: Mesh, nparts: int, rank: int, nb: np.ndarray | None = None) -> Shard:
    """Rank `rank`'s shard of `mesh` split into `nparts` contiguous element ranges (for
    the box meshes, slabs across the slowest axis), with one layer of face-neighbour
    ghosts."""
    nb = face_neighbours(mesh) if nb is None else nb
    rg = ranges(mesh.n_elem, nparts)
    owner = np.empty(mesh.n_elem, dtype=np.int64)
    for r, (lo, hi) in enumerate(rg):
        owner[lo:hi] = r
    lo, hi = rg[rank]
    owned = np.arange(lo, hi, dtype=np.int64)
    near = nb[lo:hi].ravel()
    ghosts = np.unique(near[(near >= 0) & ((near < lo) | (near >= hi))])
    local = np.concatenate([owned, ghosts])
    pos = {int(g): i for i, g in enumerate(local)}
    xg = None if mesh.xgeo is None else mesh.xgeo[local]
    bc = None if mesh.bc is None else mesh.bc[local]
    lm = Mesh(mesh.etype, mesh.xyz[local], mesh.vid[local], f"{mesh.name} rank {rank}/{nparts}", mesh.pg, xg, bc)
    recv = {}
    for g in ghosts:
        recv.setdefault(int(owner[g]), []).append(pos[int(g)])
    send = {}
    for peer in range(nparts):
        if peer == rank:
            continue
        plo, phi = rg[peer]
        pn = nb[plo:phi].ravel()
        theirs = np.unique(pn[(pn >= lo) & (pn < hi)])      # my elements that peer holds as ghosts
        if len(theirs):
            send[peer] = [pos[int(g)] for g in theirs]
    return Shard(rank, nparts, owned, ghosts, lm, {k: np.array(v) for k, v in send.items()},
                 {k: np.array(v) for k, v in recv.items()})


class GhostExchange:
    """Moves ghost blocks between ranks with ``torch.distributed`` point-to-point calls
    (NCCL for device tensors, gloo for host tensors) and sums dot products with an
    all-reduce. Blocks travel in increasing global element number on both sides."""

    def __init__(self, shard: Shard, group=None):
        self.shard = shard
        self.group = group

    def exchange(self, x, block: int):
        """Fill the ghost blocks of the element-major local vector x (a torch tensor of
        n_local * block entries) from their owners."""
        import torch
        import torch.distributed as dist
        sh = self.shard
        xv = x.view(-1, block)
        ops, bufs = [], []
        for peer in sorted(set(sh.send) | set(sh.recv)):
            if peer in sh.send:
                idx = torch.as_tensor(sh.send[peer], device=x.device)
                sb = xv.index_select(0, idx).contiguous()
                ops.append(dist.P2POp(dist.isend, sb, peer, group=self.group))
                bufs.append(sb)
            if peer in sh.recv:
                rb = torch.empty((len(sh.recv[peer]), block), dtype=x.dtype, device=x.device)
                ops.append(dist.P2POp(dist.irecv, rb, peer, group=self.group))
                bufs.append((peer, rb))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for b in bufs:
            if isinstance(b, tuple):
                peer, rb = b
                xv[torch.as_tensor(sh.recv[peer], device=x.device)] = rb
        if x.is_cuda:
            torch.cuda.synchronize(x.device)

    def allreduce_sum(self, buf):
        import torch
        import torch.distributed as dist
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=self.group)
        if buf.is_cuda:
            torch.cuda.synchronize(buf.device)


class _DevView:
    """A device pointer seen as a torch tensor (CUDA array interface, no copy)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (int(ptr), False), "version": 3}


def device_tensor(ptr, n):
    import torch
    return torch.as_tensor(_DevView(ptr, n), device="cuda")


EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p)


class LdgComm(ctypes.Structure):
    """Mirror of ``ldg_comm`` in include/ldg.h."""
    _fields_ = [("user", ctypes.c_void_p), ("exchange_ghosts", EXCHANGE_FN), ("allreduce_sum", ALLREDUCE_FN)]


def make_comm(transport, n_local: int):
    """An ``ldg_comm`` whose callbacks hand the library's device buffers to
    ``transport.exchange(tensor, block)`` and ``transport.allreduce_sum(tensor)``. Keep the
    returned object alive while the context uses it."""

    def ex(user, ptr, block, stream):
        try:
            transport.exchange(device_tensor(ptr, n_local * block), block)
            return 0
        except Exception:      # the library turns a non-zero status into LDG_ERR_CUDA
            return 1

    def ar(user, ptr, count, stream):
        try:
            transport.allreduce_sum(device_tensor(ptr, count))
            return 0
        except Exception:
            return 1

    f_ex, f_ar = EXCHANGE_FN(ex), ALLREDUCE_FN(ar)
    comm = LdgComm(None, f_ex, f_ar)
    comm._keep = (f_ex, f_ar, transport)
    return comm

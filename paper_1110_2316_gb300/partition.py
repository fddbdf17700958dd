"""One problem over several GPUs (Section 5.3 of the thesis).

The thesis evaluates the residuals of each processor's elements after the
element-boundary values of neighbouring elements have been exchanged, and
sums the two PCG scalars of every iteration over all processors.  Here a
part is a contiguous piece of a Morton-curve order of the elements
(``hpse_partition``); it runs as a mesh of its own elements followed by ghost
copies of the elements of other parts that share a face with them.  Before
each operator apply the ghosts receive the owners' current blocks
(``hpse_pack_blocks`` / ``hpse_unpack_blocks`` around a send/receive of the
packed buffers); the rows of the own elements are then exactly those of the
whole mesh, and the element-block preconditioner needs no exchange at all.

What is plain host logic here (the partition plan, the exchange schedule,
the distributed PCG loop) takes its collectives as callables, so that the
same code runs over ``torch.distributed`` (NCCL between GPUs, gloo between
CPU ranks) or between parts emulated in one process.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from types import SimpleNamespace
from typing import Callable, Dict, List

import numpy as np

from . import _lib
from ._lib import check


def partition(desc, n_parts: int) -> np.ndarray:
    """owner[e] in [0, n_parts) for every element of a box mesh (hpse_partition)."""
    lib = _lib.load()
    keep = [np.ascontiguousarray(desc.elem_W, dtype=np.int32),
            np.ascontiguousarray(desc.elem_problem, dtype=np.int32),
            np.ascontiguousarray(desc.elem_lo, dtype=np.float64),
            np.ascontiguousarray(desc.elem_hi, dtype=np.float64),
            np.ascontiguousarray(desc.elem_nbr, dtype=np.int32)]
    d = _lib.MeshDesc()
    d.n_elem = int(keep[0].shape[0])
    d.n_problem = int(desc.n_problem)
    d.n_rhs = 1
    d.coord = _lib.COORD_CARTESIAN
    d.elem_W, d.elem_problem, d.elem_lo, d.elem_hi, d.elem_nbr = (k.ctypes.data_as(C.c_void_p) for k in keep)
    owner = np.zeros(d.n_elem, dtype=np.int32)
    check(lib.hpse_partition(C.byref(d), int(n_parts), owner.ctypes.data_as(C.c_void_p)), "hpse_partition")
    return owner


@dataclass
class LocalPart:
    """Part ``rank`` of a partitioned mesh.

    gids: local element -> global element (own elements first, ascending, then
    the ghosts, ascending); desc: the local mesh (box-mesh description with
    local neighbour ids, a ghost's faces towards elements outside the part
    marked Dirichlet, local problem ids); prob_g: local problem -> global
    problem; send[q] / recv[q]: local ids of the own elements part q holds as
    ghosts / of the ghosts owned by q, both ascending in global id (so that
    the two sides of an exchange agree on the order)."""
    rank: int
    n_owned: int
    gids: np.ndarray
    desc: object
    prob_g: np.ndarray
    send: Dict[int, np.ndarray] = field(default_factory=dict)
    recv: Dict[int, np.ndarray] = field(default_factory=dict)

    def owned_dofs(self) -> int:
        W = np.asarray(self.desc.elem_W[:self.n_owned], dtype=np.int64)
        return int(np.sum((W + 1) ** 3))


def local_part(desc, owner: np.ndarray, rank: int) -> LocalPart:
    nbr = np.asarray(desc.elem_nbr)
    owned = np.nonzero(owner == rank)[0]
    adj = nbr[owned].ravel()
    adj = adj[adj >= 0]
    ghosts = np.unique(adj[owner[adj] != rank])
    gids = np.concatenate([owned, ghosts]).astype(np.int64)
    g2l = -np.ones(len(owner), dtype=np.int64)
    g2l[gids] = np.arange(len(gids))
    lnbr = nbr[gids].astype(np.int64)
    inside = lnbr >= 0
    lnbr[inside] = g2l[lnbr[inside]]          # outside the part -> -1 (only on ghosts)
    gprob = np.asarray(desc.elem_problem)[gids]
    prob_g, lprob = np.unique(gprob, return_inverse=True)
    if len(prob_g) == 0:   # a part without elements (more parts than elements)
        prob_g = np.zeros(1, dtype=np.int64)
    ldesc = SimpleNamespace(elem_lo=np.asarray(desc.elem_lo)[gids].copy(), elem_hi=np.asarray(desc.elem_hi)[gids].copy(),
                            elem_W=np.asarray(desc.elem_W)[gids].astype(np.int32),
                            elem_nbr=lnbr.astype(np.int32), elem_problem=lprob.astype(np.int32),
                            n_problem=int(len(prob_g)))
    ldesc.n_elem = len(gids)
    part = LocalPart(rank, len(owned), gids, ldesc, prob_g.astype(np.int64))
    n_owned = len(owned)
    for q in np.unique(owner[ghosts]) if len(ghosts) else []:
        q = int(q)
        part.recv[q] = n_owned + np.nonzero(owner[ghosts] == q)[0]
        # own elements with a face towards an element of q
        touch = [i for i, e in enumerate(owned) if np.any(owner[nbr[e][nbr[e] >= 0]] == q)]
        part.send[q] = np.asarray(touch, dtype=np.int64)
    return part


def local_problem(problem, part: LocalPart):
    """The data of ``problem`` (a workloads Problem, possibly a batch with
    ``parts``) on a part's local mesh."""
    out = SimpleNamespace(**{k: v for k, v in vars(problem).items()})
    out.mesh = part.desc
    parts = getattr(problem, "parts", None)
    if parts is not None:
        out.parts = [parts[int(g)] for g in part.prob_g]
    return out


class Halo:
    """Device plan of one part's exchange: per peer the element lists and
    buffer offsets, packed and unpacked by the library's block kernels."""

    def __init__(self, mesh, part: LocalPart):
        import torch
        self.mesh, self.part = mesh, part
        dev = torch.device("cuda", mesh.device)
        W = np.asarray(part.desc.elem_W, dtype=np.int64)
        self.plan = {}
        for kind, table in (("send", part.send), ("recv", part.recv)):
            for q, items in table.items():
                sz = (W[items] + 1) ** 3
                off = np.concatenate([[0], np.cumsum(sz)[:-1]]).astype(np.int64)
                self.plan[(kind, q)] = (torch.tensor(items.astype(np.int32), device=dev),
                                        torch.tensor(off, device=dev), int(len(items)), int(np.sum(sz)))

    def buffer(self, kind, q, like):
        import torch
        _, _, _, n = self.plan[(kind, q)]
        return torch.empty(self.mesh.n_rhs * n, dtype=like.dtype, device=like.device)

    def pack(self, q, vec, buf, stream=None):
        items, off, n, ln = self.plan[("send", q)]
        from .api import _ptr, _stream, _prec_of
        check(self.mesh._lib.hpse_pack_blocks(self.mesh._h, _prec_of(vec), _ptr(items), _ptr(off), n, ln,
                                              _ptr(vec), _ptr(buf), _stream(stream)), "hpse_pack_blocks")

    def unpack(self, q, buf, vec, stream=None):
        items, off, n, ln = self.plan[("recv", q)]
        from .api import _ptr, _stream, _prec_of
        check(self.mesh._lib.hpse_unpack_blocks(self.mesh._h, _prec_of(vec), _ptr(items), _ptr(off), n, ln,
                                                _ptr(buf), _ptr(vec), _stream(stream)), "hpse_unpack_blocks")

    def exchange(self, vec):
        """Ghost update over torch.distributed (one send and one receive per
        peer, posted together)."""
        import torch.distributed as dist
        reqs, bufs = [], []
        for q in sorted(self.part.recv):
            rb = self.buffer("recv", q, vec)
            bufs.append((q, rb))
            reqs.append(dist.irecv(rb, src=q))
        for q in sorted(self.part.send):
            sb = self.buffer("send", q, vec)
            self.pack(q, vec, sb)
            reqs.append(dist.isend(sb, dst=q))
        for r in reqs:
            r.wait()
        for q, rb in bufs:
            self.unpack(q, rb, vec)


def exchange_emulated(halos: List[Halo], vecs) -> None:
    """Ghost update between parts held by one process (each part's own mesh
    and vector): part r's ghosts from part q are q's packed send to r."""
    for r, h in enumerate(halos):
        for q in sorted(h.part.recv):
            buf = halos[q].buffer("send", r, vecs[q])
            halos[q].pack(r, vecs[q], buf)
            h.unpack(q, buf, vecs[r])


def dist_pcg(apply: Callable, precond: Callable, exchange: Callable, allreduce: Callable, b, n_own: int,
             tol: float = 1e-10, max_iter: int = 10000, n_rhs: int = 1):
    """PCG (Section 5.1) on a vector distributed over parts: every vector is
    the part's local vector, ``n_rhs`` right-hand sides of n_local entries
    each (own DOFs first, ghost blocks after, the library's layout); dot
    products run over each right-hand side's own DOFs and are summed over the
    parts by ``allreduce`` (FP64, one value per right-hand side); ``exchange``
    refreshes p's ghosts before each apply.  Each right-hand side keeps its
    own alpha and beta and stops at ||r|| <= tol ||b|| (global norms); the
    loop ends when all have.  Returns (x, iterations, largest relative
    residual)."""
    import torch

    R = int(n_rhs)
    if R < 1 or b.numel() % R:
        raise ValueError("b holds %d entries, not a whole number of %d right-hand sides" % (b.numel(), R))
    nl = b.numel() // R
    if not 0 <= n_own <= nl:
        raise ValueError("n_own = %d outside one right-hand side's %d entries" % (n_own, nl))

    def rows(v):
        return v.view(R, nl)

    def dot(a, c):
        return allreduce((rows(a)[:, :n_own] * rows(c)[:, :n_own]).sum(1))

    def own_only(v):
        rows(v)[:, n_own:] = 0

    x = torch.zeros_like(b)
    r = b.clone()
    own_only(r)
    bn = torch.sqrt(dot(b, b))
    bn = torch.where(bn > 0, bn, torch.ones_like(bn))
    z = torch.empty_like(b)
    precond(r, z)
    own_only(z)
    p = z.clone()
    rz = dot(r, z)
    q = torch.empty_like(b)
    rel = torch.sqrt(dot(r, r)) / bn
    it = 0
    while float(rel.max()) > tol and it < max_iter:
        live = rel > tol
        exchange(p)
        apply(p, q)
        own_only(q)
        pq = dot(p, q)
        alpha = torch.where(live, rz / torch.where(live, pq, torch.ones_like(pq)), torch.zeros_like(pq))
        rows(x).add_(alpha[:, None] * rows(p))
        rows(r).sub_(alpha[:, None] * rows(q))
        precond(r, z)
        own_only(z)
        rz_new = dot(r, z)
        beta = torch.where(live, rz_new / torch.where(live, rz, torch.ones_like(rz)), torch.zeros_like(rz))
        p = (rows(z) + beta[:, None] * rows(p)).reshape(-1)
        rz = torch.where(live, rz_new, rz)
        it += 1
        rel = torch.where(live, torch.sqrt(dot(r, r)) / bn, rel)
    return x, it, float(rel.max())

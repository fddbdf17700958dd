"""One problem over several parts (Section 5.3): the partition plan and the
ghost exchange, on CPU ranks.

* hpse_partition: every element in one part; the parts are contiguous pieces
  of the Morton order of the element centres (recomputed here) within each
  problem, balanced to one element's weight.
* local parts: symmetric local adjacency; the ghosts are exactly the
  neighbours across the cuts; part r's receive list from q is q's send list
  to r, in the same order.
* two gloo ranks: after the ghost exchange the own rows of each part's
  operator (oracle, local mesh) are the rows of the whole mesh's A u; the
  distributed PCG (own-DOF dot products summed over the ranks, ghosts
  refreshed before each apply, element-block preconditioner) reaches the
  whole mesh's solution.
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as wl
from paper_1110_2316_gb300 import partition as pt


def _morton_key(c):
    k = 0
    for b in range(21):
        for a in range(3):
            k |= ((int(c[a]) >> b) & 1) << (3 * b + a)
    return k


def _mixed_batch():
    a = wl.box_mesh((4, 3, 2), W=3)
    b = wl.box_mesh((2, 2, 2), lo=(0, 0, 0), hi=(2.0, 1.0, 1.0), W=5)
    return wl.concat_meshes([a, b])


def test_partition_is_contiguous_along_the_curve_and_balanced():
    desc = _mixed_batch()
    for n_parts in (1, 2, 3, 5):
        owner = pt.partition(desc, n_parts)
        assert owner.min() >= 0 and owner.max() < n_parts
        # Morton order recomputed from the box centres, per problem
        keys = []
        for e in range(desc.n_elem):
            p = desc.elem_problem[e]
            sel = desc.elem_problem == p
            cen = 0.5 * (desc.elem_lo + desc.elem_hi)
            lo, hi = cen[sel].min(axis=0), cen[sel].max(axis=0)
            q = [int(np.floor((cen[e, a] - lo[a]) / (hi[a] - lo[a]) * (2 ** 21 - 1) + 0.5)) if hi[a] > lo[a] else 0
                 for a in range(3)]
            keys.append((int(p), _morton_key(q), e))
        order = [k[2] for k in sorted(keys)]
        seq = owner[order]
        assert np.all(np.diff(seq) >= 0)                       # contiguous pieces
        w = (desc.elem_W.astype(np.int64) + 1) ** 3
        loads = np.array([w[owner == r].sum() for r in range(n_parts)])
        assert loads.max() - loads.min() <= 2 * w.max(), loads   # balanced to an element


def test_local_parts_and_exchange_lists():
    desc = wl.box_mesh((4, 3, 2), W=3)
    owner = pt.partition(desc, 3)
    parts = [pt.local_part(desc, owner, r) for r in range(3)]
    for p in parts:
        d = p.desc
        assert np.all(owner[p.gids[:p.n_owned]] == p.rank)
        assert np.all(owner[p.gids[p.n_owned:]] != p.rank)
        for e in range(d.n_elem):
            for f in range(6):
                n = d.elem_nbr[e, f]
                if n >= 0:
                    assert d.elem_nbr[n, f ^ 1] == e
                    assert desc.elem_nbr[p.gids[e], f] == p.gids[n]
            if e < p.n_owned:   # own elements keep every neighbour
                assert np.array_equal(d.elem_nbr[e] >= 0, desc.elem_nbr[p.gids[e]] >= 0)
        ghosts = set(p.gids[p.n_owned:].tolist())
        want = {int(n) for e in p.gids[:p.n_owned] for n in desc.elem_nbr[e] if n >= 0 and owner[n] != p.rank}
        assert ghosts == want
    for r in range(3):
        for q, items in parts[r].recv.items():
            assert np.array_equal(parts[r].gids[items], parts[q].gids[parts[q].send[r]])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _blocks(disc, items):
    return [slice(int(disc.off[i]), int(disc.off[i + 1])) for i in items]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import scipy.linalg as sla
        from oracle.functional import Discretisation
        from oracle.precond import element_block
        pb = wl.poisson_sine(n=(4, 1, 1), W=2)
        owner = pt.partition(pb.mesh, ws)
        part = pt.local_part(pb.mesh, owner, rank)
        d = Discretisation(pt.local_problem(pb, part))
        n_own = part.owned_dofs()

        def exchange(v):
            # pack own blocks for each peer, send, receive the ghosts
            reqs, recv = [], []
            for q in sorted(part.recv):
                buf = torch.empty(sum(s.stop - s.start for s in _blocks(d, part.recv[q])), dtype=v.dtype)
                recv.append((q, buf))
                reqs.append(dist.irecv(buf, src=q))
            for q in sorted(part.send):
                buf = torch.cat([v[s] for s in _blocks(d, part.send[q])])
                reqs.append(dist.isend(buf, dst=q))
            for rq in reqs:
                rq.wait()
            for q, buf in recv:
                o = 0
                for s in _blocks(d, part.recv[q]):
                    v[s] = buf[o:o + s.stop - s.start]
                    o += s.stop - s.start

        # a global vector, each rank starting from its own blocks only
        full = Discretisation(pb)
        U = wl.random_dofs(full.ndof, seed=21)
        u = torch.zeros(d.ndof, dtype=torch.float64)
        for i, g in enumerate(part.gids[:part.n_owned]):
            u[int(d.off[i]):int(d.off[i + 1])] = torch.tensor(U[full.off[g]:full.off[g + 1]])
        exchange(u)
        y = d.apply_A(u.numpy(), elems=range(part.n_owned))
        rows = {int(g): y[d.off[i]:d.off[i + 1]] for i, g in enumerate(part.gids[:part.n_owned])}

        def allreduce(t):
            dist.all_reduce(t)
            return t

        fac = [sla.cho_factor(element_block(d, e)) for e in range(part.n_owned)]

        def apply(p, q):
            q.copy_(torch.tensor(d.apply_A(p.numpy(), elems=range(part.n_owned))))

        def precond(r, z):
            z.zero_()
            for e in range(part.n_owned):
                s = slice(int(d.off[e]), int(d.off[e + 1]))
                z[s] = torch.tensor(sla.cho_solve(fac[e], r[s].numpy()))

        b = torch.tensor(d.rhs_b())
        x, it, rel = pt.dist_pcg(apply, precond, exchange, allreduce, b, n_own, tol=1e-11, max_iter=2000)
        xs = {int(g): x[d.off[i]:d.off[i + 1]].numpy() for i, g in enumerate(part.gids[:part.n_owned])}
        got = [None] * ws
        dist.all_gather_object(got, (rows, xs, it, rel))
        if rank == 0:
            out.put(got)
    finally:
        dist.destroy_process_group()


def test_two_rank_ghost_exchange_apply_and_pcg():
    from oracle.functional import Discretisation
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=600)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pb = wl.poisson_sine(n=(4, 1, 1), W=2)
    full = Discretisation(pb)
    U = wl.random_dofs(full.ndof, seed=21)
    y = full.apply_A(U)
    rows = {**got[0][0], **got[1][0]}
    assert sorted(rows) == list(range(full.E))
    for g, v in rows.items():
        np.testing.assert_allclose(v, y[full.off[g]:full.off[g + 1]], rtol=0, atol=1e-13 * np.abs(y).max())
    x_ref = np.linalg.solve(full.dense_A(), full.rhs_b())
    xs = {**got[0][1], **got[1][1]}
    x = np.concatenate([xs[g] for g in range(full.E)])
    assert got[0][3] <= 1e-11 and got[0][2] == got[1][2]
    assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)


def test_more_parts_than_elements():
    desc = wl.box_mesh((2, 1, 1), W=2)
    owner = pt.partition(desc, 4)
    assert sorted(np.unique(owner).tolist()) == sorted(set(owner.tolist()))
    assert np.bincount(owner, minlength=4).sum() == 2
    for r in range(4):
        p = pt.local_part(desc, owner, r)
        assert p.n_owned == int(np.sum(owner == r)) and p.desc.n_problem >= 1
        if p.n_owned == 0:
            assert p.desc.n_elem == 0 and not p.send and not p.recv


def test_dist_pcg_several_rhs_each_converges():
    # one part, no peers: the vectors hold 3 right-hand sides of n_local
    # entries each (own DOFs first, then ghost entries that must stay out of
    # every dot product); each right-hand side has its own alpha and beta and
    # the result equals three separate dense solves
    rng = np.random.default_rng(3)
    n_own, n_gh, R = 12, 5, 3
    nl = n_own + n_gh
    M = rng.standard_normal((n_own, n_own))
    A = M @ M.T + n_own * np.eye(n_own)
    scales = [1.0, 1e3, 1e-2]
    B = np.zeros((R, nl))
    for r in range(R):
        B[r, :n_own] = scales[r] * rng.standard_normal(n_own)
        B[r, n_own:] = 1e6  # ghost entries: must not enter the sums
    Ad = torch.tensor(A)

    def apply(p, q):
        pv, qv = p.view(R, nl), q.view(R, nl)
        qv[:, :n_own] = pv[:, :n_own] @ Ad.T
        qv[:, n_own:] = 7.0

    def precond(r, z):
        z.copy_(r / float(A[0, 0]))

    x, it, rel = pt.dist_pcg(apply, precond, lambda v: None, lambda t: t, torch.tensor(B.ravel()), n_own,
                             tol=1e-12, max_iter=200, n_rhs=R)
    assert rel <= 1e-12
    X = x.view(R, nl).numpy()
    for r in range(R):
        xo = np.linalg.solve(A, B[r, :n_own])
        assert np.linalg.norm(X[r, :n_own] - xo) <= 1e-10 * np.linalg.norm(xo), r
    try:
        pt.dist_pcg(apply, precond, lambda v: None, lambda t: t, torch.zeros(nl * R + 1), n_own, n_rhs=R)
        raise AssertionError("a vector that is not a whole number of right-hand sides was accepted")
    except ValueError:
        pass

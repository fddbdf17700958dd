"""One problem over several parts through the CUDA library (Section 5.3),
the parts emulated on one GPU: each part is its own mesh (own elements +
ghost copies), the ghost exchange runs through hpse_pack_blocks /
hpse_unpack_blocks, and no kernel ever waits for another part (the parts
synchronise on the host only).

* pack / unpack move element blocks exactly (FP64 and FP32, several rhs).
* After the exchange the own rows of every part's A u equal the whole mesh's.
* The distributed PCG (one host thread per part, own-DOF dot products summed
  on the host, element-block preconditioner) reaches the whole mesh's
  solution.
"""
import threading

import numpy as np
import pytest
import torch

import workloads as wl
from paper_1110_2316_gb300 import partition as pt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api as A
    return A


def _parts(api, pb, n_parts, n_rhs=1):
    owner = pt.partition(pb.mesh, n_parts)
    parts = [pt.local_part(pb.mesh, owner, r) for r in range(n_parts)]
    meshes = []
    for p in parts:
        m = api.Mesh(p.desc, n_rhs=n_rhs, coef_kind=api.COEF_SCALAR if pb.a is not None else api.COEF_LAPLACE)
        m.set_data(**api.problem_data_arrays(m, pt.local_problem(pb, p)))
        meshes.append(m)
    return parts, meshes, [pt.Halo(m, p) for m, p in zip(meshes, parts)]


def _offsets(W):
    return np.concatenate([[0], np.cumsum((np.asarray(W, dtype=np.int64) + 1) ** 3)])


def _scatter(parts, U, W_glob, dtype, n_rhs=1):
    """Each part's local vector holding only its own blocks of the global U."""
    og = _offsets(W_glob)
    nd = og[-1]
    out = []
    for p in parts:
        ol = _offsets(p.desc.elem_W)
        v = np.zeros((n_rhs, ol[-1]))
        for i, g in enumerate(p.gids[:p.n_owned]):
            v[:, ol[i]:ol[i + 1]] = U.reshape(n_rhs, nd)[:, og[g]:og[g + 1]]
        out.append(torch.tensor(v.ravel(), dtype=dtype, device="cuda"))
    return out


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_pack_unpack_blocks_exact(api, dtype):
    pb = wl.varcoef_random_rhs(n=3, W=4, n_rhs=3)
    parts, meshes, halos = _parts(api, pb, 3, n_rhs=3)
    for r, (p, m, h) in enumerate(zip(parts, meshes, halos)):
        v = torch.randn(3 * m.ndof, dtype=dtype, device="cuda")
        ol = _offsets(p.desc.elem_W)
        for q in p.send:
            buf = h.buffer("send", q, v)
            h.pack(q, v, buf)
            want = torch.cat([v.view(3, -1)[:, ol[i]:ol[i + 1]] for i in p.send[q]], dim=1).reshape(-1)
            assert torch.equal(buf, want)
        for q in p.recv:
            buf = torch.randn(3 * sum(int(ol[i + 1] - ol[i]) for i in p.recv[q]), dtype=dtype, device="cuda")
            w = v.clone()
            h.unpack(q, buf, w)
            got = torch.cat([w.view(3, -1)[:, ol[i]:ol[i + 1]] for i in p.recv[q]], dim=1).reshape(-1)
            assert torch.equal(got, buf)
            mask = torch.ones(m.ndof, dtype=torch.bool, device="cuda")
            for i in p.recv[q]:
                mask[ol[i]:ol[i + 1]] = False
            assert torch.equal(w.view(3, -1)[:, mask], v.view(3, -1)[:, mask])
    for m in meshes:
        m.close()


@pytest.mark.parametrize("n_parts", [2, 3])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_partitioned_apply_equals_whole_mesh(api, n_parts, dtype):
    pb = wl.varcoef_random_rhs(n=4, W=5, n_rhs=1)
    whole = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_SCALAR)
    whole.set_data(**api.problem_data_arrays(whole, pb))
    U = wl.random_dofs(whole.ndof, seed=31)
    u = torch.tensor(U, dtype=dtype, device="cuda")
    y = torch.empty_like(u)
    whole.apply_operator(u, y)
    y = y.double().cpu().numpy()
    parts, meshes, halos = _parts(api, pb, n_parts)
    vecs = _scatter(parts, U, pb.mesh.elem_W, dtype)
    pt.exchange_emulated(halos, vecs)
    og = _offsets(pb.mesh.elem_W)
    for p, m, v in zip(parts, meshes, vecs):
        yl = torch.empty_like(v)
        m.apply_operator(v, yl)
        yl = yl.double().cpu().numpy()
        ol = _offsets(p.desc.elem_W)
        for i, g in enumerate(p.gids[:p.n_owned]):
            # the same arithmetic on the same data: equal to the last bit
            np.testing.assert_array_equal(yl[ol[i]:ol[i + 1]], y[og[g]:og[g + 1]])
        m.close()
    whole.close()


def test_distributed_pcg_equals_whole_mesh_solve(api):
    pb = wl.varcoef_random_rhs(n=4, W=4, n_rhs=1)
    whole = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_SCALAR)
    whole.set_data(**api.problem_data_arrays(whole, pb))
    whole.setup_block_preconditioner()
    xw = torch.zeros(whole.ndof, dtype=torch.float64, device="cuda")
    assert whole.pcg_solve(xw, tol=1e-11, prec=api.FP64, max_iter=20000)["status"] == 0
    xw = xw.cpu().numpy()
    n = 2
    parts, meshes, halos = _parts(api, pb, n)
    for m in meshes:
        m.setup_block_preconditioner()
    barrier = threading.Barrier(n, timeout=120)
    shared, results = {}, [None] * n

    def run(r):
        p, m, h = parts[r], meshes[r], halos[r]

        def exchange(v):
            for q in p.send:
                buf = h.buffer("send", q, v)
                h.pack(q, v, buf)
                shared[(r, q)] = buf
            barrier.wait()
            for q in p.recv:
                h.unpack(q, shared[(q, r)], v)
            barrier.wait()

        def allreduce(t):
            shared[("s", r)] = t.clone()
            barrier.wait()
            s = sum(shared[("s", q)] for q in range(n))
            barrier.wait()
            return s

        b = torch.empty(m.ndof, dtype=torch.float64, device="cuda")
        m.get_rhs(b)
        x, it, rel = pt.dist_pcg(lambda a, c: m.apply_operator(a, c), lambda a, c: m.apply_preconditioner(a, c),
                                 exchange, allreduce, b, p.owned_dofs(), tol=1e-11, max_iter=5000,
                                 n_rhs=m.n_rhs)
        torch.cuda.synchronize()
        results[r] = (x.cpu().numpy(), it, rel)

    threads = [threading.Thread(target=run, args=(r,)) for r in range(n)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert all(res is not None for res in results)
    assert results[0][1] == results[1][1] and results[0][2] <= 1e-11
    og = _offsets(pb.mesh.elem_W)
    x = np.zeros_like(xw)
    for p, (xl, _, _) in zip(parts, results):
        ol = _offsets(p.desc.elem_W)
        for i, g in enumerate(p.gids[:p.n_owned]):
            x[og[g]:og[g + 1]] = xl[ol[i]:ol[i + 1]]
    assert np.linalg.norm(x - xw) <= 1e-8 * np.linalg.norm(xw)
    for m in meshes:
        m.close()
    whole.close()

"""GPU parity of the PCG driver (FP64 and FP32 applies + FP64 refinement) and
of the H^1 error against the CPU oracle.

Tolerances:
* solution vs oracle solution: both stop at ||b - A x|| <= 1e-10 ||b||, so they
  may differ by up to kappa(A) * 1e-10 in the small eigen-directions; the
  comparison is made in the relative H^1 norm and required <= 1e-8;
* H^1 error computed on the GPU vs the oracle's on the same vector: 1e-10 relative.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.functional import Discretisation
from oracle.h1 import h1_error_exact, h1_rel_diff
from oracle.pcg import pcg
from oracle.precond import apply_Cinv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api as A
    return A


def _mesh(api, pb, n_rhs=1):
    kind = api.COEF_SCALAR if pb.a is not None else api.COEF_LAPLACE
    m = api.Mesh(pb.mesh, n_rhs=n_rhs, coef_kind=kind)
    m.set_data(**api.problem_data_arrays(m, pb))
    return m


def _solve(api, mesh, prec, tol=1e-10, **kw):
    x = torch.zeros(mesh.n_rhs * mesh.ndof, dtype=torch.float64, device="cuda")
    rep = mesh.pcg_solve(x, tol=tol, prec=prec, **kw)
    torch.cuda.synchronize()
    return x.cpu().numpy(), rep


@pytest.mark.parametrize("maker", [lambda: wl.poisson_sine(n=2, W=4),
                                   lambda: wl.varcoef_manufactured(n=(3, 2, 2), W=5)])
def test_fp64_and_mixed_solutions_match_oracle(api, maker):
    pb = maker()
    mesh = _mesh(api, pb)
    disc = Discretisation(pb)
    xo, it_o, rel_o = pcg(disc.apply_A, lambda r: apply_Cinv(disc, r), disc.rhs_b(), tol=1e-10)
    x64, rep64 = _solve(api, mesh, api.FP64)
    assert rep64["status"] == 0 and rep64["rel_residual"] <= 1e-10
    assert abs(rep64["iterations"] - it_o) <= max(3, it_o // 20), (rep64, it_o)
    assert h1_rel_diff(disc, x64, xo) <= 1e-8
    xm, repm = _solve(api, mesh, api.FP32)
    assert repm["status"] == 0 and repm["rel_residual"] <= 1e-10, repm
    assert h1_rel_diff(disc, xm, x64) <= 1e-8
    e_or = h1_error_exact(disc, xo)
    assert abs(h1_error_exact(disc, xm) - e_or) <= 1e-6 * e_or


def test_polynomial_reproduction_on_gpu(api):
    pb = wl.polynomial_exact(n=2, W=3)
    mesh = _mesh(api, pb)
    disc = Discretisation(pb)
    x, rep = _solve(api, mesh, api.FP64, tol=1e-12)
    assert np.abs(x - disc.nodal_interpolant(pb.u_exact[0])).max() < 1e-9


def test_h1_error_matches_oracle(api):
    pb = wl.poisson_sine(n=2, W=5)
    mesh = _mesh(api, pb)
    disc = Discretisation(pb)
    U = disc.nodal_interpolant(pb.u_exact[0]) + 1e-3 * wl.random_dofs(mesh.ndof, seed=2)
    u = torch.tensor(U, device="cuda")
    # exact solution sampled at the volume points
    ax, _ = mesh.query_points()
    vq, gq = [], [[], [], []]
    o = 0
    for e in range(mesh.n_elem):
        Q = 2 * int(mesh.elem_W[e]) + 1
        xs, ys, zs = ax[o:o + Q], ax[o + Q:o + 2 * Q], ax[o + 2 * Q:o + 3 * Q]
        o += 3 * Q
        vq.append(pb.u_exact[0](xs, ys, zs).ravel())
        for k, g in enumerate(pb.grad_u_exact[0](xs, ys, zs)):
            gq[k].append(np.broadcast_to(g, (Q, Q, Q)).ravel())
    vq = torch.tensor(np.concatenate(vq), device="cuda")
    gq = torch.tensor(np.concatenate([np.concatenate(g) for g in gq]), device="cuda")
    out = mesh.h1_error(u, vq=vq, gq=gq)
    rel_gpu = np.sqrt(out[0, 0] / out[0, 1])
    rel_or = h1_error_exact(disc, U)
    assert abs(rel_gpu - rel_or) <= 1e-10 * rel_or
    # against a reference DOF vector
    V = disc.nodal_interpolant(pb.u_exact[0])
    out2 = mesh.h1_error(u, ref=torch.tensor(V, device="cuda"))
    assert abs(np.sqrt(out2[0, 0] / out2[0, 1]) - h1_rel_diff(disc, U, V)) <= 1e-10 * h1_rel_diff(disc, U, V)


def test_batched_rhs_and_problems(api):
    # two problems (degrees 3 and 4) x 2 right-hand sides, solved together
    meshes = [wl.box_mesh((2, 1, 1), W=3), wl.box_mesh((1, 2, 2), W=4)]
    batch = wl.concat_meshes(meshes)
    p1 = wl.poisson_sine(n=1, W=3)
    pb = wl.Problem(batch, [p1.f[0], lambda x, y, z: 2 * p1.f[0](x, y, z)], [wl._zero, wl._zero])
    mesh = api.Mesh(batch, n_rhs=2, coef_kind=api.COEF_LAPLACE)
    mesh.set_data(**api.problem_data_arrays(mesh, pb))
    x, rep = _solve(api, mesh, api.FP32)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-10
    x = x.reshape(2, -1)
    assert np.allclose(x[1], 2 * x[0], rtol=1e-7, atol=1e-9 * np.abs(x[1]).max())
    x64, _ = _solve(api, mesh, api.FP64)
    x64 = x64.reshape(2, -1)
    for r in range(2):
        d = Discretisation(wl.Problem(batch, [pb.f[r]], [wl._zero]))
        assert h1_rel_diff(d, x[r], x64[r]) <= 1e-8


def test_iteration_cap_reports_no_convergence(api):
    pb = wl.poisson_sine(n=2, W=4)
    mesh = _mesh(api, pb)
    x = torch.zeros(mesh.ndof, dtype=torch.float64, device="cuda")
    rep = mesh.pcg_solve(x, tol=1e-14, prec=api.FP64, max_iter=4, check_every=2, raise_on_error=False)
    assert rep["status"] == 5  # HPSE_ERR_NO_CONVERGENCE


@pytest.mark.parametrize("mode,delta", [(0, 1e-1), (0, 1e-3), (1, 1e-4)])
def test_refinement_modes(api, mode, delta):
    pb = wl.varcoef_manufactured(n=(2, 2, 2), W=4)
    mesh = _mesh(api, pb)
    disc = Discretisation(pb)
    x64, _ = _solve(api, mesh, api.FP64)
    xm, rep = _solve(api, mesh, api.FP32, refine_mode=mode, inner_tol=delta)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-10, rep
    assert h1_rel_diff(disc, xm, x64) <= 1e-8


def test_set_data_twice_then_solve(api):
    # new data on an existing handle must invalidate every captured solver graph
    pb = wl.varcoef_manufactured(n=(2, 2, 1), W=4)
    mesh = _mesh(api, pb)
    _solve(api, mesh, api.FP32)
    _solve(api, mesh, api.FP64)
    f2 = lambda xs, ys, zs: 3.0 * pb.f[0](xs, ys, zs)
    pb2 = wl.Problem(pb.mesh, [f2], pb.g, pb.a, pb.grad_a)
    mesh.set_data(**api.problem_data_arrays(mesh, pb2))
    disc2 = Discretisation(pb2)
    for prec in (api.FP32, api.FP64):
        x, rep = _solve(api, mesh, prec)
        assert rep["status"] == 0 and rep["rel_residual"] <= 1e-10
        xo, _, _ = pcg(disc2.apply_A, lambda r: apply_Cinv(disc2, r), disc2.rhs_b(), tol=1e-10)
        assert h1_rel_diff(disc2, x, xo) <= 1e-8

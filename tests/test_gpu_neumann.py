"""Neumann and Robin faces on the GPU (eq. 2.1, the last sum of eq. 4.2) for box
meshes of the Laplacian, against the oracle.

* Operator apply (FP64 1e-12, FP32 2e-5 of max|y|) and right-hand side
  (1e-12) of Table 6.3's mixed problem (Dirichlet on x = -1, x = 1, y = -1,
  Neumann on y = 1, z = +-1) and of the same problem with Robin faces
  (du/dnu + gamma u = h, gamma = 0.7), several right-hand sides;
* the GPU solution against the oracle's dense solution (the oracle's own
  residual and the kappa(A) bound, as for the other solution tests);
* Table 6.3's relative H^1 error from GPU solutions at W = 2, 4 within 5x of
  the table (the oracle's own pin) and decaying;
* the conforming correction leaves the Neumann faces free (parity with the
  oracle's correction, which also does).
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.conforming import conforming_correction
from oracle.functional import Discretisation
from oracle.h1 import h1_error_exact

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53


@pytest.fixture(scope="module")
def api():
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api as A
    return A


def _problem(kind, W, n_rhs=1):
    pb = wl.poisson_mixed(n=2, W=W)
    if kind == "robin":
        pb.mesh.elem_bc = np.where(pb.mesh.elem_bc == 1, 2, 0).astype(np.int32)
        pb.robin_gamma = 0.7
    if n_rhs > 1:
        pb = wl.Problem(pb.mesh, pb.f * n_rhs, pb.g * n_rhs, None, None, pb.u_exact * n_rhs,
                        pb.grad_u_exact * n_rhs, flux=pb.flux * n_rhs, robin_gamma=pb.robin_gamma)
    return pb


def _mesh(api, pb):
    m = api.Mesh(pb.mesh, n_rhs=pb.n_rhs, coef_kind=api.COEF_LAPLACE, robin_gamma=pb.robin_gamma)
    m.set_data(**api.problem_data_arrays(m, pb))
    return m


@pytest.mark.parametrize("kind", ["neumann", "robin"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_mixed_apply_matches_oracle(api, kind, prec, tol):
    pb = _problem(kind, 3)
    d = Discretisation(pb)
    m = _mesh(api, pb)
    U = wl.random_dofs(d.ndof, seed=13)
    ref = d.apply_A(U)
    dt = torch.float64 if prec == "fp64" else torch.float32
    u = torch.tensor(U, dtype=dt, device="cuda")
    y = torch.empty_like(u)
    m.apply_operator(u, y)
    got = y.double().cpu().numpy()
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    m.close()


@pytest.mark.parametrize("kind", ["neumann", "robin"])
def test_mixed_rhs_matches_oracle(api, kind):
    pb = _problem(kind, 4, n_rhs=2)
    d = Discretisation(pb)
    m = _mesh(api, pb)
    b = torch.empty(2 * m.ndof, dtype=torch.float64, device="cuda")
    m.get_rhs(b)
    b = b.cpu().numpy().reshape(2, m.ndof)
    for r in range(2):
        ref = d.rhs_b(r)
        assert np.abs(b[r] - ref).max() <= 1e-12 * np.abs(ref).max(), r
    m.close()


@pytest.mark.parametrize("kind", ["neumann", "robin"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mixed_solve_matches_oracle(api, kind, prec):
    pb = _problem(kind, 2)
    d = Discretisation(pb)
    A = d.dense_A()
    b = d.rhs_b()
    xo = np.linalg.solve(A, b)
    m = _mesh(api, pb)
    m.setup_block_preconditioner()
    x = torch.zeros(m.ndof, dtype=torch.float64, device="cuda")
    rep = m.pcg_solve(x, tol=1e-11, prec=api.FP64 if prec == "fp64" else api.FP32, max_iter=200000)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-11
    kA = np.linalg.cond(A)
    assert kA * 2e-11 <= 2e-6, kA
    X = x.cpu().numpy()
    res = np.linalg.norm(b - A @ X) / np.linalg.norm(b)
    assert res <= 1.5e-11 + 32 * EPS64 * np.linalg.norm(A, 2) * np.linalg.norm(X) / np.linalg.norm(b), res
    assert np.linalg.norm(X - xo) <= kA * 2e-11 * np.linalg.norm(xo), kA
    m.close()


def test_table_6_3_h1_error_from_gpu_solutions(api):
    from golden_tables import rel_error
    errs = {}
    for W in (2, 4):
        pb = _problem("neumann", W)
        d = Discretisation(pb)
        m = _mesh(api, pb)
        m.setup_block_preconditioner()
        x = torch.zeros(m.ndof, dtype=torch.float64, device="cuda")
        assert m.pcg_solve(x, tol=1e-12, prec=api.FP32, max_iter=200000)["status"] == 0
        errs[W] = h1_error_exact(d, x.cpu().numpy())
        ref = rel_error("table6_3_poisson_mixed.txt", W)
        assert ref / 5 < errs[W] < ref * 5, (W, errs[W], ref)
        m.close()
    assert errs[4] < 0.2 * errs[2], errs


def test_conforming_correction_with_neumann_faces(api):
    pb = _problem("neumann", 3)
    d = Discretisation(pb)
    m = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_LAPLACE)
    U = np.random.default_rng(21).standard_normal(d.ndof)
    p = torch.empty(d.ndof, dtype=torch.float64, device="cuda")
    m.conforming_correction(torch.tensor(U, device="cuda"), p)
    ref = conforming_correction(d, U)
    assert np.abs(p.cpu().numpy() - ref).max() <= 1e-14 * np.abs(ref).max()
    m.close()

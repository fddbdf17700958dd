"""GPU parity: operator apply, preconditioner and right-hand side vs the CPU oracle.

Tolerances:
* FP64: max |y_gpu - y_oracle| <= 1e-12 * max |y_oracle|, the bound fixed for
  FP64 operator applies (the two sides sum the same terms in different orders:
  about sqrt(n) eps64 growth over n ~ 10^3 terms, well inside 1e-12);
* FP32: max |y_gpu - y_oracle| <= 2e-5 * max |y_oracle| at W <= 8: the FP32
  unit roundoff 6e-8 amplified by the second-derivative matrices, whose
  entries grow like W^4 and cancel inside the sum factorisation, so that
  y carries a few hundred unit roundoffs of its largest terms.
All inputs are seeded; every call goes through the C ABI.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.functional import Discretisation
from oracle.precond import apply_Cinv

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


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


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _apply(mesh, U, dtype):
    u = torch.tensor(U, dtype=dtype, device="cuda")
    y = torch.full_like(u, float("nan"))
    mesh.apply_operator(u, y)
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


CASES = {
    "poisson_2x2x2_W4": lambda: wl.poisson_sine(n=2, W=4),
    "varcoef_3x2x2_W5": lambda: wl.varcoef_manufactured(n=(3, 2, 2), W=5),
    "laplace_sinh_1x2x3_W3": lambda: wl.laplace_sinh(n=(1, 2, 3), W=3),
    "single_element_W6": lambda: wl.poisson_sine(n=1, W=6),
    "varcoef_ragged_5x1x2_W2": lambda: wl.varcoef_manufactured(n=(5, 1, 2), W=2),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_apply_fp64_matches_oracle(api, name):
    pb = CASES[name]()
    mesh = _mesh(api, pb)
    disc = Discretisation(pb)
    U = wl.random_dofs(mesh.ndof, seed=11)
    ref = disc.apply_A(U)
    got = _apply(mesh, U, torch.float64)
    assert _rel(got, ref) <= TOL64, _rel(got, ref)


@pytest.mark.parametrize("W", list(range(1, 11)))
@pytest.mark.parametrize("coef", ["laplace", "scalar"])
def test_apply_every_degree(api, W, coef):
    n = (2, 1, 1) if W > 6 else (2, 2, 1)
    pb = wl.poisson_sine(n=n, W=W) if coef == "laplace" else wl.varcoef_manufactured(n=n, W=W)
    mesh = _mesh(api, pb)
    disc = Discretisation(pb)
    U = wl.random_dofs(mesh.ndof, seed=100 + W)
    ref = disc.apply_A(U)
    got = _apply(mesh, U, torch.float64)
    assert _rel(got, ref) <= TOL64, (W, _rel(got, ref))
    got32 = _apply(mesh, U, torch.float32)
    tol32 = TOL32 if W <= 8 else 1e-4
    assert _rel(got32, ref) <= tol32, (W, _rel(got32, ref))


def test_apply_multiple_rhs(api):
    pb = wl.varcoef_manufactured(n=(2, 2, 1), W=3)
    mesh = _mesh(api, wl.Problem(pb.mesh, pb.f * 3, pb.g * 3, pb.a, pb.grad_a), n_rhs=3)
    disc = Discretisation(pb)
    U = wl.random_dofs(3 * mesh.ndof, seed=5).reshape(3, mesh.ndof)
    got = _apply(mesh, U.ravel(), torch.float64).reshape(3, -1)
    for r in range(3):
        assert _rel(got[r], disc.apply_A(U[r])) <= TOL64


def test_apply_uneven_degree_batch(api):
    # three independent problems of degrees 2, 5 and 3 in one handle
    meshes = [wl.box_mesh((2, 1, 1), W=2), wl.box_mesh((1, 2, 1), W=5), wl.box_mesh((1, 1, 2), W=3)]
    batch = wl.concat_meshes(meshes)
    pb = wl.Problem(batch, [wl._zero], [wl._zero])
    mesh = _mesh(api, pb)
    disc = Discretisation(pb)
    U = wl.random_dofs(mesh.ndof, seed=9)
    assert _rel(_apply(mesh, U, torch.float64), disc.apply_A(U)) <= TOL64


@pytest.mark.parametrize("W", [1, 4, 8, 10])
def test_preconditioner_matches_oracle(api, W):
    pb = wl.poisson_sine(n=(2, 1, 1), W=W)
    mesh = _mesh(api, pb)
    disc = Discretisation(pb)
    R = wl.random_dofs(mesh.ndof, seed=W)
    r = torch.tensor(R, device="cuda")
    z = torch.empty_like(r)
    mesh.apply_preconditioner(r, z)
    zr = apply_Cinv(disc, R)
    # C^{-1} has condition number kappa_C = 3 mu_max + 1 (eq. 5.20); two
    # independent eigendecompositions agree to O(eps kappa_C)
    from oracle.precond import eigenbasis
    kappa_C = 3 * eigenbasis(W)[0].max() + 1
    tol = max(TOL64, 4 * np.finfo(np.float64).eps * kappa_C)
    assert _rel(z.cpu().numpy(), zr) <= tol, (_rel(z.cpu().numpy(), zr), tol)
    r32 = r.float()
    z32 = torch.empty_like(r32)
    mesh.apply_preconditioner(r32, z32)
    assert _rel(z32.double().cpu().numpy(), zr) <= 1e-4


@pytest.mark.parametrize("name", ["laplace_sinh_1x2x3_W3", "varcoef_3x2x2_W5", "poisson_2x2x2_W4"])
def test_rhs_matches_oracle(api, name):
    pb = CASES[name]()
    mesh = _mesh(api, pb)
    disc = Discretisation(pb)
    b = torch.empty(mesh.ndof, dtype=torch.float64, device="cuda")
    mesh.get_rhs(b)
    torch.cuda.synchronize()
    assert _rel(b.cpu().numpy(), disc.rhs_b()) <= TOL64


def test_deterministic_bitwise(api):
    pb = wl.varcoef_manufactured(n=(2, 2, 2), W=4)
    mesh = _mesh(api, pb)
    U = wl.random_dofs(mesh.ndof, seed=3)
    a = _apply(mesh, U, torch.float64)
    b = _apply(mesh, U, torch.float64)
    assert np.array_equal(a, b)

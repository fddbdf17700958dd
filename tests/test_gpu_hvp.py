"""Hessian-vector products of a solution functional on the GPU (the
second-order adjoint through autograd.Solve's differentiable backward), and
the library pieces they use.

* hpse_apply_fields_transpose is the transpose of hpse_eval_fields:
  <F u, w> = <u, F^T w> for random u, w (1e-12), several degrees.
* hpse_data_gradient_vjp is the derivative of hpse_data_gradient: its
  contraction with a direction equals the central difference of the data
  gradient in u-fields, lambda-fields and data (the formulas are polynomial of
  degree 2 in the inputs, so the central difference is exact up to rounding).
* The GPU Hessian-vector product of J(theta) = sum_q wJ (u_h - u_t)^2 with
  respect to (f, a, grad a) at the points, along a random direction, against
  the oracle's (central differences of its exact dense adjoint gradient) within
  1e-6 (solves to 1e-12), and the symmetry w^T H v = v^T H w of the GPU
  products within 1e-8.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.adjoint import DenseAdjoint, point_data
from oracle.functional import Discretisation

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api as A
    return A


def _mesh(api, pb):
    m = api.Mesh(pb.mesh, n_rhs=pb.n_rhs, coef_kind=api.COEF_SCALAR)
    m.set_data(**api.problem_data_arrays(m, pb))
    return m


@pytest.mark.parametrize("W", [2, 5, 9])
def test_fields_transpose_is_the_adjoint_of_fields(api, W):
    pb = wl.varcoef_manufactured(n=(2, 1, 1), W=W)
    m = _mesh(api, pb)
    rng = np.random.default_rng(W)
    u = torch.tensor(rng.standard_normal(m.ndof), device="cuda")
    wf = torch.tensor(rng.standard_normal((1, 5, m.nquad)), device="cuda")
    F = torch.empty(1, 5, m.nquad, dtype=torch.float64, device="cuda")
    m.eval_fields(u, F)
    y = torch.empty_like(u)
    m.apply_fields_transpose(wf, y)
    lhs, rhs = float((F * wf).sum()), float((u * y).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), float(F.abs().sum()))
    m.close()


def test_data_gradient_vjp_against_differences(api):
    pb = wl.varcoef_manufactured(n=(2, 1, 1), W=3)
    m = _mesh(api, pb)
    rng = np.random.default_rng(2)
    R, nq = 1, m.nquad
    uf = torch.tensor(rng.standard_normal((R, 5, nq)), device="cuda")
    lf = torch.tensor(rng.standard_normal((R, 5, nq)), device="cuda")
    ob = torch.tensor(rng.standard_normal((R, 5, nq)), device="cuda")
    du = torch.tensor(rng.standard_normal((R, 5, nq)), device="cuda")
    dl = torch.tensor(rng.standard_normal((R, 5, nq)), device="cuda")
    for with_f in (True, False):
        ub, lb, db = torch.empty_like(uf), torch.empty_like(uf), torch.empty_like(uf)
        m.data_gradient_vjp(with_f, uf, lf, ob, ub, lb, db)

        def G(u, l):
            out = torch.empty_like(uf)
            (m.data_gradient if with_f else m.data_gradient_bilinear)(u, l, out)
            return out
        h = 1e-3
        fd = ((G(uf + h * du, lf + h * dl) - G(uf - h * du, lf - h * dl)) * ob).sum() / (2 * h)
        lin = (ub * du).sum() + (lb * dl).sum()
        assert abs(float(fd - lin)) <= 1e-10 * float(abs(fd) + 1.0), with_f
    m.close()


def _target(disc):
    out = []
    for e in range(disc.E):
        x, y, z = wl._grid(*disc.qpoints(e))
        out.append((np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)).ravel())
    return np.concatenate(out)


def test_hessian_vector_product_matches_oracle(api):
    from paper_1110_2316_gb300.autograd import PointValues, Solve
    pb = wl.varcoef_manufactured(n=(2, 1, 1), W=2)
    disc = Discretisation(pb)
    m = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_SCALAR)
    d = api.problem_data_arrays(m, pb)
    ut_np = _target(disc)
    ut = torch.tensor(ut_np, device="cuda")
    w = torch.empty(m.nquad, dtype=torch.float64, device="cuda")
    theta = [torch.tensor(d["f"], device="cuda", requires_grad=True),
             torch.tensor(d["a"], device="cuda", requires_grad=True),
             torch.tensor(d["grad_a"], device="cuda", requires_grad=True)]
    rng = np.random.default_rng(6)
    nq = m.nquad
    vs = [(rng.standard_normal((1, nq)), 0.1 * rng.standard_normal(nq), 0.1 * rng.standard_normal((3, nq)))
          for _ in range(2)]
    u = Solve.apply(*theta, m, d["g"], 1e-12)
    m.quad_weights(w)
    J = (w * (PointValues.apply(u, m)[0] - ut) ** 2).sum()
    g = torch.autograd.grad(J, theta, create_graph=True)
    Hv = []
    for v in vs:
        vt = [torch.tensor(x, device="cuda") for x in v]
        s = sum((gi * vi).sum() for gi, vi in zip(g, vt))
        Hv.append([h.detach().cpu().numpy() for h in torch.autograd.grad(s, theta, retain_graph=True)])
    # the oracle: central differences of its exact dense adjoint gradient
    dn = DenseAdjoint(disc, ut_np)
    th0 = point_data(disc)
    ref = dn.hessian_vector(*th0, (vs[0][0][0], vs[0][1], vs[0][2]), 1e-4)
    got = (Hv[0][0][0], Hv[0][1], Hv[0][2])
    for k, (x, r) in enumerate(zip(got, ref)):
        err = np.abs(x - r).max() / np.abs(r).max()
        print("H v component", k, "rel err", err)
        assert err <= 1e-6, (k, err)
    # symmetry of the GPU products
    wHv = sum(float(np.sum(a * b)) for a, b in zip(vs[1], Hv[0]))
    vHw = sum(float(np.sum(a * b)) for a, b in zip(vs[0], Hv[1]))
    assert abs(wHv - vHw) <= 1e-8 * max(abs(wHv), 1e-30), (wHv, vHw)
    m.close()

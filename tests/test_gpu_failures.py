"""Failure paths of the library, each caused on the host (no device fault):

* a right-hand side holding a NaN -> HPSE_ERR_BREAKDOWN from hpse_pcg_solve
  (FP64 and mixed), and the handle still solves the next, finite problem;
* a coefficient a <= 0 or non-finite -> HPSE_ERR_INVALID_ARG from
  hpse_set_data (the operator of eq. 2.1 must be elliptic), and the handle
  still accepts valid data afterwards;
* a wall-clock limit far below one solve -> HPSE_ERR_TIMEOUT, with the handle
  usable for the next solve;
* autograd.Solve.backward after the mesh was given other data: the gradient
  is that of the forward solve's data.
"""
import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu

BREAKDOWN, INVALID_ARG, TIMEOUT = 4, 1, 6


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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("refine_mode", [0, 1])
def test_nan_rhs_is_breakdown(api, prec, refine_mode):
    if prec == "fp64" and refine_mode == 1:
        pytest.skip("restarted refinement is a mixed-precision mode")
    m = _mesh(api, wl.poisson_sine(n=2, W=3))
    P = api.FP64 if prec == "fp64" else api.FP32
    b = torch.empty(m.ndof, dtype=torch.float64, device="cuda")
    m.get_rhs(b)
    bad = b.clone()
    bad[m.ndof // 3] = float("nan")
    m.set_rhs(bad)
    x = torch.zeros_like(b)
    rep = m.pcg_solve(x, tol=1e-10, prec=P, refine_mode=refine_mode, raise_on_error=False)
    assert rep["status"] == BREAKDOWN, rep
    with pytest.raises(api._lib.HpseError):
        m.pcg_solve(x, tol=1e-10, prec=P, refine_mode=refine_mode)
    # the handle is intact: the finite problem still solves
    m.set_rhs(b)
    x.zero_()
    rep = m.pcg_solve(x, tol=1e-10, prec=P, refine_mode=refine_mode)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-10
    assert torch.isfinite(x).all()
    m.close()


@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan"), float("inf")])
def test_nonpositive_coefficient_is_invalid_arg(api, bad):
    pb = wl.varcoef_manufactured(n=(2, 1, 1), W=3)
    m = _mesh(api, pb)
    d = api.problem_data_arrays(m, pb)
    a = d["a"].copy()
    a[a.size // 2] = bad
    with pytest.raises(api._lib.HpseError) as ei:
        m.set_data(f=d["f"], a=a, grad_a=d["grad_a"], g=d["g"])
    assert ei.value.status == INVALID_ARG
    m.set_data(**d)
    x = torch.zeros(m.ndof, dtype=torch.float64, device="cuda")
    rep = m.pcg_solve(x, tol=1e-10, prec=api.FP64)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-10
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_time_limit_is_timeout(api, prec):
    # the separable preconditioner on W = 6 needs far more than one graph
    # replay (16 iterations); a 1 ns limit stops the solve at the first check
    pb = wl.varcoef_manufactured(n=(2, 2, 2), W=6)
    m = _mesh(api, pb)
    P = api.FP64 if prec == "fp64" else api.FP32
    x = torch.zeros(m.ndof, dtype=torch.float64, device="cuda")
    rep = m.pcg_solve(x, tol=1e-10, prec=P, time_limit_s=1e-9, raise_on_error=False)
    assert rep["status"] == TIMEOUT, rep
    assert rep["rel_residual"] > 1e-10 and np.isfinite(rep["rel_residual"])
    x.zero_()
    rep = m.pcg_solve(x, tol=1e-10, prec=P)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-10
    m.close()


def test_solve_backward_uses_forward_data(api):
    from paper_1110_2316_gb300.autograd import PointValues, Solve
    pb = wl.varcoef_manufactured(n=(2, 1, 1), W=3)
    m = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_SCALAR)
    d = api.problem_data_arrays(m, pb)
    w = torch.empty(m.nquad, dtype=torch.float64, device="cuda")

    def grads(disturb):
        f = torch.tensor(d["f"], device="cuda", requires_grad=True)
        a = torch.tensor(d["a"], device="cuda", requires_grad=True)
        ga = torch.tensor(d["grad_a"], device="cuda", requires_grad=True)
        u = Solve.apply(f, a, ga, m, d["g"], 1e-12)
        m.quad_weights(w)
        J = (w * PointValues.apply(u, m)[0] ** 2).sum()
        if disturb:
            # another problem on the same handle between forward and backward
            m.set_data(f=2.0 * d["f"], a=3.0 * d["a"], grad_a=3.0 * d["grad_a"], g=d["g"])
        J.backward()
        return f.grad.clone(), a.grad.clone(), ga.grad.clone()

    ref = grads(False)
    got = grads(True)
    for r, g in zip(ref, got):
        assert float((g - r).abs().max()) <= 1e-9 * float(r.abs().max())
    m.close()

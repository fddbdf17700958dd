"""hpse_set_data with device data and a stream, and the FP32 residual map.

* Data given as CUDA tensors (read on a side stream) build the same right-hand
  side b, operator and solution as the same data given from the host: the
  coefficient transform runs in a kernel with the host's FP64 formulas, so b
  agrees to 1e-14 relative and the FP64 apply to the last bit.
* A coefficient a <= 0 in device data: HPSE_ERR_INVALID_ARG, after which the
  handle has no data (a solve reports HPSE_ERR_NO_DATA) until valid data is set.
* Host and device arrays mixed in one call: HPSE_ERR_INVALID_ARG.
* hpse_apply_residual / hpse_apply_transpose in FP32 against FP64, for
  -div(a grad u) and the Laplacian: 1e-5 of the largest value (FP32 unit roundoff 6e-8 times the O(W^4) second-derivative
  entries at W <= 4), and the transposition identity <S u, z> = <u, S^T z> in
  FP32 to 1e-5 of |S u| |z|.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu

INVALID_ARG, NO_DATA = 1, 9


@pytest.fixture(scope="module")
def api():
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api as A
    return A


def _dev(d):
    return {k: (None if v is None else torch.tensor(v, device="cuda")) for k, v in d.items()}


@pytest.mark.parametrize("case", ["varcoef", "laplace_dirichlet", "edge"])
def test_device_data_equals_host_data(api, case):
    if case == "varcoef":
        pb = wl.varcoef_manufactured(n=(2, 2, 1), W=4)
        kind, n_rhs = api.COEF_SCALAR, 1
    elif case == "laplace_dirichlet":
        base = wl.laplace_sinh(n=(1, 2, 2), W=3)
        pb = wl.Problem(base.mesh, base.f * 2, base.g * 2, None, None, base.u_exact * 2, base.grad_u_exact * 2)
        kind, n_rhs = api.COEF_LAPLACE, 2
    else:
        pb = wl.edge_laplace_singular(N=3, W=3)
        kind, n_rhs = api.COEF_LAPLACE, 1
    mh = api.Mesh(pb.mesh, n_rhs=n_rhs, coef_kind=kind)
    md = api.Mesh(pb.mesh, n_rhs=n_rhs, coef_kind=kind)
    data = api.problem_data_arrays(mh, pb)
    mh.set_data(**data)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        dd = _dev(data)
        md.set_data(**dd, stream=side.cuda_stream)
    torch.cuda.synchronize()
    n = n_rhs * mh.ndof
    bh = torch.empty(n, dtype=torch.float64, device="cuda")
    bd = torch.empty_like(bh)
    mh.get_rhs(bh)
    md.get_rhs(bd)
    assert float((bh - bd).abs().max()) <= 1e-14 * float(bh.abs().max())
    u = torch.tensor(wl.random_dofs(n, seed=5), device="cuda")
    yh, yd = torch.empty_like(u), torch.empty_like(u)
    mh.apply_operator(u, yh)
    md.apply_operator(u, yd)
    assert torch.equal(yh, yd)
    xh, xd = torch.zeros_like(u), torch.zeros_like(u)
    assert mh.pcg_solve(xh, tol=1e-11, prec=api.FP64, max_iter=200000)["status"] == 0
    assert md.pcg_solve(xd, tol=1e-11, prec=api.FP64, max_iter=200000)["status"] == 0
    assert float((xh - xd).abs().max()) <= 1e-12 * float(xh.abs().max())
    mh.close()
    md.close()


def test_device_data_rejects_nonpositive_coefficient(api):
    pb = wl.varcoef_manufactured(n=(2, 1, 1), W=3)
    m = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_SCALAR)
    data = api.problem_data_arrays(m, pb)
    dd = _dev(data)
    bad = dd["a"].clone()
    bad[bad.numel() // 3] = -0.5
    with pytest.raises(api._lib.HpseError) as ei:
        m.set_data(f=dd["f"], a=bad, grad_a=dd["grad_a"], g=dd["g"])
    assert ei.value.status == INVALID_ARG
    x = torch.zeros(m.ndof, dtype=torch.float64, device="cuda")
    rep_status = None
    try:
        m.pcg_solve(x, tol=1e-10, prec=api.FP64)
    except api._lib.HpseError as err:
        rep_status = err.status
    assert rep_status == NO_DATA
    m.set_data(**dd)
    x.zero_()
    rep = m.pcg_solve(x, tol=1e-10, prec=api.FP64)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-10
    m.close()


def test_mixed_host_and_device_data_rejected(api):
    pb = wl.varcoef_manufactured(n=(2, 1, 1), W=2)
    m = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_SCALAR)
    data = api.problem_data_arrays(m, pb)
    with pytest.raises(TypeError):
        m.set_data(f=torch.tensor(data["f"], device="cuda"), a=data["a"], grad_a=data["grad_a"], g=data["g"])
    # the same through the C ABI: f on the device, a and grad a on the host
    from paper_1110_2316_gb300 import _lib
    f = torch.tensor(data["f"], device="cuda")
    a = np.ascontiguousarray(data["a"])
    ga = np.ascontiguousarray(data["grad_a"])
    d = _lib.Data(C.c_void_p(f.data_ptr()), a.ctypes.data_as(C.c_void_p), ga.ctypes.data_as(C.c_void_p), None)
    assert _lib.load().hpse_set_data(m._h, C.byref(d), None) == INVALID_ARG
    m.close()


@pytest.mark.parametrize("W", [2, 4])
@pytest.mark.parametrize("coef", ["scalar", "laplace"])
def test_fp32_residual_and_transpose(api, W, coef):
    if coef == "scalar":
        pb = wl.varcoef_manufactured(n=(2, 1, 2), W=W)
        m = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_SCALAR)
    else:
        pb = wl.poisson_sine(n=(2, 1, 2), W=W)
        m = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_LAPLACE)
    m.set_data(**api.problem_data_arrays(m, pb))
    u64 = torch.tensor(wl.random_dofs(m.ndof, seed=W), device="cuda")
    u32 = u64.float()
    z64 = torch.empty(1, m.nquad, dtype=torch.float64, device="cuda")
    z32 = torch.empty(1, m.nquad, dtype=torch.float32, device="cuda")
    m.apply_residual(u32.double(), z64)
    m.apply_residual(u32, z32)
    assert float((z32.double() - z64).abs().max()) <= 1e-5 * float(z64.abs().max())
    g = torch.tensor(np.random.default_rng(W).standard_normal(m.nquad), device="cuda").reshape(1, -1)
    y64 = torch.empty(m.ndof, dtype=torch.float64, device="cuda")
    y32 = torch.empty(m.ndof, dtype=torch.float32, device="cuda")
    m.apply_transpose(g.float().double(), y64)
    m.apply_transpose(g.float(), y32)
    assert float((y32.double() - y64).abs().max()) <= 1e-5 * float(y64.abs().max())
    # transposition identity of the FP32 pair (the data term f drops out of
    # the difference of two residuals)
    zero = torch.zeros_like(u32)
    z0 = torch.empty_like(z32)
    m.apply_residual(zero, z0)
    su = (z32 - z0).double()
    lhs = float((su * g).sum())
    rhs = float((u32.double() * y32.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * float(su.norm() * g.norm())
    m.close()

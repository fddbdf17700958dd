"""torch.autograd wrappers over the C ABI (argument marshalling only).

* ``ResidualMap``: u -> z = sqrt(w J)(L u - f) at the volume points (the
  weighted PDE residual of eq. (4.2), Section 5.3), FP64 or FP32 after u's
  dtype; backward = the hand-written transpose kernel (hpse_apply_transpose).
* ``PointValues``: u -> u(x_q) at the volume points; backward = the transpose
  of point evaluation (hpse_apply_eval_transpose), itself differentiable.
* ``Fields``: u -> (v, grad v, Lap v) at the volume points; backward = their
  transpose (hpse_apply_fields_transpose).
* ``Solve``: the data (f, a, grad a at the volume points; Dirichlet data g
  on the boundary-face points, not differentiated) -> the solution u of the
  normal equations.  Backward: the adjoint state lambda solves
  A lambda = dJ/du by PCG (recomputed, no iterate is stored; A is symmetric),
  and hpse_data_gradient returns dJ/df, dJ/da, dJ/d(grad a) at the points.
  The adjoint right-hand side of a solution functional lies mostly in the
  low end of A's spectrum, so its attainable relative residual is about
  eps kappa(A), above that of the forward solve: ``adjoint_tol`` (default:
  the forward ``tol``) sets it separately, and an adjoint solve that stops at
  its attainable level within 10x of it is accepted (and logged).  Backward works on the data of
  its own forward solve: if the mesh has been given other data in between,
  that solve's data is set again first (the mesh then keeps it).
  The backward is made of differentiable functions (``AdjointSolve``,
  ``Fields``, ``DataGrad`` with hpse_data_gradient_vjp as its backward), so
  differentiating the gradient again gives Hessian-vector products by the
  second-order adjoint: the tangent of the solution and of the adjoint state
  each cost one more solve with A.

All tensors are CUDA float64 tensors (ResidualMap: float64 or float32); shapes: u [n_rhs * ndof], z and f
[n_rhs, nquad], a [nquad], grad_a [3, nquad].
"""
from __future__ import annotations

import torch

from .api import FP64


def _data(t, like=None):
    """A datum for Mesh.set_data: CUDA tensors stay on the device; host arrays
    given beside device data (Dirichlet data g) are moved to f's device."""
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return t.detach()
    if like is not None and isinstance(like, torch.Tensor) and like.is_cuda:
        return torch.as_tensor(t, dtype=torch.float64, device=like.device)
    return t


class ResidualMap(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, mesh):
        z = torch.empty(mesh.n_rhs, mesh.nquad, dtype=u.dtype, device=u.device)
        mesh.apply_residual(u.contiguous(), z)
        ctx.mesh = mesh
        return z

    @staticmethod
    def backward(ctx, gz):
        m = ctx.mesh
        y = torch.empty(m.n_rhs * m.ndof, dtype=gz.dtype, device=gz.device)
        m.apply_transpose(gz.contiguous(), y)
        return y, None


class PointValues(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, mesh):
        f = torch.empty(mesh.n_rhs, 5, mesh.nquad, dtype=torch.float64, device=u.device)
        mesh.eval_fields(u.contiguous(), f)
        ctx.mesh = mesh
        return f[:, 0, :].contiguous()

    @staticmethod
    def backward(ctx, gv):
        return PointValuesT.apply(gv, ctx.mesh), None


class PointValuesT(torch.autograd.Function):
    """rho -> sum_q rho_q dv(x_q)/dV, the transpose of PointValues (its backward)."""

    @staticmethod
    def forward(ctx, rho, mesh):
        y = torch.empty(mesh.n_rhs * mesh.ndof, dtype=torch.float64, device=rho.device)
        mesh.apply_eval_transpose(rho.contiguous(), y)
        ctx.mesh = mesh
        return y

    @staticmethod
    def backward(ctx, gy):
        return PointValues.apply(gy, ctx.mesh), None


class Fields(torch.autograd.Function):
    """u -> (v, v_x, v_y, v_z, Lap v) at the volume points, [n_rhs, 5, nquad]."""

    @staticmethod
    def forward(ctx, u, mesh):
        f = torch.empty(mesh.n_rhs, 5, mesh.nquad, dtype=torch.float64, device=u.device)
        mesh.eval_fields(u.contiguous(), f)
        ctx.mesh = mesh
        return f

    @staticmethod
    def backward(ctx, gf):
        return FieldsT.apply(gf, ctx.mesh), None


class FieldsT(torch.autograd.Function):
    """The transpose of Fields (its backward)."""

    @staticmethod
    def forward(ctx, wf, mesh):
        y = torch.empty(mesh.n_rhs * mesh.ndof, dtype=torch.float64, device=wf.device)
        mesh.apply_fields_transpose(wf.contiguous(), y)
        ctx.mesh = mesh
        return y

    @staticmethod
    def backward(ctx, gy):
        return Fields.apply(gy, ctx.mesh), None


class _DataRef:
    """The data of one forward solve, shared by the functions of its backward:
    restore() sets it on the mesh again if the mesh has been given other data
    since (once, for all of them)."""

    def __init__(self, mesh, data):
        self.mesh, self.data, self.version = mesh, data, mesh.data_version

    def restore(self):
        m = self.mesh
        if m.data_version != self.version:
            f, a, grad_a, g = self.data
            m.set_data(f=_data(f), a=_data(a), grad_a=_data(grad_a), g=_data(g, f))
            self.version = m.data_version


def _adjoint_solve(ref, rhs, tol, prec, tag):
    """lambda = A^{-1} rhs with the solve's data (A symmetric); b is kept."""
    ref.restore()
    m = ref.mesh
    b = torch.empty(m.n_rhs * m.ndof, dtype=torch.float64, device=rhs.device)
    m.get_rhs(b)
    m.set_rhs(rhs.contiguous())
    lam = torch.zeros_like(b)
    rep = m.pcg_solve(lam, tol=tol, prec=prec, raise_on_error=False)
    m.set_rhs(b)
    if isinstance(getattr(m, "solve_log", None), list):
        m.solve_log.append((tag, rep))
    # the adjoint right-hand side sits in the low end of A's spectrum: its
    # FP64-attainable residual (about eps kappa(A)) can lie just above the
    # requested tolerance; a solve that stopped there (within 10x) is kept
    if rep["status"] != 0 and not (rep["status"] == 5 and rep["rel_residual"] <= 10 * tol):
        from ._lib import HpseError
        raise HpseError(rep["status"], "adjoint hpse_pcg_solve")
    return lam


class DataGrad(torch.autograd.Function):
    """(fields of u, fields of lambda, f, a, grad a) -> the pointwise data
    gradient of hpse_data_gradient ([n_rhs, 5, nquad]; with_f = False: the
    bilinear form, f taken as 0).  f, a, grad a enter through the mesh's data
    (the solve's, restored if needed); backward: hpse_data_gradient_vjp."""

    @staticmethod
    def forward(ctx, uf, lf, f, a, grad_a, ref, with_f):
        ref.restore()
        out = torch.empty_like(uf)
        m = ref.mesh
        (m.data_gradient if with_f else m.data_gradient_bilinear)(uf.contiguous(), lf.contiguous(), out)
        ctx.ref, ctx.with_f = ref, with_f
        ctx.save_for_backward(uf, lf)
        return out

    @staticmethod
    def backward(ctx, go):
        uf, lf = ctx.saved_tensors
        ctx.ref.restore()
        ub, lb, db = torch.empty_like(uf), torch.empty_like(uf), torch.empty_like(uf)
        ctx.ref.mesh.data_gradient_vjp(ctx.with_f, uf, lf, go.contiguous(), ub, lb, db)
        need = ctx.needs_input_grad
        gf = db[:, 0, :] if (ctx.with_f and need[2]) else None
        ga = db[:, 1, :].sum(0) if need[3] else None
        gga = db[:, 2:5, :].sum(0) if need[4] else None
        return ub, lb, gf, ga, gga, None, None


class AdjointSolve(torch.autograd.Function):
    """rhs -> lambda = A(a)^{-1} rhs (A symmetric), differentiable in rhs and
    in the coefficient a, grad a: d lambda = A^{-1} (d rhs - dA lambda), so the
    backward solves A nu = lambda-bar once more and returns nu for rhs and
    hpse_data_gradient_bilinear(fields of nu, fields of lambda) for a, grad a."""

    @staticmethod
    def forward(ctx, rhs, f, a, grad_a, ref, tol, prec):
        lam = _adjoint_solve(ref, rhs, tol, prec, "adjoint")
        ctx.ref, ctx.tol, ctx.prec = ref, tol, prec
        ctx.save_for_backward(lam)
        return lam

    @staticmethod
    def backward(ctx, gl):
        (lam,) = ctx.saved_tensors
        ref = ctx.ref
        f, a, grad_a, _ = ref.data
        nu = AdjointSolve.apply(gl, f, a, grad_a, ref, ctx.tol, ctx.prec)
        need = ctx.needs_input_grad
        ga = gga = None
        if need[2] or need[3]:
            g = DataGrad.apply(Fields.apply(nu, ref.mesh), Fields.apply(lam, ref.mesh), f, a, grad_a, ref, False)
            ga = g[:, 1, :].sum(0) if need[2] else None
            gga = g[:, 2:5, :].sum(0) if need[3] else None
        return nu, None, ga, gga, None, None, None


class Solve(torch.autograd.Function):
    """u = A(a)^{-1} b(f, a) for the data sampled at the volume points.

    The backward is built from differentiable pieces (AdjointSolve, Fields,
    DataGrad), so a second differentiation of the gradient -- a
    Hessian-vector product of a solution functional, by the second-order
    adjoint (two more solves per product) -- runs through the same library
    calls (torch.autograd.grad with create_graph=True)."""

    @staticmethod
    def forward(ctx, f, a, grad_a, mesh, g=None, tol=1e-12, prec=FP64, adjoint_prec=FP64, adjoint_tol=None):
        mesh.set_data(f=_data(f), a=_data(a), grad_a=_data(grad_a), g=_data(g, f))
        x = torch.zeros(mesh.n_rhs * mesh.ndof, dtype=torch.float64, device=f.device)
        rep = mesh.pcg_solve(x, tol=tol, prec=prec)
        if isinstance(getattr(mesh, "solve_log", None), list):
            mesh.solve_log.append(("forward", rep))
        ctx.save_for_backward(x)
        # the data this solve used: backward restores it if the mesh has been
        # given other data since (another solve, a finite-difference probe)
        ctx.ref = _DataRef(mesh, (f, a, grad_a, g))
        ctx.adjoint_prec = adjoint_prec
        ctx.tol = tol if adjoint_tol is None else adjoint_tol
        ctx.has_a = a is not None
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        ref = ctx.ref
        m = ref.mesh
        f, a, grad_a, _ = ref.data
        lam = AdjointSolve.apply(gx, f, a, grad_a, ref, ctx.tol, ctx.adjoint_prec)
        G = DataGrad.apply(Fields.apply(x, m), Fields.apply(lam, m), f, a, grad_a, ref, True)
        gf = G[:, 0, :]
        ga = G[:, 1, :].sum(0) if ctx.has_a else None
        gga = G[:, 2:5, :].sum(0) if ctx.has_a else None
        return gf, ga, gga, None, None, None, None, None, None

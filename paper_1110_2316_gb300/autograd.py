"""torch.autograd wrappers over the C ABI (argument marshalling only).

* ``ResidualMap``: u -> z = sqrt(w J)(L u - f) at the volume points (the
  weighted PDE residual of eq. (4.2), Section 5.3), FP64 or FP32 after u's
  dtype; backward = the hand-written transpose kernel (hpse_apply_transpose).
* ``PointValues``: u -> u(x_q) at the volume points; backward = the transpose
  of point evaluation (hpse_apply_eval_transpose).
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
        m = ctx.mesh
        y = torch.empty(m.n_rhs * m.ndof, dtype=torch.float64, device=gv.device)
        m.apply_eval_transpose(gv.contiguous(), y)
        return y, None


class Solve(torch.autograd.Function):
    """u = A(a)^{-1} b(f, a) for the data sampled at the volume points."""

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
        ctx.data = (f, a, grad_a, g)
        ctx.data_version = mesh.data_version
        ctx.mesh, ctx.adjoint_prec = mesh, adjoint_prec
        ctx.tol = tol if adjoint_tol is None else adjoint_tol
        ctx.has_a = a is not None
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        m = ctx.mesh
        if m.data_version != ctx.data_version:
            # A(a) and b(f, a) of the forward solve, not of the mesh's current data
            f, a, grad_a, g = ctx.data
            m.set_data(f=_data(f), a=_data(a), grad_a=_data(grad_a), g=_data(g, f))
        b = torch.empty_like(x)
        m.get_rhs(b)
        m.set_rhs(gx.contiguous())
        lam = torch.zeros_like(x)
        rep = m.pcg_solve(lam, tol=ctx.tol, prec=ctx.adjoint_prec, raise_on_error=False)
        if isinstance(getattr(m, "solve_log", None), list):
            m.solve_log.append(("adjoint", rep))
        # the adjoint right-hand side sits in the low end of A's spectrum: its
        # FP64-attainable residual (about eps kappa(A)) can lie just above the
        # requested tolerance; a solve that stopped there (within 10x) is kept
        if rep["status"] != 0 and not (rep["status"] == 5 and rep["rel_residual"] <= 10 * ctx.tol):
            from ._lib import HpseError
            m.set_rhs(b)
            raise HpseError(rep["status"], "adjoint hpse_pcg_solve")
        m.set_rhs(b)
        uf = torch.empty(m.n_rhs, 5, m.nquad, dtype=torch.float64, device=x.device)
        lf = torch.empty_like(uf)
        m.eval_fields(x, uf)
        m.eval_fields(lam, lf)
        g = torch.empty_like(uf)
        m.data_gradient(uf, lf, g)
        gf = g[:, 0, :]
        ga = g[:, 1, :].sum(0) if ctx.has_a else None
        gga = g[:, 2:5, :].sum(0) if ctx.has_a else None
        return gf, ga, gga, None, None, None, None, None, None

"""Adjoint gradients of a solution functional (oracle, FP64).

Test infrastructure only (see the package docstring).

The discrete solution U of A(a) U = b(f, a) (normal equations of eq. 4.2,
Section 5.3) depends on the data sampled at the volume quadrature points: the
source f_q, the coefficient a_q and its gradient (grad a)_q.  For a functional
J(U) the adjoint state lambda solves A lambda = dJ/dU (A is symmetric) and

    dJ/dtheta = - lambda^T d(A U - b)/dtheta .

Only the volume term of eq. (4.2) depends on the data:
    R_vol = sum_q z_q^2,  z_q = sqrt(w_q J) (L U - f)_q,  L U = -a Lap U - grad a . grad U,
so, with L lambda the operator applied to lambda (no data),

    dJ/df_q         = w_q J (L lambda)_q
    dJ/da_q         = w_q J [ (Lap U)_q (L lambda)_q + (L U - f)_q (Lap lambda)_q ]
    dJ/d(d_k a)_q   = w_q J [ (d_k U)_q (L lambda)_q + (L U - f)_q (d_k lambda)_q ]

Each line is the derivative of -lambda^T sum_q z_q dz_q/dU with respect to that
datum, written out; the tests check it against finite differences of J.
The functional used is J(U) = sum_e sum_q w_q J_e (u_h - u_t)^2 (the element
(2W+1)^3 GLL rule), whose gradient is dJ/dU = 2 sum_q w_q J (u_h - u_t)_q dU(x_q)/dU.
"""
from __future__ import annotations

import numpy as np

from .functional import eval_tensor, eval_tensor_T, tables


def element_fields(disc, U, e):
    """(v, v_x, v_y, v_z, Lap v) in physical coordinates at the (2W+1)^3 points."""
    B0, B1, B2 = tables(disc.W[e])["B"]
    u = disc.block(U, e)
    s = disc.scale(e)
    v = eval_tensor(u, B0, B0, B0)
    vx = s[0] * eval_tensor(u, B1, B0, B0)
    vy = s[1] * eval_tensor(u, B0, B1, B0)
    vz = s[2] * eval_tensor(u, B0, B0, B1)
    lap = (s[0] ** 2 * eval_tensor(u, B2, B0, B0) + s[1] ** 2 * eval_tensor(u, B0, B2, B0) +
           s[2] ** 2 * eval_tensor(u, B0, B0, B2))
    return v, vx, vy, vz, lap


def l2_misfit(disc, U, u_target):
    """J(U) = sum_q w_q J (u_h - u_t)^2 over all elements."""
    J = 0.0
    for e in range(disc.E):
        xs, ys, zs = disc.qpoints(e)
        d = element_fields(disc, U, e)[0] - u_target(xs, ys, zs)
        J += float(np.sum(disc.vol_weight(e) * d * d))
    return J


def l2_misfit_gradient(disc, U, u_target):
    """dJ/dU = 2 sum_q w_q J (u_h - u_t)_q dU(x_q)/dU."""
    g = np.zeros(disc.ndof)
    for e in range(disc.E):
        B0 = tables(disc.W[e])["B"][0]
        xs, ys, zs = disc.qpoints(e)
        d = element_fields(disc, U, e)[0] - u_target(xs, ys, zs)
        g[disc.off[e]:disc.off[e + 1]] = eval_tensor_T(2.0 * disc.vol_weight(e) * d, B0, B0, B0).ravel()
    return g


def data_gradient(disc, U, lam, rhs=0):
    """Per element e: (dJ/df, dJ/da, dJ/d a_x, dJ/d a_y, dJ/d a_z) at its (2W+1)^3 points."""
    out = []
    for e in range(disc.E):
        a, (ax, ay, az) = disc.coef(e)
        f = disc.f_at(e, rhs)
        wJ = disc.vol_weight(e)
        u, ux, uy, uz, lu = element_fields(disc, U, e)
        l, lx, ly, lz, ll = element_fields(disc, lam, e)
        Lu = -a * lu - (ax * ux + ay * uy + az * uz)
        Ll = -a * ll - (ax * lx + ay * ly + az * lz)
        res = Lu - f
        out.append((wJ * Ll, wJ * (lu * Ll + res * ll), wJ * (ux * Ll + res * lx),
                    wJ * (uy * Ll + res * ly), wJ * (uz * Ll + res * lz)))
    return out


# ---------------------------------------------------------------------------
# Second order: the same functional with the data as free point arrays
# theta = (f [nquad], a [nquad], grad a [3, nquad]) (element-major, each
# element's points in [c, b, a] order), by dense algebra on small meshes.
#   S(theta) U = sqrt(wJ) (-a Lap U - grad a . grad U)   (the volume residual's
#                                                          linear part)
#   A(theta) = S^T S + A_faces,  b(theta) = S^T sqrt(wJ) f + b_faces
# where A_faces, b_faces (the face and Dirichlet terms of eq. 4.2) do not
# depend on theta and are taken from the Discretisation at its own data.
# The Hessian-vector product is the central difference of the exact
# adjoint gradient (dense Cholesky solves); its pins are the symmetry of the
# Hessian and the second difference of J itself.
# ---------------------------------------------------------------------------
def field_matrices(disc):
    """[5, nquad, ndof] dense maps U -> (v, v_x, v_y, v_z, Lap v) at all points."""
    nq = sum((2 * w + 1) ** 3 for w in disc.W)
    F = np.zeros((5, nq, disc.ndof))
    o = 0
    for e in range(disc.E):
        n = (2 * disc.W[e] + 1) ** 3
        for j in range(disc.off[e], disc.off[e + 1]):
            U = np.zeros(disc.ndof)
            U[j] = 1.0
            for k, fld in enumerate(element_fields(disc, U, e)):
                F[k, o:o + n, j] = fld.ravel()
        o += n
    return F


def point_weights(disc):
    return np.concatenate([disc.vol_weight(e).ravel() for e in range(disc.E)])


def point_data(disc, rhs=0):
    """theta of the Discretisation's own problem: (f, a, grad a) at the points."""
    f = np.concatenate([disc.f_at(e, rhs).ravel() for e in range(disc.E)])
    a = np.concatenate([np.asarray(disc.coef(e)[0]).ravel() for e in range(disc.E)])
    ga = np.stack([np.concatenate([np.asarray(disc.coef(e)[1][k]).ravel() for e in range(disc.E)])
                   for k in range(3)])
    return f, a, ga


class DenseAdjoint:
    """J(theta) = sum_q wJ (v(U) - u_t)^2 with A(theta) U = b(theta), its adjoint
    gradient and Hessian-vector products, for a small box-mesh Discretisation."""

    def __init__(self, disc, ut):
        self.disc = disc
        self.F = field_matrices(disc)
        self.w = point_weights(disc)
        self.ut = np.asarray(ut, dtype=np.float64)
        f0, a0, ga0 = point_data(disc)
        S0 = self.S(a0, ga0)
        self.A_faces = disc.dense_A() - S0.T @ S0
        self.b_faces = disc.rhs_b() - S0.T @ (np.sqrt(self.w) * f0)

    def S(self, a, ga):
        F = self.F
        L = -(a[:, None] * F[4]) - sum(ga[k][:, None] * F[1 + k] for k in range(3))
        return np.sqrt(self.w)[:, None] * L

    def solve(self, f, a, ga):
        S = self.S(a, ga)
        A = S.T @ S + self.A_faces
        b = S.T @ (np.sqrt(self.w) * f) + self.b_faces
        return A, np.linalg.solve(A, b)

    def J(self, f, a, ga):
        _, U = self.solve(f, a, ga)
        d = self.F[0] @ U - self.ut
        return float(np.sum(self.w * d * d))

    def gradient(self, f, a, ga):
        """(dJ/df, dJ/da, dJ/d grad a) by the adjoint state (the formulas of
        data_gradient with the point arrays)."""
        A, U = self.solve(f, a, ga)
        lam = np.linalg.solve(A, self.F[0].T @ (2.0 * self.w * (self.F[0] @ U - self.ut)))
        u = [self.F[k] @ U for k in range(5)]
        lm = [self.F[k] @ lam for k in range(5)]
        Lu = -a * u[4] - sum(ga[k] * u[1 + k] for k in range(3))
        Ll = -a * lm[4] - sum(ga[k] * lm[1 + k] for k in range(3))
        res = Lu - f
        w = self.w
        return (w * Ll, w * (u[4] * Ll + res * lm[4]),
                np.stack([w * (u[1 + k] * Ll + res * lm[1 + k]) for k in range(3)]))

    def hessian_vector(self, f, a, ga, v, h):
        """Central difference of the adjoint gradient along v = (vf, va, vga)."""
        gp = self.gradient(f + h * v[0], a + h * v[1], ga + h * v[2])
        gm = self.gradient(f - h * v[0], a - h * v[1], ga - h * v[2])
        return tuple((p - m) / (2.0 * h) for p, m in zip(gp, gm))

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

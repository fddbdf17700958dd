"""The volume variation in integration-by-parts form (oracle, FP64).

Test infrastructure only (see the package docstring).

Section 5.3, eq. (5.45)-(5.48): the variation of the volume term of one
element, sum_q w_q (L v)(xi_q) z_q over the (2W+1)^3 GLL points of the master
cube, is read as the integral of (L v) Z, Z the interpolant of degree 2W of
the point values z in each variable (the quadrature is exact for it), and
integrated by parts onto Z:

  int_Q (L v) Z = int_Q v (L^T Z) + sum over the six faces of boundary terms,

where L^T is the formal adjoint of L, the derivatives of Z are taken with the
(2W+1)-point differentiation matrix (eq. 5.47: exact for a polynomial of
degree 2W) and every integral with the same GLL rule.  A coefficient c(xi)
of a term is applied to the point values first: sum_q w_q c_q v_aa(xi_q) z_q
is exactly int v_aa I(c z), I the degree-2W interpolant, and the adjoint
differentiates I(c z), the (c z)_{xi xi} of eq. (5.46).  Every integrand is
then a polynomial of degree at most 4W - 1 in each variable, which the
(2W+1)-point GLL rule integrates exactly, so the result equals the direct
transpose of the sum factorisation (the reverse of eq. 5.45's evaluation)
up to rounding, for constant and for pointwise-sampled coefficients alike.

L here: a box element in reference coordinates with
L v = sum_a alpha_a v_aa + sum_a beta_a v_a + gamma v (no mixed terms; the
Laplacian is alpha_a = -s_a^2, beta = gamma = 0); alpha_a, beta_a, gamma are
constants or arrays of point values.  Per variable a, with [g]_a the
difference of g at xi_a = 1 and xi_a = -1 integrated over the face:

  int v_aa I(c z) = int v I(c z)_aa + [v_a I(c z) - v I(c z)_a]_a,
  int v_a I(c z)  = -int v I(c z)_a + [v I(c z)]_a,

so y_k = int phi_k (sum_a A_a,aa - sum_a B_a,a + G)
       + sum_a [phi_k,a A_a - phi_k A_a,a + phi_k B_a]_a
with A_a = I(alpha_a z), B_a = I(beta_a z), G = I(gamma z).
"""
from __future__ import annotations

import numpy as np

from .functional import eval_tensor_T, tables
from .gll import diff_matrix, gll


def _along(M, Z, axis):
    """Apply the matrix M along axis (0 = x, the last index of the [z, y, x] array)."""
    ax = 2 - axis
    return np.moveaxis(np.tensordot(M, Z, axes=([1], [ax])), 0, ax)


def ibp_transpose(W, z, alpha, beta=(0.0, 0.0, 0.0), gamma=0.0):
    """y[P, P, P] = sum_q w_q (L phi_k)(xi_q) z_q for the point values
    z[Q, Q, Q] ([z, y, x] order), by eq. (5.46)-(5.48); alpha, beta: three
    constants or [Q, Q, Q] arrays each, gamma one."""
    t = tables(W)
    P, Q = W + 1, 2 * W + 1
    B0 = t["B"][0]
    xq, wq = gll(Q)
    DQ = diff_matrix(xq)
    xp, _ = gll(P)
    DP = diff_matrix(xp)
    Z = np.asarray(z, dtype=np.float64).reshape(Q, Q, Q)
    A = [np.broadcast_to(alpha[a], (Q, Q, Q)) * Z for a in range(3)]
    B = [np.broadcast_to(beta[a], (Q, Q, Q)) * Z for a in range(3)]
    V = np.broadcast_to(gamma, (Q, Q, Q)) * Z
    # volume: the formal adjoint at the points, weighted, projected onto the nodal basis
    for a in range(3):
        V = V + _along(DQ, _along(DQ, A[a], a), a) - _along(DQ, B[a], a)
    w3 = wq[:, None, None] * wq[None, :, None] * wq[None, None, :]
    y = eval_tensor_T(w3 * V, B0, B0, B0)
    # the six faces: phi_k(+-1) picks the end node, phi_k'(+-1) is a row of D_P
    for a in range(3):
        Aa = _along(DQ, A[a], a)
        shape = [Q if i != 2 - a else 1 for i in range(3)]
        w2 = (wq[:, None] * wq[None, :]).reshape(shape)
        for side in (0, 1):
            sg = 1.0 if side else -1.0
            n = Q - 1 if side else 0
            e = P - 1 if side else 0
            sl = [slice(None)] * 3
            sl[2 - a] = slice(n, n + 1)
            sl = tuple(sl)
            val = np.zeros((1, P))
            val[0, e] = 1.0
            mats = [B0, B0, B0]
            mats[a] = DP[e:e + 1, :]
            y = y + sg * eval_tensor_T(w2 * A[a][sl], *mats)
            mats[a] = val
            y = y + sg * eval_tensor_T(w2 * (B[a][sl] - Aa[sl]), *mats)
    return y

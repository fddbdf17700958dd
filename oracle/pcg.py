"""Preconditioned conjugate gradients on the normal equations (oracle, FP64).

Test infrastructure only (see the package docstring).

Section 5.1 / 6.1: PCG on A U = b with the block-diagonal preconditioner,
stopped when the relative norm of the normal-equation residual drops below
eps.  Reading: x_0 = 0 and the criterion is ||b - A x_k||_2 <= eps ||b||_2
(Euclidean norm of the nodal coefficient vector), with the recursively
updated residual.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def pcg(apply_A, apply_M, b, tol=1e-10, maxit=10000, x0=None):
    """Textbook PCG.  Returns (x, iterations, final relative residual)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_A(x) if x0 is not None else b.copy()
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return x, 0, 0.0
    z = apply_M(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    rel = float(np.linalg.norm(r)) / bn
    while rel > tol and it < maxit:
        q = apply_A(p)
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        z = apply_M(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
        it += 1
        rel = float(np.linalg.norm(r)) / bn
    return x, it, rel


def cholesky_solve(A, b):
    """Direct solve of the normal equations (tiny meshes)."""
    c = sla.cho_factor(A)
    return sla.cho_solve(c, b)

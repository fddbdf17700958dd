"""Relative H^1 error (oracle, FP64).

Test infrastructure only (see the package docstring).

Section 6.1: ||E||_rel = ||u_appx - u_ex||_{H^1} / ||u_ex||_{H^1}.  Reading:
both norms are computed element by element in physical coordinates with the
(2W+1)^3-point GLL rule of the element (exact for the difference of two
discrete solutions, spectrally accurate against a smooth exact solution).
"""
from __future__ import annotations

import numpy as np

from .functional import eval_tensor, tables


def _element_fields(disc, U, e):
    B0, B1, _ = tables(disc.W[e])["B"]
    u = disc.block(U, e)
    s = disc.scale(e)
    return (eval_tensor(u, B0, B0, B0), s[0] * eval_tensor(u, B1, B0, B0),
            s[1] * eval_tensor(u, B0, B1, B0), s[2] * eval_tensor(u, B0, B0, B1))


def h1_error_exact(disc, U, rhs=0):
    """Relative H^1 error of the discrete U against the problem's exact solution."""
    pb = disc.problem
    num = 0.0
    den = 0.0
    for e in range(disc.E):
        xs, ys, zs = disc.qpoints(e)
        ue = pb.u_exact[rhs](xs, ys, zs)
        ge = pb.grad_u_exact[rhs](xs, ys, zs)
        uh = _element_fields(disc, U, e)
        wJ = disc.vol_weight(e)
        num += float(np.sum(wJ * ((uh[0] - ue) ** 2 + sum((uh[k + 1] - ge[k]) ** 2 for k in range(3)))))
        den += float(np.sum(wJ * (ue ** 2 + sum(g ** 2 for g in ge))))
    return float(np.sqrt(num / den))


def h1_norm_sq(disc, U):
    tot = 0.0
    for e in range(disc.E):
        uh = _element_fields(disc, U, e)
        tot += float(np.sum(disc.vol_weight(e) * sum(f ** 2 for f in uh)))
    return tot


def h1_rel_diff(disc, U, Uref):
    """||U - Uref||_{H^1} / ||Uref||_{H^1} for two discrete solutions."""
    return float(np.sqrt(h1_norm_sq(disc, U - Uref) / h1_norm_sq(disc, Uref)))

"""Gauss-Lobatto-Legendre rules and Lagrange evaluation matrices (oracle).

Section 5.3: the residual is collocated on the (2W+1)-point GLL grid, the
unknowns live on the (W+1)-point GLL grid, and eq. (5.47) defines the GLL
differentiation matrix.  Everything here is the textbook definition written
out directly (product formulas for the Lagrange basis), FP64.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def legendre(n: int, x):
    """L_n(x) by the three-term recurrence (n+1) L_{n+1} = (2n+1) x L_n - n L_{n-1}."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0
    p1 = x.copy()
    for m in range(1, n):
        p0, p1 = p1, ((2 * m + 1) * x * p1 - m * p0) / (m + 1)
    return p1


def gll(n_points: int):
    """GLL nodes and weights with n_points = N+1 points.

    Nodes: -1, +1 and the N-1 roots of L'_N; weights w_i = 2 / (N (N+1) L_N(x_i)^2).
    """
    N = n_points - 1
    if N < 1:
        raise ValueError("a GLL rule needs at least 2 points")
    c = np.zeros(N + 1)
    c[N] = 1.0
    inner = np.sort(np.real(npleg.legroots(npleg.legder(c)))) if N >= 2 else np.zeros(0)
    x = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (N * (N + 1) * legendre(N, x) ** 2)
    return x, w


def lagrange_eval(nodes, points, order: int = 0):
    """Matrix M[q, j] = d^order/dx^order l_j(points[q]) for the Lagrange basis on nodes.

    l_j(x) = prod_{m != j} (x - x_m) / (x_j - x_m); the derivatives are the
    product rule written out (sums over the removed factors).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    pts = np.atleast_1d(np.asarray(points, dtype=np.float64))
    P = len(nodes)
    M = np.zeros((len(pts), P))
    for j in range(P):
        others = [m for m in range(P) if m != j]
        den = np.prod([nodes[j] - nodes[m] for m in others])
        if order == 0:
            val = np.ones_like(pts)
            for m in others:
                val = val * (pts - nodes[m])
        elif order == 1:
            val = np.zeros_like(pts)
            for a in others:
                t = np.ones_like(pts)
                for m in others:
                    if m != a:
                        t = t * (pts - nodes[m])
                val = val + t
        elif order == 2:
            val = np.zeros_like(pts)
            for a in others:
                for b in others:
                    if b == a:
                        continue
                    t = np.ones_like(pts)
                    for m in others:
                        if m != a and m != b:
                            t = t * (pts - nodes[m])
                    val = val + t
        else:
            raise ValueError("order must be 0, 1 or 2")
        M[:, j] = val / den
    return M


def diff_matrix(nodes):
    """GLL differentiation matrix of eq. (5.47): (dl/dx)(x_i) = sum_j d_ij l(x_j)."""
    return lagrange_eval(nodes, nodes, 1)

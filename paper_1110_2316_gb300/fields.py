"""Differentiable coefficient fields at a mesh's volume points (torch).

A user-side model over the library: maps parameters to the coefficient data
that ``Mesh.set_data`` / ``autograd.Solve`` take, so that torch autograd
carries the library's point gradients dJ/da, dJ/d(grad a) on to the
parameters.  Vectorised per degree group (elements of one W share the point
count), one index_copy per group back into the mesh's point order.

``LegendreLogField``: a = exp(g) with g = sum_{i,j,k<=K} theta_ijk L_i L_j L_k
on each problem's box [lo, hi]^3 mapped to (-1,1)^3 (Legendre polynomials
L_i), theta of shape [n_problem, K+1, K+1, K+1].  Point order per element is
(z, y, x) with x fastest, as in ``Mesh.query_points``.
"""
from __future__ import annotations

import numpy as np
import torch


def _legendre(K, t):
    """L_0..L_K and their derivatives at t (any shape), stacked on a new axis -2."""
    L = [torch.ones_like(t), t]
    dL = [torch.zeros_like(t), torch.ones_like(t)]
    for m in range(1, K):
        L.append(((2 * m + 1) * t * L[m] - m * L[m - 1]) / (m + 1))
        dL.append(dL[m - 1] + (2 * m + 1) * L[m])
    return torch.stack(L[:K + 1], -2), torch.stack(dL[:K + 1], -2)


class LegendreLogField:
    """ax: per element the 1-D point coordinates (x, y, z), 3Q values each,
    concatenated (``Mesh.query_points()[0]``); Ws: degree per element."""

    def __init__(self, ax, Ws, elem_problem, K=3, lo=0.0, hi=1.0, device="cuda"):
        Ws = [int(w) for w in Ws]
        self.K, self.nq = K, int(sum((2 * w + 1) ** 3 for w in Ws))
        off_ax = np.cumsum([0] + [3 * (2 * w + 1) for w in Ws])
        off_q = np.cumsum([0] + [(2 * w + 1) ** 3 for w in Ws])
        eprob = np.asarray(elem_problem)
        self.groups = []
        sc = 2.0 / (hi - lo)
        for W in sorted(set(Ws)):
            Q = 2 * W + 1
            idx = np.array([e for e, w in enumerate(Ws) if w == W])
            coords = np.stack([ax[off_ax[e]:off_ax[e] + 3 * Q].reshape(3, Q) for e in idx])  # [E,3,Q]
            t = torch.tensor(sc * (coords - lo) - 1.0, dtype=torch.float64, device=device)
            L, dL = _legendre(K, t)  # [E,3,K+1,Q]
            qidx = torch.tensor((off_q[idx][:, None] + np.arange(Q ** 3)[None, :]).ravel(), device=device)
            self.groups.append(dict(L=L, dL=dL * sc, prob=torch.tensor(eprob[idx], device=device),
                                    qidx=qidx, coords=torch.tensor(coords, device=device)))

    @classmethod
    def from_mesh(cls, mesh, elem_problem, **kw):
        return cls(mesh.query_points()[0], mesh.elem_W, elem_problem, **kw)

    def __call__(self, theta):
        """(a [nq], grad_a [3, nq]) for theta [n_problem, K+1, K+1, K+1]."""
        a = torch.zeros(self.nq, dtype=theta.dtype, device=theta.device)
        ga = torch.zeros(3, self.nq, dtype=theta.dtype, device=theta.device)
        for gr in self.groups:
            th = theta[gr["prob"]]
            L, dL = gr["L"], gr["dL"]
            Lx, Ly, Lz = L[:, 0], L[:, 1], L[:, 2]

            def ev(X, Y, Z):
                return torch.einsum("eijk,eia,ejb,ekc->ecba", th, X, Y, Z).reshape(-1)
            ea = torch.exp(ev(Lx, Ly, Lz))
            a = a.index_copy(0, gr["qidx"], ea)
            comps = [ea * ev(dL[:, 0], Ly, Lz), ea * ev(Lx, dL[:, 1], Lz), ea * ev(Lx, Ly, dL[:, 2])]
            ga = ga.index_copy(1, gr["qidx"], torch.stack(comps))
        return a, ga

    def separable(self, fx, fy, fz):
        """fz(z) fy(y) fx(x) at every volume point (torch callables on 1-D tensors)."""
        out = torch.zeros(self.nq, dtype=torch.float64, device=self.groups[0]["L"].device)
        for gr in self.groups:
            c = gr["coords"]
            v = torch.einsum("ea,eb,ec->ecba", fx(c[:, 0]), fy(c[:, 1]), fz(c[:, 2])).reshape(-1)
            out = out.index_copy(0, gr["qidx"], v)
        return out

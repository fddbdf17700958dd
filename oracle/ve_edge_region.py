"""The vertex-edge cone and the edge neighbourhood above it, joined on the
plane x3 = delta (oracle, FP64).

Test infrastructure only (see the package docstring).

Along an edge leaving a vertex, Section 2.3 splits the edge's neighbourhood
into the vertex-edge cone (x3 < delta_v, oracle/vertex_edge.py) and the edge
neighbourhood (x3 > delta_v, oracle/edge.py).  The functional is the sum of
the two regions' functionals, the plane x3 = delta excluded from both, plus
the terms of that interface.

Reading of the interface (the thesis's sums run inside one region): the face
belongs to the vertex-edge side and takes its interior-face terms (eq. 2.29 on
a face zeta = const: [u] in L2 times F G, the jumps of u_psi, u_theta and
E u_zeta in the norm of eq. 2.27); the edge side's modified derivatives are
converted there by the chain rule of tau = psi + zeta, x3 = e^zeta:
u_psi = u_tau, u_theta = u_theta, u_zeta = u_tau + x3 u_x3 (x3 = delta).
With the edge layers r_i = delta tan(phi_i) the two face grids are the same
points.  The corner regions that meet across the plane (r < r_1) have
infinite measure in modified coordinates and no face term there.

Layout: the vertex-edge elements, the edge elements, the vertex-edge corner
sets, the edge corner sets.
"""
from __future__ import annotations

import numpy as np

from .edge import EdgeDiscretisation, l2_literal
from .vertex_edge import VertexEdgeDiscretisation


class VertexEdgeEdgeDiscretisation:

    def __init__(self, ve_problem, edge_problem, pairs, delta):
        self.vd = VertexEdgeDiscretisation(ve_problem)
        self.ed = EdgeDiscretisation(edge_problem)
        self.pairs = list(pairs)
        self.delta = float(delta)
        for a, b in self.pairs:
            self.vd.skip_faces.add((a, 5))
            self.ed.skip_faces.add((b, 4))
        self.nV, self.nE = int(self.vd.off[-1]), int(self.ed.off[-1])
        self.nVC, self.nEC = self.vd.ndof - self.nV, self.ed.ndof - self.nE
        self.ndof = self.nV + self.nE + self.nVC + self.nEC

    def split(self, U):
        a, b, c = self.nV, self.nV + self.nE, self.nV + self.nE + self.nVC
        return np.concatenate([U[:a], U[b:c]]), np.concatenate([U[a:b], U[c:]])

    def merge(self, yv, ye):
        return np.concatenate([yv[:self.nV], ye[:self.nE], yv[self.nV:], ye[self.nE:]])

    def _Qf(self, a, b):
        return 2 * max(self.vd.W[a], self.ed.W[b]) + 1

    def _jumps(self, Uv, Ue, a, b, Qf):
        fv = self.vd.face_fields(self.vd.block(Uv, a), a, 5, Qf)
        fe = self.ed.face_fields(self.ed.block(Ue, b), b, 4, Qf)
        conv = [fe[0], fe[1], fe[2], fe[1] + self.delta * fe[3]]
        return [fv[k] - conv[k] for k in range(4)]

    def functional(self, U):
        Uv, Ue = self.split(U)
        R = self.vd.functional(Uv) + self.ed.functional(Ue)
        for a, b in self.pairs:
            Qf = self._Qf(a, b)
            J = self._jumps(Uv, Ue, a, b, Qf)
            c = self.vd.norm_weights(a, 5)
            E = self.vd.E_sup(a, 5)
            R += self.vd._u_weight(a, 5, False) * l2_literal(J[0], Qf)
            R += self.vd._norm_literal(J[1], Qf, c) + self.vd._norm_literal(J[2], Qf, c)
            R += E * E * self.vd._norm_literal(J[3], Qf, c)
        return R

    def apply_A(self, U):
        Uv, Ue = self.split(U)
        yv, ye = self.vd.apply_A(Uv), self.ed.apply_A(Ue)
        for a, b in self.pairs:
            Qf = self._Qf(a, b)
            J = self._jumps(Uv, Ue, a, b, Qf)
            M = self.vd.jump_forms(a, 5, Qf)
            g = [(M[k] @ J[k].ravel()).reshape(Qf, Qf) for k in range(4)]
            yv[self.vd.off[a]:self.vd.off[a + 1]] += self.vd.face_fields_T(g, a, 5, Qf).ravel()
            ge = [g[0], g[1] + g[3], g[2], self.delta * g[3]]
            ye[self.ed.off[b]:self.ed.off[b + 1]] -= self.ed.face_fields_T(ge, b, 4, Qf).ravel()
        return self.merge(yv, ye)

    def rhs_b(self):
        return self.merge(self.vd.rhs_b(), self.ed.rhs_b())

    def h1_error_exact(self, U):
        Uv, Ue = self.split(U)
        e1, n1 = self.vd.h1_error_exact(Uv)
        e2, n2 = self.ed.h1_error_exact(Ue)
        return np.sqrt((e1 + e2) / (n1 + n2))

"""A vertex neighbourhood with one re-entrant edge: the vertex part and the
vertex-edge cone joined on phi = phi_v (oracle, FP64).

Test infrastructure only (see the package docstring).

Section 2.3 splits a vertex neighbourhood into the vertex-edge cones around
its edges and the rest; on the corner elements both hold the same constant
h_v (the vertex-edge corner value is the vertex's).  The functional is the
sum of the two regions' functionals (oracle/vertex.py, oracle/vertex_edge.py),
the cone phi = phi_v excluded from both, plus the terms of that interface.

Reading of the interface (the thesis's sums run inside one region): the face
belongs to the vertex-edge side and takes its interior-face terms (eq. 2.29:
[u] in L2 times F G, the jumps of u_psi, u_theta and E u_zeta in the norm of
eq. 2.27); the vertex side's modified derivatives are converted at the face
(phi = phi_v, tan phi = e^psi, chi = zeta - ln cos phi) by the chain rule:
u_psi = sin(phi) cos(phi) u_phi + sin^2(phi) u_chi, u_theta = u_theta,
u_zeta = u_chi.  On the face chi and zeta differ by the constant ln cos phi_v,
so the two sides' face grids are the same points when their layers match
(delta_v = rho_v cos phi_v, the thesis's choice).

Layout: the vertex elements, the vertex-edge elements, the shared constant,
then the vertex-edge corner polynomials.
"""
from __future__ import annotations

import numpy as np

from .vertex import VertexDiscretisation
from .vertex_edge import VertexEdgeDiscretisation


class VertexRegionDiscretisation:

    def __init__(self, vertex_problem, ve_problem, pairs):
        self.vd = VertexDiscretisation(vertex_problem)
        self.ed = VertexEdgeDiscretisation(ve_problem)
        self.pairs = list(pairs)
        for ve_e, v_e in self.pairs:
            self.ed.skip_faces.add((ve_e, 1))
            self.vd.skip_faces.add((v_e, 0))
        assert self.vd.C == 1 and self.vd.Wc[0] == 0
        self.kconst = self.ed.cface.index(4)                       # the vertex-edge constant
        self.polys = [c for c in range(self.ed.C) if c != self.kconst]
        self.nV = int(self.vd.off[-1])
        self.nE = int(self.ed.off[-1])
        self.nP = sum(self.ed.Wc[c] + 1 for c in self.polys)
        self.ndof = self.nV + self.nE + 1 + self.nP
        phi = float(self.vd.mesh.elem_lo[self.pairs[0][1], 0])
        self.sc, self.s2 = np.sin(phi) * np.cos(phi), np.sin(phi) ** 2

    # --- layout ---------------------------------------------------------------
    def split(self, U):
        h = U[self.nV + self.nE]
        Uv = np.concatenate([U[:self.nV], [h]])
        Ue = np.zeros(self.ed.ndof)
        Ue[:self.nE] = U[self.nV:self.nV + self.nE]
        o = self.nV + self.nE + 1
        for c in self.polys:
            n = self.ed.Wc[c] + 1
            Ue[self.ed.coff[c]:self.ed.coff[c] + n] = U[o:o + n]
            o += n
        Ue[self.ed.coff[self.kconst]] = h
        return Uv, Ue

    def merge(self, yv, ye):
        y = np.zeros(self.ndof)
        y[:self.nV] = yv[:self.nV]
        y[self.nV:self.nV + self.nE] = ye[:self.nE]
        y[self.nV + self.nE] = yv[self.vd.coff[0]] + ye[self.ed.coff[self.kconst]]
        o = self.nV + self.nE + 1
        for c in self.polys:
            n = self.ed.Wc[c] + 1
            y[o:o + n] = ye[self.ed.coff[c]:self.ed.coff[c] + n]
            o += n
        return y

    # --- the interface --------------------------------------------------------
    def _Qf(self, ve_e, v_e):
        return 2 * max(self.ed.W[ve_e], self.vd.W[v_e]) + 1

    def _jumps(self, Uv, Ue, ve_e, v_e, Qf):
        fe = self.ed.face_fields(self.ed.block(Ue, ve_e), ve_e, 1, Qf)
        fv = self.vd.face_fields(self.vd.block(Uv, v_e), v_e, 0, Qf)
        conv = [fv[0], self.sc * fv[1] + self.s2 * fv[3], fv[2], fv[3]]
        return [fe[k] - conv[k] for k in range(4)]

    def functional(self, U):
        from .edge import l2_literal
        Uv, Ue = self.split(U)
        R = self.vd.functional(Uv) + self.ed.functional(Ue)
        for ve_e, v_e in self.pairs:
            Qf = self._Qf(ve_e, v_e)
            J = self._jumps(Uv, Ue, ve_e, v_e, Qf)
            c = self.ed.norm_weights(ve_e, 1)
            E = self.ed.E_sup(ve_e, 1)
            R += self.ed._u_weight(ve_e, 1, False) * l2_literal(J[0], Qf)
            R += self.ed._norm_literal(J[1], Qf, c) + self.ed._norm_literal(J[2], Qf, c)
            R += E * E * self.ed._norm_literal(J[3], Qf, c)
        return R

    def apply_A(self, U):
        Uv, Ue = self.split(U)
        yv, ye = self.vd.apply_A(Uv), self.ed.apply_A(Ue)
        for ve_e, v_e in self.pairs:
            Qf = self._Qf(ve_e, v_e)
            J = self._jumps(Uv, Ue, ve_e, v_e, Qf)
            M = self.ed.jump_forms(ve_e, 1, Qf)
            g = [(M[k] @ J[k].ravel()).reshape(Qf, Qf) for k in range(4)]
            ye[self.ed.off[ve_e]:self.ed.off[ve_e + 1]] += self.ed.face_fields_T(g, ve_e, 1, Qf).ravel()
            gv = [g[0], self.sc * g[1], g[2], self.s2 * g[1] + g[3]]
            yv[self.vd.off[v_e]:self.vd.off[v_e + 1]] -= self.vd.face_fields_T(gv, v_e, 0, Qf).ravel()
        return self.merge(yv, ye)

    def rhs_b(self):
        return self.merge(self.vd.rhs_b(), self.ed.rhs_b())

    def h1_error_exact(self, U):
        Uv, Ue = self.split(U)
        e1, n1 = self.vd.h1_error_exact(Uv)
        e2, n2 = self.ed.h1_error_exact(Ue)
        return np.sqrt((e1 + e2) / (n1 + n2))

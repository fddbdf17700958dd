"""The L-shaped prism: an edge neighbourhood next to curved regular elements
(oracle, FP64).

Test infrastructure only (see the package docstring).

((0,1)^2 minus (0.5,1)^2) x (0,1) with its re-entrant edge on the line
x = y = 0.5: the edge neighbourhood r < Z (modified coordinates
(tau, theta', x3), eq. 4.7; oracle/edge.py) and the regular region r > Z in
polar-blend sectors (oracle/curved.py).  The functional is the sum of the two
regions' functionals, the circle r = Z excluded from both, plus the terms of
that interface.

Reading of the interface (the thesis's sums run over faces inside each region
and do not say which coordinates and weights a face between two regions
takes): the face belongs to the singular side.  Its terms are those of an
interior face of the edge neighbourhood (eq. 4.7: [u] in L2, the jumps of
u_tau, u_theta and G u_x3 in the anisotropic norm of eq. 2.34, with that
face's weights), the regular side's gradient converted into the edge's
modified derivatives at the face points by the chain rule:
u_tau = r u_r = (x - c) u_x + (y - c) u_y, u_theta = u_phi =
-(y - c) u_x + (x - c) u_y, u_x3 = u_z, with phi = theta' + pi/2 the polar
angle about the edge c = (0.5, 0.5).

Layout: the edge elements' blocks, then the regular elements' blocks, then
the edge neighbourhood's corner sets.
"""
from __future__ import annotations

import numpy as np

from .curved import CurvedDiscretisation
from .edge import EdgeDiscretisation


class LPrismDiscretisation:
    """Composite oracle of an edge problem (one x3 slab, the outer layer's
    face tau = ln Z towards the regular region) and a curved problem (one
    sector element per edge sector, its face t = 0 towards the edge)."""

    C = 0.5

    def __init__(self, edge_problem, curved_problem, pairs):
        """pairs: list of (edge element, curved element) sharing the circle r = Z
        (edge face 1, curved face 0, the same (theta, x3) parametrisation)."""
        self.ed = EdgeDiscretisation(edge_problem)
        self.cu = CurvedDiscretisation(curved_problem)
        self.pairs = list(pairs)
        for e, j in self.pairs:
            self.ed.skip_faces.add((e, 1))
            self.cu.skip_faces.add((j, 0))
        self.nE = int(self.ed.off[-1])              # edge element DOFs
        self.nR = self.cu.ndof
        self.nC = self.ed.ndof - self.nE            # corner DOFs
        self.ndof = self.nE + self.nR + self.nC

    # --- layout ---------------------------------------------------------------
    def split(self, U):
        Ue = np.concatenate([U[:self.nE], U[self.nE + self.nR:]])
        return Ue, U[self.nE:self.nE + self.nR]

    def merge(self, Ue, Ur):
        return np.concatenate([Ue[:self.nE], Ur, Ue[self.nE:]])

    # --- the interface --------------------------------------------------------
    def _Qf(self, e, j):
        return 2 * max(self.ed.W[e], self.cu.W[j]) + 1

    def _to_modified(self, fr, j, Qf):
        """Regular side's [u, u_x, u_y, u_z] -> [u, u_tau, u_theta, u_x3]."""
        x, _ = self.cu.face_geom(j, 0, Qf)
        dx, dy = x[0] - self.C, x[1] - self.C
        return [fr[0], dx * fr[1] + dy * fr[2], -dy * fr[1] + dx * fr[2], fr[3]]

    def _from_modified_T(self, gs, j, Qf):
        """Transpose of _to_modified on the field weights."""
        x, _ = self.cu.face_geom(j, 0, Qf)
        dx, dy = x[0] - self.C, x[1] - self.C
        return [gs[0], dx * gs[1] - dy * gs[2], dy * gs[1] + dx * gs[2], gs[3]]

    def _jumps(self, Ue, Ur, e, j, Qf):
        fe = self.ed.face_fields(self.ed.block(Ue, e), e, 1, Qf)
        fr = self._to_modified(self.cu.face_fields(self.cu.block(Ur, j), j, 0, Qf), j, Qf)
        return [fe[k] - fr[k] for k in range(4)]

    # --- functional, operator, right-hand side -------------------------------
    def functional(self, U):
        Ue, Ur = self.split(U)
        R = self.ed.functional(Ue) + self.cu.functional(Ur)
        from .edge import l2_literal
        for e, j in self.pairs:
            Qf = self._Qf(e, j)
            J = self._jumps(Ue, Ur, e, j, Qf)
            _, _, t1, t2 = self.ed.face_axes(1)
            hh = self.ed.h(e) / 2.0
            G = self.ed.G(e, 1)
            c = self.ed.norm_weights(e, 1)
            R += hh[t1] * hh[t2] * l2_literal(J[0], Qf)      # H = 1 on a face tau = const
            R += self.ed._norm_literal(J[1], Qf, c) + self.ed._norm_literal(J[2], Qf, c)
            R += G * G * self.ed._norm_literal(J[3], Qf, c)
        return R

    def apply_A(self, U):
        Ue, Ur = self.split(U)
        ye = self.ed.apply_A(Ue)
        yr = self.cu.apply_A(Ur)
        for e, j in self.pairs:
            Qf = self._Qf(e, j)
            J = self._jumps(Ue, Ur, e, j, Qf)
            M = self.ed.jump_forms(e, 1, Qf)
            gs = [(M[k] @ J[k].ravel()).reshape(Qf, Qf) for k in range(4)]
            ye[self.ed.off[e]:self.ed.off[e + 1]] += self.ed.face_fields_T(gs, e, 1, Qf).ravel()
            gr = self._from_modified_T(gs, j, Qf)
            yr[self.cu.off[j]:self.cu.off[j + 1]] -= self.cu.face_fields_T(gr, j, 0, Qf).ravel()
        return self.merge(ye, yr)

    def rhs_b(self):
        return self.merge(self.ed.rhs_b(), self.cu.rhs_b())

    def dense_A(self):
        A = np.zeros((self.ndof, self.ndof))
        for k in range(self.ndof):
            v = np.zeros(self.ndof)
            v[k] = 1.0
            A[:, k] = self.apply_A(v)
        return A

    def h1_error_exact(self, U):
        Ue, Ur = self.split(U)
        e1, n1 = self.ed.h1_error_exact(Ue)
        e2, n2 = self.cu.h1_parts(Ur)
        return np.sqrt((e1 + e2) / (n1 + n2))

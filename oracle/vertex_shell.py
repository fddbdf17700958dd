"""A vertex neighbourhood inside a spherical shell of curved regular elements,
joined on the sphere rho = rho_v (oracle, FP64).

Test infrastructure only (see the package docstring).

The vertex neighbourhood rho < rho_v (oracle/vertex.py, modified coordinates
(phi, theta, chi = ln rho)) and the regular region rho_v < rho < 1 in curved
shell elements (oracle/curved.py).  The functional is the sum of the two
regions' functionals, the sphere excluded from both, plus the terms of that
interface.

Reading of the interface (the thesis's sums run inside one region): the face
belongs to the singular side and takes the vertex neighbourhood's
interior-face terms (eq. 4.3: ||sqrt(R)[u]||_0^2 + sum_k ||sqrt(R)[u_{x_k^v}]||_{1/2}^2);
the regular side's physical gradient is converted there into the vertex's
modified derivatives by the chain rule of the spherical map:
u_phi = rho e_phi . grad u, u_theta = rho sin(phi) e_theta . grad u,
u_chi = rho e_rho . grad u.

Layout: the vertex elements, the shell elements, the vertex corner constant.
"""
from __future__ import annotations

import numpy as np

from .curved import CurvedDiscretisation
from .edge import l2_literal
from .vertex import VertexDiscretisation


class VertexShellDiscretisation:

    def __init__(self, vertex_problem, curved_problem, pairs):
        self.vd = VertexDiscretisation(vertex_problem)
        self.cu = CurvedDiscretisation(curved_problem)
        self.pairs = list(pairs)
        for e, j in self.pairs:
            self.vd.skip_faces.add((e, 5))
            self.cu.skip_faces.add((j, 4))
        self.nV, self.nR = int(self.vd.off[-1]), self.cu.ndof
        self.nC = self.vd.ndof - self.nV
        self.ndof = self.nV + self.nR + self.nC

    def split(self, U):
        return np.concatenate([U[:self.nV], U[self.nV + self.nR:]]), U[self.nV:self.nV + self.nR]

    def merge(self, yv, yr):
        return np.concatenate([yv[:self.nV], yr, yv[self.nV:]])

    def _Qf(self, e, j):
        return 2 * max(self.vd.W[e], self.cu.W[j]) + 1

    def _basis(self, j, Qf):
        """rho e_phi, rho sin(phi) e_theta, rho e_rho at the face points [3 vectors of 3 arrays]."""
        x, _ = self.cu.face_geom(j, 4, Qf)
        r = np.sqrt(x[0] ** 2 + x[1] ** 2 + x[2] ** 2)
        p = np.arccos(np.clip(x[2] / r, -1.0, 1.0))
        t = np.arctan2(x[1], x[0])
        sp, cp, st, ct = np.sin(p), np.cos(p), np.sin(t), np.cos(t)
        return [(r * cp * ct, r * cp * st, -r * sp), (-r * sp * st, r * sp * ct, 0 * r), (x[0], x[1], x[2])]

    def _jumps(self, Uv, Ur, e, j, Qf):
        fv = self.vd.face_fields(self.vd.block(Uv, e), e, 5, Qf)
        fr = self.cu.face_fields(self.cu.block(Ur, j), j, 4, Qf)
        B = self._basis(j, Qf)
        conv = [fr[0]] + [sum(B[a][i] * fr[i + 1] for i in range(3)) for a in range(3)]
        return [fv[k] - conv[k] for k in range(4)]

    def functional(self, U):
        Uv, Ur = self.split(U)
        R = self.vd.functional(Uv) + self.cu.functional(Ur)
        for e, j in self.pairs:
            Qf = self._Qf(e, j)
            J = self._jumps(Uv, Ur, e, j, Qf)
            _, _, t1, t2 = self.vd.face_axes(5)
            hh = self.vd.h(e) / 2.0
            c = self.vd.norm_weights(e, 5)
            R += self.vd.G(e, 5) * hh[t1] * hh[t2] * l2_literal(J[0], Qf)
            for k in range(1, 4):
                R += self.vd._norm_literal(J[k], Qf, c)
        return R

    def apply_A(self, U):
        Uv, Ur = self.split(U)
        yv, yr = self.vd.apply_A(Uv), self.cu.apply_A(Ur)
        for e, j in self.pairs:
            Qf = self._Qf(e, j)
            J = self._jumps(Uv, Ur, e, j, Qf)
            M = self.vd.jump_forms(e, 5, Qf)
            g = [(M[k] @ J[k].ravel()).reshape(Qf, Qf) for k in range(4)]
            yv[self.vd.off[e]:self.vd.off[e + 1]] += self.vd.face_fields_T(g, e, 5, Qf).ravel()
            B = self._basis(j, Qf)
            gr = [g[0]] + [sum(B[a][i] * g[a + 1] for a in range(3)) for i in range(3)]
            yr[self.cu.off[j]:self.cu.off[j + 1]] -= self.cu.face_fields_T(gr, j, 4, Qf).ravel()
        return self.merge(yv, yr)

    def rhs_b(self):
        return self.merge(self.vd.rhs_b(), self.cu.rhs_b())

    def h1_error_exact(self, U):
        Uv, Ur = self.split(U)
        e1, n1 = self.vd.h1_error_exact(Uv)
        e2, n2 = self.cu.h1_parts(Ur)
        return np.sqrt((e1 + e2) / (n1 + n2))

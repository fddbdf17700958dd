"""Regular elements with a curved map (oracle, FP64).

Test infrastructure only (see the package docstring).

Eq. (4.2) on regular elements Omega_l = M_l(Q), Q = (-1,1)^3, with an analytic
map M_l that need not be affine (the thesis's regular region next to a
neighbourhood, e.g. the polar blend of an L-shaped prism):

  R(u) = sum_l int_Q |L u_l(M_l(lambda)) - f|^2 |J_l| dlambda
       + sum_{interior faces} ( ||[u]||_0^2 + sum_k ||[u_{x_k}]||_{1/2}^2 )
       + sum_{Dirichlet faces} ||u_l - g||_{3/2}^2

with L u = -Lap u in physical coordinates.  With K = (dx/dlambda)^{-1}
(K_ai = d lambda_a / d x_i), the chain rule gives
  u_{x_i} = sum_a K_ai u_a,
  Lap u = sum_ab g^{ab} u_ab + sum_a (Lap lambda_a) u_a,
  g^{ab} = sum_i K_ai K_bi,
  Lap lambda_a = - sum_k K_ak sum_bc (d^2 x_k / d lambda_b d lambda_c) g^{bc}
(the second derivatives of the inverse map from those of the map).

Readings (those of oracle/functional.py carry over):

* Face norms in reference-face coordinates (no area Jacobian, eq. 2.17b);
  jumps of the physical gradient, each side through its own map, at the
  (2W+1)^2 GLL points of the reference face; the two sides of a face share
  its parametrisation (the meshes here are built that way).
* Dirichlet faces: ||u - g||_0^2 + sum_t ||d(u - g)/dlambda_t||_{1/2}^2
  (eq. 2.18) with the lambda-tangential derivative of g's interpolant.
* Data are pointwise functions of physical coordinates, f(x, y, z) on arrays
  of any (equal) shape.

A mesh gives, per element, map(l1, l2, l3) -> (x [3, ...], Dx [3, 3, ...]
(Dx[k, a] = d x_k / d lambda_a), D2x [3, 3, 3, ...] (d^2 x_k / d lambda_a
d lambda_b)) on broadcast arrays of reference coordinates.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from .functional import (_face_eval_mats, eval_tensor, eval_tensor_T, face_mats, h12_face_literal,
                         l2_face_literal, tables)
from .gll import diff_matrix, gll, lagrange_eval


@dataclass
class CurvedMesh:
    maps: List[Callable]
    elem_W: np.ndarray
    elem_nbr: np.ndarray          # [E, 6]: neighbour or -1 (Dirichlet)

    @property
    def n_elem(self) -> int:
        return len(self.maps)


@dataclass
class CurvedProblem:
    mesh: CurvedMesh
    f: Callable
    g: Callable
    u_exact: Optional[Callable] = None
    grad_exact: Optional[Callable] = None    # (u_x, u_y, u_z) pointwise
    meta: dict = field(default_factory=dict)


def _geometry(Dx, D2x):
    """K = Dx^{-1}, |det Dx|, g^{ab}, Lap lambda_a at every point ([..., 3, 3] layout)."""
    J = np.moveaxis(Dx, (0, 1), (-2, -1))            # [..., k, a]
    K = np.linalg.inv(J)                              # [..., a, k]
    det = np.abs(np.linalg.det(J))
    G = np.einsum("...ai,...bi->...ab", K, K)
    H = np.moveaxis(D2x, (0, 1, 2), (-3, -2, -1))    # [..., k, b, c]
    lap = -np.einsum("...ak,...kbc,...bc->...a", K, H, G)
    return K, det, G, lap


class CurvedDiscretisation:
    """Oracle discretisation of a CurvedProblem."""

    FIELDS = [((2, 0, 0), (0, 0)), ((0, 2, 0), (1, 1)), ((0, 0, 2), (2, 2)),
              ((1, 1, 0), (0, 1)), ((1, 0, 1), (0, 2)), ((0, 1, 1), (1, 2))]

    def __init__(self, problem):
        self.problem = problem
        m = problem.mesh
        self.mesh = m
        self.E = m.n_elem
        self.W = [int(w) for w in m.elem_W]
        self.P = [w + 1 for w in self.W]
        off = np.zeros(self.E + 1, dtype=np.int64)
        for e in range(self.E):
            off[e + 1] = off[e] + self.P[e] ** 3
        self.off = off
        self.ndof = int(off[-1])
        self._vol = {}
        # (element, face) pairs whose terms a composite discretisation owns
        self.skip_faces = set()

    def block(self, U, e):
        P = self.P[e]
        return U[self.off[e]:self.off[e + 1]].reshape(P, P, P)

    # --- volume ------------------------------------------------------------
    def vol_geom(self, e):
        """x, K, |J|, g^{ab}, Lap lambda at the (2W+1)^3 GLL points [c, b, a]."""
        if e not in self._vol:
            xq = tables(self.W[e])["xq"]
            l3, l2, l1 = np.meshgrid(xq, xq, xq, indexing="ij")
            x, Dx, D2x = self.mesh.maps[e](l1, l2, l3)
            self._vol[e] = (x,) + _geometry(Dx, D2x)
        return self._vol[e]

    def vol_weight(self, e):
        wq = tables(self.W[e])["wq"]
        _, _, det, _, _ = self.vol_geom(e)
        return wq[:, None, None] * wq[None, :, None] * wq[None, None, :] * det

    def _terms(self, e):
        B = tables(self.W[e])["B"]
        _, _, _, G, lap = self.vol_geom(e)
        out = []
        for order, (a, b) in self.FIELDS:
            coef = -(1.0 if a == b else 2.0) * G[..., a, b]
            out.append((coef, B[order[0]], B[order[1]], B[order[2]]))
        for a in range(3):
            order = [0, 0, 0]
            order[a] = 1
            out.append((-lap[..., a], B[order[0]], B[order[1]], B[order[2]]))
        return out

    def L_apply(self, u, e):
        """-Lap u at the volume points by the chain rule through the map."""
        return sum(c * eval_tensor(u, Mx, My, Mz) for c, Mx, My, Mz in self._terms(e))

    def L_apply_T(self, r, e):
        return sum(eval_tensor_T(c * r, Mx, My, Mz) for c, Mx, My, Mz in self._terms(e))

    def f_at(self, e):
        x = self.vol_geom(e)[0]
        return self.problem.f(x[0], x[1], x[2])

    # --- faces ---------------------------------------------------------------
    @staticmethod
    def face_axes(fi):
        axis, side = fi // 2, fi % 2
        t1, t2 = [a for a in range(3) if a != axis]
        return axis, side, t1, t2

    def Qf(self, e, fi):
        n = int(self.mesh.elem_nbr[e, fi])
        return 2 * (self.W[e] if n < 0 else max(self.W[e], self.W[n])) + 1

    def face_geom(self, e, fi, Qf):
        """x and K at the face's GLL points, arrays [t2, t1, ...]."""
        axis, side, t1, t2 = self.face_axes(fi)
        xf, _ = gll(Qf)
        lam = [None, None, None]
        lam[t2], lam[t1] = np.meshgrid(xf, xf, indexing="ij")
        lam[axis] = np.full((Qf, Qf), -1.0 if side == 0 else 1.0)
        x, Dx, D2x = self.mesh.maps[e](lam[0], lam[1], lam[2])
        K, _, _, _ = _geometry(Dx, D2x)
        return x, K

    def face_eval(self, u, e, fi, Qf, orders):
        Mx, My, Mz = _face_eval_mats(self.P[e], fi, Qf, tuple(orders))
        return eval_tensor(u, Mx, My, Mz).reshape(Qf, Qf)

    def face_eval_T(self, g, e, fi, Qf, orders):
        axis = fi // 2
        Mx, My, Mz = _face_eval_mats(self.P[e], fi, Qf, tuple(orders))
        shape = [Qf, Qf, Qf]
        shape[2 - axis] = 1
        return eval_tensor_T(g.reshape(shape), Mx, My, Mz)

    @staticmethod
    def _unit(a):
        o = [0, 0, 0]
        o[a] = 1
        return tuple(o)

    def face_fields(self, u, e, fi, Qf):
        """u and the physical gradient u_{x_i} = sum_a K_ai u_a on the face."""
        _, K = self.face_geom(e, fi, Qf)
        ua = [self.face_eval(u, e, fi, Qf, self._unit(a)) for a in range(3)]
        out = [self.face_eval(u, e, fi, Qf, (0, 0, 0))]
        for i in range(3):
            out.append(sum(K[..., a, i] * ua[a] for a in range(3)))
        return out

    def face_fields_T(self, gs, e, fi, Qf):
        _, K = self.face_geom(e, fi, Qf)
        y = self.face_eval_T(gs[0], e, fi, Qf, (0, 0, 0))
        for a in range(3):
            y = y + self.face_eval_T(sum(K[..., a, i] * gs[i + 1] for i in range(3)), e, fi, Qf, self._unit(a))
        return y

    def dirichlet_samples(self, u, e, fi, Qf):
        _, _, t1, t2 = self.face_axes(fi)
        return [self.face_eval(u, e, fi, Qf, (0, 0, 0)), self.face_eval(u, e, fi, Qf, self._unit(t1)),
                self.face_eval(u, e, fi, Qf, self._unit(t2))]

    def dirichlet_samples_T(self, gs, e, fi, Qf):
        _, _, t1, t2 = self.face_axes(fi)
        return (self.face_eval_T(gs[0], e, fi, Qf, (0, 0, 0)) + self.face_eval_T(gs[1], e, fi, Qf, self._unit(t1)) +
                self.face_eval_T(gs[2], e, fi, Qf, self._unit(t2)))

    def dirichlet_data(self, e, fi, Qf):
        x, _ = self.face_geom(e, fi, Qf)
        gv = self.problem.g(x[0], x[1], x[2])
        xf, _ = gll(Qf)
        D = diff_matrix(xf)
        return [gv, gv @ D.T, D @ gv]

    # --- the functional (literal norm sums) and the normal operator ----------
    def functional(self, U):
        R = 0.0
        for e in range(self.E):
            z = np.sqrt(self.vol_weight(e)) * (self.L_apply(self.block(U, e), e) - self.f_at(e))
            R += float(np.sum(z * z))
        for e in range(self.E):
            u = self.block(U, e)
            for fi in range(6):
                if (e, fi) in self.skip_faces:
                    continue
                n = int(self.mesh.elem_nbr[e, fi])
                Qf = self.Qf(e, fi)
                if n >= 0:
                    if n < e:
                        continue
                    fe = self.face_fields(u, e, fi, Qf)
                    fn = self.face_fields(self.block(U, n), n, fi ^ 1, Qf)
                    R += l2_face_literal(fe[0] - fn[0], Qf)
                    for k in range(1, 4):
                        R += h12_face_literal(fe[k] - fn[k], Qf)
                else:
                    sm = self.dirichlet_samples(u, e, fi, Qf)
                    dd = self.dirichlet_data(e, fi, Qf)
                    R += l2_face_literal(sm[0] - dd[0], Qf)
                    R += h12_face_literal(sm[1] - dd[1], Qf) + h12_face_literal(sm[2] - dd[2], Qf)
        return R

    def element_apply(self, U, e):
        u = self.block(U, e)
        y = self.L_apply_T(self.vol_weight(e) * self.L_apply(u, e), e)
        for fi in range(6):
            if (e, fi) in self.skip_faces:
                continue
            n = int(self.mesh.elem_nbr[e, fi])
            Qf = self.Qf(e, fi)
            W2, H = face_mats(Qf)
            if n >= 0:
                fe = self.face_fields(u, e, fi, Qf)
                fn = self.face_fields(self.block(U, n), n, fi ^ 1, Qf)
                gs = [(W2 @ (fe[0] - fn[0]).ravel()).reshape(Qf, Qf)]
                gs += [(H @ (fe[k] - fn[k]).ravel()).reshape(Qf, Qf) for k in range(1, 4)]
                y = y + self.face_fields_T(gs, e, fi, Qf)
            else:
                sm = self.dirichlet_samples(u, e, fi, Qf)
                gs = [(W2 @ sm[0].ravel()).reshape(Qf, Qf), (H @ sm[1].ravel()).reshape(Qf, Qf),
                      (H @ sm[2].ravel()).reshape(Qf, Qf)]
                y = y + self.dirichlet_samples_T(gs, e, fi, Qf)
        return y.ravel()

    def apply_A(self, U):
        y = np.zeros(self.ndof)
        for e in range(self.E):
            y[self.off[e]:self.off[e + 1]] = self.element_apply(U, e)
        return y

    def rhs_b(self):
        b = np.zeros(self.ndof)
        for e in range(self.E):
            y = self.L_apply_T(self.vol_weight(e) * self.f_at(e), e)
            for fi in range(6):
                if int(self.mesh.elem_nbr[e, fi]) >= 0 or (e, fi) in self.skip_faces:
                    continue
                Qf = self.Qf(e, fi)
                W2, H = face_mats(Qf)
                dd = self.dirichlet_data(e, fi, Qf)
                gs = [(W2 @ dd[0].ravel()).reshape(Qf, Qf), (H @ dd[1].ravel()).reshape(Qf, Qf),
                      (H @ dd[2].ravel()).reshape(Qf, Qf)]
                y = y + self.dirichlet_samples_T(gs, e, fi, Qf)
            b[self.off[e]:self.off[e + 1]] = y.ravel()
        return b

    def dense_A(self):
        A = np.zeros((self.ndof, self.ndof))
        for j in range(self.ndof):
            v = np.zeros(self.ndof)
            v[j] = 1.0
            A[:, j] = self.apply_A(v)
        return A

    def nodal_interpolant(self, fun):
        U = np.zeros(self.ndof)
        for e in range(self.E):
            xp, _ = gll(self.P[e])
            l3, l2, l1 = np.meshgrid(xp, xp, xp, indexing="ij")
            x, _, _ = self.mesh.maps[e](l1, l2, l3)
            U[self.off[e]:self.off[e + 1]] = fun(x[0], x[1], x[2]).ravel()
        return U

    def h1_error_exact(self, U, nq=20):
        """Relative H^1 error against the problem's exact solution."""
        err, nrm = self.h1_parts(U, nq)
        return np.sqrt(err / nrm)

    def h1_parts_gll(self, U):
        """(||u_h - w||_{H^1}^2, ||w||_{H^1}^2) with each element's own
        (2W+1)^3 GLL rule in lambda times |J| (the rule of the volume term)."""
        err = nrm = 0.0
        for e in range(self.E):
            B0, B1 = tables(self.W[e])["B"][:2]
            wq = tables(self.W[e])["wq"]
            u = self.block(U, e)
            x, K, det, _, _ = self.vol_geom(e)
            v = eval_tensor(u, B0, B0, B0)
            va = [eval_tensor(u, *[B1 if b == a else B0 for b in range(3)]) for a in range(3)]
            w = self.problem.u_exact(x[0], x[1], x[2])
            gw = self.problem.grad_exact(x[0], x[1], x[2])
            d2 = (v - w) ** 2
            n2 = w ** 2
            for i in range(3):
                vi = sum(K[..., a, i] * va[a] for a in range(3))
                d2 = d2 + (vi - gw[i]) ** 2
                n2 = n2 + gw[i] ** 2
            wt = wq[:, None, None] * wq[None, :, None] * wq[None, None, :] * det
            err += float(np.sum(wt * d2))
            nrm += float(np.sum(wt * n2))
        return err, nrm

    def h1_parts(self, U, nq=20):
        """(||u_h - w||_{H^1}^2, ||w||_{H^1}^2), each element by an nq^3
        Gauss-Legendre rule in lambda times |J|."""
        xg, wg = np.polynomial.legendre.leggauss(nq)
        l3, l2, l1 = np.meshgrid(xg, xg, xg, indexing="ij")
        wq = wg[:, None, None] * wg[None, :, None] * wg[None, None, :]
        err = nrm = 0.0
        for e in range(self.E):
            xp, _ = gll(self.P[e])
            B = [lagrange_eval(xp, xg, d) for d in range(2)]
            u = self.block(U, e)
            x, Dx, D2x = self.mesh.maps[e](l1, l2, l3)
            K, det, _, _ = _geometry(Dx, D2x)
            v = eval_tensor(u, B[0], B[0], B[0])
            va = [eval_tensor(u, *[B[1] if b == a else B[0] for b in range(3)]) for a in range(3)]
            w = self.problem.u_exact(x[0], x[1], x[2])
            gw = self.problem.grad_exact(x[0], x[1], x[2])
            d2 = (v - w) ** 2
            n2 = w ** 2
            for i in range(3):
                vi = sum(K[..., a, i] * va[a] for a in range(3))
                d2 = d2 + (vi - gw[i]) ** 2
                n2 = n2 + gw[i] ** 2
            err += float(np.sum(wq * det * d2))
            nrm += float(np.sum(wq * det * n2))
        return err, nrm

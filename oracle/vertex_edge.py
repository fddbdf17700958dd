"""Vertex-edge-neighbourhood least-squares functional in modified coordinates (oracle, FP64).

Test infrastructure only (see the package docstring).

Section 2.3 / Section 4.2: where an edge on the x3 axis leaves a vertex at
the origin, the modified coordinates are x^{v-e} = (psi, theta, zeta) with
psi = ln tan phi and zeta = ln x3 (so r = e^{psi + zeta}, x3 = e^zeta), and
the geometric mesh in phi and in x3 makes every element a box in x^{v-e}.
Eq. (2.29) (eq. 4.5 for the functional of the method) gives, for -Lap u = f,

  R_ve(u) = sum_{finite l} int |L^{v-e} u_l - F^{v-e}|^2 dx^{v-e}
          + sum_{interior faces, finite measure} ( ||sqrt(F G) [u]||_0^2 + |||[u_psi]|||^2
                                                  + |||[u_theta]|||^2 + |||E [u_zeta]|||^2 )
          + sum_{Dirichlet faces, finite measure} ( ||sqrt(F) (u - g)||_0^2 + |||(u - g)_t|||^2 ... )

with E = sup_face sin phi, F = sup_face e^zeta, G = E on the faces
zeta = const and 1 otherwise, and the anisotropic face norm of eq. (2.27):
on zeta = const  E F (L2 + psi-difference quotient + theta-difference quotient),
on psi = const   F (L2 + theta-DQ + E zeta-DQ),
on theta = const F (L2 + psi-DQ + E zeta-DQ).
L^{v-e} is the operator with int |L^{v-e} u|^2 dx^{v-e} = int rho^2 sin^2(phi) |L u|^2 dx
(eq. 2.28).  For the Laplacian, with rho sin phi = r and
dx = r^2 x3 dx^{v-e} = e^{2 psi + 3 zeta} dx^{v-e}:
  r^2 Lap u = u_psipsi + u_thetatheta + e^{2 psi} (u_psipsi - 2 u_psizeta + u_zetazeta + u_psi - u_zeta),
  L^{v-e} u = -e^{zeta/2} r^2 Lap u,   F^{v-e} = e^{zeta/2} r^2 f.
Corner sets: for each zeta layer the elements psi < psi_1 hold one polynomial
in zeta shared by every theta sector (their face psi = psi_1 with psi layer 1
is finite; the rest is infinite); the elements zeta < zeta_1 hold the vertex
constant h_v (their face zeta = zeta_1 with zeta layer 1 is finite).

Readings (in addition to those of oracle/edge.py that carry over):

* Axes (x, y, z) = (psi, theta, zeta); every finite element has degree W in
  each modified coordinate (the thesis's (W_q, W_q, V_q) with both equal to
  W), each zeta-polynomial corner set degree W.
* Norm integrals in modified coordinates as for the edge: on a face with
  tangential half-lengths h1, h2 the L2 term carries h1 h2, the difference
  quotient along t1 (t2) carries h2 (h1).
* Dirichlet faces: ||sqrt(F) (u - g)||_0^2 plus |||.|||^2 of the derivatives
  of u - g along the face's two tangential modified coordinates, the zeta
  derivative multiplied by E (eq. 2.29 writes u_psi and E u_zeta, the
  tangential derivatives of the faces theta = const; on the outer faces
  psi = const and zeta = const the same rule takes their own tangential
  derivatives).
* Data are functions of the modified coordinates on tensor grids,
  fun(psis, thetas, zetas) -> [len zetas, len thetas, len psis].

Layout: the finite elements' (W+1)^3 nodal blocks (psi fastest) in element
order, then the corner sets in order: a zeta polynomial's W+1 nodal values,
the constant's one value.
"""
from __future__ import annotations

import numpy as np

from .edge import EdgeDiscretisation, face_form, l2_literal
from .functional import eval_tensor, eval_tensor_T, tables
from .gll import diff_matrix, gll, lagrange_eval


def sin_of_psi(psi):
    """sin phi for psi = ln tan phi (0 < phi < pi / 2)."""
    return 1.0 / np.sqrt(1.0 + np.exp(-2.0 * np.asarray(psi)))


class VertexEdgeDiscretisation(EdgeDiscretisation):
    """Oracle discretisation of a vertex-edge workloads.EdgeProblem (kind "vertex-edge")."""

    def __init__(self, problem):
        super().__init__(problem)
        # the face of layer 1 through which each corner set enters: 0 (a zeta
        # polynomial on psi = psi_1) or 4 (the constant on zeta = zeta_1)
        self.cface = []
        for c in range(self.C):
            f0 = any(int(self.mesh.elem_nbr[e, 0]) == -2 - c for e in range(self.E))
            self.cface.append(0 if f0 else 4)

    # --- volume term (eq. 2.28) -------------------------------------------
    def _coefs(self, e):
        """e^{zeta/2} [zeta, 1, 1] and e^{2 psi} [1, 1, psi] at the Q points."""
        psis, _, zets = self.qpoints(e)
        return np.exp(0.5 * zets)[:, None, None], np.exp(2.0 * psis)[None, None, :]

    def _terms(self, e):
        """(coefficient, x, y, z matrices) of each term of r^2 Lap u."""
        B0, B1, B2 = tables(self.W[e])["B"]
        s = self.scale(e)
        _, k = self._coefs(e)
        return [((1.0 + k) * s[0] ** 2, B2, B0, B0),
                (s[1] ** 2, B0, B2, B0),
                (k * s[2] ** 2, B0, B0, B2),
                (-2.0 * k * s[0] * s[2], B1, B0, B1),
                (k * s[0], B1, B0, B0),
                (-k * s[2], B0, B0, B1)]

    def L_apply(self, u, e):
        c, _ = self._coefs(e)
        return -c * sum(a * eval_tensor(u, Bx, By, Bz) for a, Bx, By, Bz in self._terms(e))

    def L_apply_T(self, r, e):
        c, _ = self._coefs(e)
        cr = -c * r
        return sum(eval_tensor_T(a * cr, Bx, By, Bz) for a, Bx, By, Bz in self._terms(e))

    def f_at(self, e, rhs):
        """F^{v-e} = e^{zeta/2} r^2 f at the volume points."""
        psis, ths, zets = self.qpoints(e)
        c, _ = self._coefs(e)
        r2 = np.exp(2.0 * (psis[None, None, :] + zets[:, None, None]))
        return c * r2 * self.problem.f[rhs](psis, ths, zets)

    # --- faces (eq. 2.27, 2.29) ---------------------------------------------
    def _face_sup(self, e, fi, axis_of):
        axis, side, _, _ = self.face_axes(fi)
        if axis == axis_of and side == 0:
            return float(self.mesh.elem_lo[e, axis_of])
        return float(self.mesh.elem_hi[e, axis_of])

    def E_sup(self, e, fi):
        """sup over the face of sin phi (increasing in psi)."""
        return float(sin_of_psi(self._face_sup(e, fi, 0)))

    def F_sup(self, e, fi):
        """sup over the face of e^zeta."""
        return float(np.exp(self._face_sup(e, fi, 2)))

    def norm_weights(self, e, fi):
        axis, _, t1, t2 = self.face_axes(fi)
        hh = self.h(e) / 2.0
        E, F = self.E_sup(e, fi), self.F_sup(e, fi)
        c = [F * hh[t1] * hh[t2], F * hh[t2], F * hh[t1]]
        if t1 == 2:
            c[1] *= E
        if t2 == 2:
            c[2] *= E
        if axis == 2:
            c = [E * v for v in c]
        return tuple(c)

    def _u_weight(self, e, fi, dirichlet):
        axis, _, t1, t2 = self.face_axes(fi)
        hh = self.h(e) / 2.0
        G = self.E_sup(e, fi) if (axis == 2 and not dirichlet) else 1.0
        return self.F_sup(e, fi) * G * hh[t1] * hh[t2]

    def jump_forms(self, e, fi, Qf):
        """Face matrices of [u], [u_psi], [u_theta], E [u_zeta]."""
        E = self.E_sup(e, fi)
        Mk = face_form(Qf, *self.norm_weights(e, fi))
        return [face_form(Qf, self._u_weight(e, fi, False), 0.0, 0.0), Mk, Mk, E * E * Mk]

    def dirichlet_forms(self, e, fi, Qf):
        _, _, t1, t2 = self.face_axes(fi)
        E = self.E_sup(e, fi)
        Mk = face_form(Qf, *self.norm_weights(e, fi))
        return [face_form(Qf, self._u_weight(e, fi, True), 0.0, 0.0),
                (E * E if t1 == 2 else 1.0) * Mk, (E * E if t2 == 2 else 1.0) * Mk]

    def corner_fields(self, p, c, e, Qf):
        """Corner fields on the face with layer-1 element e: a zeta polynomial on
        psi = psi_1 (face 0, grid [zeta (t2), theta (t1)]): p, 0, 0, p_zeta; the
        constant on zeta = zeta_1: p, 0, 0, 0."""
        z = np.zeros((Qf, Qf))
        if self.cface[c] == 4:
            return [np.full((Qf, Qf), float(p[0])), z, z, z]
        B0z, B1z = self._corner_mats(c, Qf)
        s3 = self.scale(e)[2]
        one = np.ones(Qf)
        return [np.outer(B0z @ p, one), z, z, s3 * np.outer(B1z @ p, one)]

    def corner_fields_T(self, gs, c, e, Qf):
        if self.cface[c] == 4:
            return np.array([gs[0].sum()])
        B0z, B1z = self._corner_mats(c, Qf)
        s3 = self.scale(e)[2]
        return B0z.T @ gs[0].sum(axis=1) + s3 * (B1z.T @ gs[3].sum(axis=1))

    def dirichlet_data(self, e, fi, Qf, rhs):
        _, _, t1, t2 = self.face_axes(fi)
        psis, ths, zets = self.face_points(e, fi, Qf)
        gv = self.problem.g[rhs](psis, ths, zets).reshape(Qf, Qf)
        xf, _ = gll(Qf)
        D = diff_matrix(xf)
        s = self.scale(e)
        return [gv, s[t1] * (gv @ D.T), s[t2] * (D @ gv)]

    # --- the functional (literal norm sums, eq. 2.29) -----------------------
    def functional(self, U, rhs=0):
        R = 0.0
        for e in range(self.E):
            u = self.block(U, e)
            z = np.sqrt(self.vol_weight(e)) * (self.L_apply(u, e) - self.f_at(e, rhs))
            R += float(np.sum(z * z))
        for e in range(self.E):
            u = self.block(U, e)
            for fi in range(6):
                if (e, fi) in self.skip_faces:
                    continue
                Qf = self.Qf(e, fi)
                n = int(self.mesh.elem_nbr[e, fi])
                _, _, t1, t2 = self.face_axes(fi)
                E = self.E_sup(e, fi)
                c = self.norm_weights(e, fi)
                if n == -1:
                    sm = self.dirichlet_samples(u, e, fi, Qf)
                    dd = self.dirichlet_data(e, fi, Qf, rhs)
                    R += self._u_weight(e, fi, True) * l2_literal(sm[0] - dd[0], Qf)
                    R += (E * E if t1 == 2 else 1.0) * self._norm_literal(sm[1] - dd[1], Qf, c)
                    R += (E * E if t2 == 2 else 1.0) * self._norm_literal(sm[2] - dd[2], Qf, c)
                    continue
                if n >= 0 and n < e:
                    continue
                fe = self.face_fields(u, e, fi, Qf)
                if n >= 0:
                    fn = self.face_fields(self.block(U, n), n, fi ^ 1, Qf)
                else:
                    fn = self.corner_fields(self.corner(U, -2 - n), -2 - n, e, Qf)
                R += self._u_weight(e, fi, False) * l2_literal(fe[0] - fn[0], Qf)
                R += self._norm_literal(fe[1] - fn[1], Qf, c)
                R += self._norm_literal(fe[2] - fn[2], Qf, c)
                R += E * E * self._norm_literal(fe[3] - fn[3], Qf, c)
        return R

    def corner_apply(self, U, c):
        p = self.corner(U, c)
        y = np.zeros_like(p)
        f = self.cface[c]
        for e in range(self.E):
            if int(self.mesh.elem_nbr[e, f]) != -2 - c:
                continue
            Qf = self.Qf(e, f)
            fe = self.face_fields(self.block(U, e), e, f, Qf)
            fn = self.corner_fields(p, c, e, Qf)
            M = self.jump_forms(e, f, Qf)
            gs = [(M[k] @ (fn[k] - fe[k]).ravel()).reshape(Qf, Qf) for k in range(4)]
            y = y + self.corner_fields_T(gs, c, e, Qf)
        return y

    def nodal_interpolant(self, fun):
        """fun(psi, theta, zeta) on every finite element's nodes; a zeta
        polynomial takes fun on psi = psi_1 at theta of its first sector, the
        constant takes fun at the centre of its first face zeta = zeta_1."""
        U = np.zeros(self.ndof)
        for e in range(self.E):
            xp, _ = gll(self.P[e])
            ps, ts, zs = (self.coord(e, a, xp) for a in range(3))
            U[self.off[e]:self.off[e + 1]] = fun(ps, ts, zs).ravel()
        for c in range(self.C):
            f = self.cface[c]
            e = next(e for e in range(self.E) if int(self.mesh.elem_nbr[e, f]) == -2 - c)
            lo, hi = self.mesh.elem_lo[e], self.mesh.elem_hi[e]
            if f == 4:
                U[self.coff[c]] = float(fun(np.array([0.5 * (lo[0] + hi[0])]), np.array([0.5 * (lo[1] + hi[1])]),
                                            np.array([lo[2]])).ravel()[0])
            else:
                xp, _ = gll(self.Wc[c] + 1)
                zs = lo[2] + (xp + 1.0) * (hi[2] - lo[2]) / 2.0
                U[self.coff[c]:self.coff[c] + self.Wc[c] + 1] = fun(lo[0:1], lo[1:2], zs).ravel()
        return U

    # --- H^1 error in physical coordinates (Section 6.1) -------------------
    def h1_error_exact(self, U, nq=24):
        """(||u_h - w||_{H^1}^2, ||w||_{H^1}^2) over the vertex-edge neighbourhood.

        Finite elements: Gauss-Legendre in (psi, theta, zeta) with
        dx = e^{2 psi + 3 zeta} dx^{v-e}; with v_psi = r v_r and
        v_zeta = r v_r + x3 v_x3 the physical gradient is
        (v_psi / r, v_theta / r, (v_zeta - v_psi) / x3).
        Corner sets: a zeta polynomial on psi < psi_1 of its zeta layer and
        sector, integrated in (s, theta, zeta) with r = x3 e^{psi_1} s^3; the
        constant on x3 < x3_1 inside the cone psi < psi_top, integrated in
        (s, theta, t) with e^psi = e^{psi_top} s^3 and x3 = x3_1 t^3 (both
        substitutions make the singular integrands smooth)."""
        w_fun, gw = self.problem.u_exact, self.problem.grad_exact
        xg, wg = np.polynomial.legendre.leggauss(nq)
        err = nrm = 0.0
        for e in range(self.E):
            xp, _ = gll(self.P[e])
            B = [lagrange_eval(xp, xg, d) for d in range(2)]
            lo, hh = self.mesh.elem_lo[e], self.h(e) / 2.0
            ps, ts, zs = (lo[a] + (xg + 1.0) * hh[a] for a in range(3))
            u = self.block(U, e)
            s = self.scale(e)
            v = eval_tensor(u, B[0], B[0], B[0])
            vp = s[0] * eval_tensor(u, B[1], B[0], B[0])
            vt = s[1] * eval_tensor(u, B[0], B[1], B[0])
            vz = s[2] * eval_tensor(u, B[0], B[0], B[1])
            r = np.exp(ps[None, None, :] + zs[:, None, None])
            x3 = np.exp(zs)[:, None, None]
            wv = w_fun(ps, ts, zs)
            wr, wth, wz = gw(ps, ts, zs)
            dx = wg[:, None, None] * wg[None, :, None] * wg[None, None, :] * float(np.prod(hh)) * r * r * x3
            err += float(np.sum(dx * ((v - wv) ** 2 + (vp / r - wr) ** 2 + (vt / r - wth) ** 2 +
                                      ((vz - vp) / x3 - wz) ** 2)))
            nrm += float(np.sum(dx * (wv ** 2 + wr ** 2 + wth ** 2 + wz ** 2)))
        sg = (xg + 1.0) / 2.0
        for c in range(self.C):
            f = self.cface[c]
            pc = self.corner(U, c)
            for e in range(self.E):
                if int(self.mesh.elem_nbr[e, f]) != -2 - c:
                    continue
                lo, hi, hh = self.mesh.elem_lo[e], self.mesh.elem_hi[e], self.h(e) / 2.0
                ts = lo[1] + (xg + 1.0) * hh[1]
                if f == 0:
                    # r = x3 e^{psi_1} s^3: psi = psi_1 + 3 ln s; dr = 3 x3 e^{psi_1} s^2 ds
                    zs = lo[2] + (xg + 1.0) * hh[2]
                    ps = lo[0] + 3.0 * np.log(sg)
                    x3 = np.exp(zs)[:, None, None]
                    r = x3 * np.exp(ps)[None, None, :]
                    dr = 3.0 * x3 * np.exp(lo[0]) * (sg ** 2)[None, None, :] * 0.5
                    dx = (wg * hh[2])[:, None, None] * (wg * hh[1])[None, :, None] * wg[None, None, :] * r * dr * x3
                    xp, _ = gll(self.Wc[c] + 1)
                    uz = (lagrange_eval(xp, xg, 0) @ pc)[:, None, None]
                    udz = ((2.0 / (hi[2] - lo[2])) * (lagrange_eval(xp, xg, 1) @ pc))[:, None, None] / x3
                    wv = w_fun(ps, ts, zs)
                    wr, wth, wz = gw(ps, ts, zs)
                    err += float(np.sum(dx * ((uz - wv) ** 2 + wr ** 2 + wth ** 2 + (udz - wz) ** 2)))
                else:
                    # the cone psi < psi_top = sup psi of this theta sector's elements
                    ptop = max(float(self.mesh.elem_hi[q, 0]) for q in range(self.E)
                               if int(self.mesh.elem_nbr[q, 4]) == -2 - c and
                               abs(self.mesh.elem_lo[q, 1] - lo[1]) < 1e-14)
                    if abs(hi[0] - ptop) > 1e-14:
                        continue  # one integral per theta sector
                    x31 = float(np.exp(lo[2]))
                    ps = ptop + 3.0 * np.log(sg)
                    zs = lo[2] + 3.0 * np.log(sg)
                    x3 = np.exp(zs)[:, None, None]
                    r = x3 * np.exp(ps)[None, None, :]
                    dr = 3.0 * x3 * np.exp(ptop) * (sg ** 2)[None, None, :] * 0.5
                    dx3 = (3.0 * x31 * sg ** 2 * 0.5)[:, None, None]
                    dx = (wg[:, None, None] * dx3) * (wg * hh[1])[None, :, None] * wg[None, None, :] * r * dr
                    wv = w_fun(ps, ts, zs)
                    wr, wth, wz = gw(ps, ts, zs)
                    err += float(np.sum(dx * ((float(pc[0]) - wv) ** 2 + wr ** 2 + wth ** 2 + wz ** 2)))
                nrm += float(np.sum(dx * (wv ** 2 + wr ** 2 + wth ** 2 + wz ** 2)))
        return err, nrm


def h1_diff(disc, U, V):
    """(||u_h - v_h||_{H^1}^2, ||v_h||_{H^1}^2) of two discrete solutions on a
    vertex-edge neighbourhood, in physical coordinates (Section 6.1).

    Finite elements in (psi, theta, zeta), r = e^{psi + zeta}, x3 = e^zeta:
    dx = r^2 x3 dpsi dtheta dzeta and the physical gradient is
    (v_psi / r, v_theta / r, (v_zeta - v_psi) / x3), by the element's
    (2W+1)-point GLL rule.  Corner sets: the zeta polynomial p on psi < psi_1
    of its layer and sector, exactly in r (int_0^{x3 e^{psi_1}} r dr =
    x3^2 e^{2 psi_1} / 2) with its own (2W+1)-point GLL rule in zeta:
    (e^{2 psi_1} / 2) (e^{3 zeta} p^2 + e^zeta p_zeta^2) per unit theta; the
    constant on x3 < x3_1 inside the cone psi < psi_top of each theta sector,
    exactly: p^2 theta-span e^{2 psi_top} / 2 x3_1^3 / 3."""
    out = []
    for X in (U - V, V):
        tot = 0.0
        for e in range(disc.E):
            xp, _ = gll(disc.P[e])
            xg, wg = gll(2 * disc.W[e] + 1)
            B = [lagrange_eval(xp, xg, d) for d in range(2)]
            lo, hh = disc.mesh.elem_lo[e], disc.h(e) / 2.0
            ps = lo[0] + (xg + 1.0) * hh[0]
            zs = lo[2] + (xg + 1.0) * hh[2]
            s = disc.scale(e)
            u = disc.block(X, e)
            v = eval_tensor(u, B[0], B[0], B[0])
            vp = s[0] * eval_tensor(u, B[1], B[0], B[0])
            vt = s[1] * eval_tensor(u, B[0], B[1], B[0])
            vz = s[2] * eval_tensor(u, B[0], B[0], B[1])
            r = np.exp(ps[None, None, :] + zs[:, None, None])
            x3 = np.exp(zs)[:, None, None]
            dx = wg[:, None, None] * wg[None, :, None] * wg[None, None, :] * float(np.prod(hh)) * r * r * x3
            tot += float(np.sum(dx * (v * v + (vp * vp + vt * vt) / (r * r) + (vz - vp) ** 2 / (x3 * x3))))
        for c in range(disc.C):
            f = disc.cface[c]
            p = disc.corner(X, c)
            done = set()
            for e in range(disc.E):
                if int(disc.mesh.elem_nbr[e, f]) != -2 - c:
                    continue
                lo, hi = disc.mesh.elem_lo[e], disc.mesh.elem_hi[e]
                th = hi[1] - lo[1]
                if f == 0:
                    xp, _ = gll(disc.Wc[c] + 1)
                    xg, wg = gll(2 * disc.Wc[c] + 1)
                    hz = hi[2] - lo[2]
                    zs = lo[2] + (xg + 1.0) * hz / 2.0
                    p0 = lagrange_eval(xp, xg, 0) @ p
                    pz = (2.0 / hz) * (lagrange_eval(xp, xg, 1) @ p)
                    ez = np.exp(zs)
                    tot += 0.5 * np.exp(2.0 * lo[0]) * th * 0.5 * hz * float(
                        np.sum(wg * (ez ** 3 * p0 * p0 + ez * pz * pz)))
                else:
                    key = round(float(lo[1]), 12)
                    if key in done:
                        continue
                    done.add(key)
                    ptop = max(float(disc.mesh.elem_hi[q, 0]) for q in range(disc.E)
                               if int(disc.mesh.elem_nbr[q, f]) == -2 - c and abs(disc.mesh.elem_lo[q, 1] - lo[1]) < 1e-14)
                    x31 = float(np.exp(lo[2]))
                    tot += float(p[0]) ** 2 * th * 0.5 * np.exp(2.0 * ptop) * x31 ** 3 / 3.0
        out.append(tot)
    return tuple(out)

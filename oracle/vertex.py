"""Vertex-neighbourhood least-squares functional in modified coordinates (oracle, FP64).

Test infrastructure only (see the package docstring).

Section 2.3 / Section 4.2: around a vertex at the origin the modified
coordinates are x^v = (phi, theta, chi) with chi = ln rho (spherical
coordinates), and the geometric mesh makes every element a box in x^v.
Eq. (4.3) gives, for -Lap u = f,

  R_v(u) = sum_{finite l} int |L^v u_l - F^v|^2 dx^v
         + sum_{interior faces, finite measure} ( ||sqrt(R) [u]||_0^2 + sum_k ||sqrt(R) [u_{x_k}]||_{1/2}^2 )
         + sum_{Dirichlet faces, finite measure} ||sqrt(R) (u - g)||_{3/2}^2

with R = sup_face e^chi, F^v = e^{5 chi / 2} sqrt(sin phi) f, and L^v the
operator with int |L^v u|^2 dx^v = int rho^2 |L u|^2 dx: for the Laplacian,
rho^2 Lap u = u_chichi + u_chi + u_phiphi + cot(phi) u_phi + u_thetatheta / sin^2 phi
and dx = e^{3 chi} sin(phi) dx^v, so
L^v u = -e^{chi / 2} sqrt(sin phi) (u_chichi + u_chi + u_phiphi + cot(phi) u_phi + u_thetatheta / sin^2 phi).
The corner elements chi < ln rho_1 hold one constant shared by every
(phi, theta) sector (Section 4.2: u^v_l = h_v); their volume and their other
faces have infinite measure, so they enter only through the faces
chi = ln rho_1 with layer 1.

Readings (in addition to those of oracle/edge.py that carry over):

* Axes (x, y, z) = (phi, theta, chi); every finite element has degree W in
  each modified coordinate.
* Norms are integrals in the modified coordinates: on a face with tangential
  half-lengths h1, h2 the L2 term carries h1 h2 and the difference quotient
  along t1 (t2) carries h2 (h1); the whole face norm carries R.
* Dirichlet faces: ||sqrt(R) w||_{3/2}^2 = R (||w||_0^2 + sum_t ||w_t||_{1/2}^2)
  (eq. 2.18) with w = u - g and the derivatives along the face's two
  tangential modified coordinates.
"""
from __future__ import annotations

import numpy as np

from .edge import EdgeDiscretisation, face_form
from .functional import eval_tensor, eval_tensor_T, tables
from .gll import gll, lagrange_eval


class VertexDiscretisation(EdgeDiscretisation):
    """Oracle discretisation of a vertex-neighbourhood workloads.EdgeProblem (kind "vertex")."""

    CORNER_FACE = 4

    def _coefs(self, e):
        """c = e^{chi/2} sqrt(sin phi), cot(phi), 1/sin^2(phi) at the Q points, broadcast [chi, theta, phi]."""
        phis, _, chis = self.qpoints(e)
        sp = np.sin(phis)
        c = np.exp(0.5 * chis)[:, None, None] * np.sqrt(sp)[None, None, :]
        return c, (1.0 / np.tan(phis))[None, None, :], (1.0 / (sp * sp))[None, None, :]

    def L_apply(self, u, e):
        B0, B1, B2 = tables(self.W[e])["B"]
        s = self.scale(e)
        c, cot, isin2 = self._coefs(e)
        return -c * (s[2] ** 2 * eval_tensor(u, B0, B0, B2) + s[2] * eval_tensor(u, B0, B0, B1) +
                     s[0] ** 2 * eval_tensor(u, B2, B0, B0) + cot * s[0] * eval_tensor(u, B1, B0, B0) +
                     isin2 * s[1] ** 2 * eval_tensor(u, B0, B2, B0))

    def L_apply_T(self, r, e):
        B0, B1, B2 = tables(self.W[e])["B"]
        s = self.scale(e)
        c, cot, isin2 = self._coefs(e)
        cr = -c * r
        return (eval_tensor_T(s[2] ** 2 * cr, B0, B0, B2) + eval_tensor_T(s[2] * cr, B0, B0, B1) +
                eval_tensor_T(s[0] ** 2 * cr, B2, B0, B0) + eval_tensor_T(cot * s[0] * cr, B1, B0, B0) +
                eval_tensor_T(isin2 * s[1] ** 2 * cr, B0, B2, B0))

    def f_at(self, e, rhs):
        """F^v = e^{5 chi / 2} sqrt(sin phi) f at the volume points."""
        phis, ths, chis = self.qpoints(e)
        c, _, _ = self._coefs(e)
        return c * np.exp(2.0 * chis)[:, None, None] * self.problem.f[rhs](phis, ths, np.exp(chis))

    # --- faces -----------------------------------------------------------
    def G(self, e, fi):
        """R = sup over the face of e^chi."""
        axis, side, _, _ = self.face_axes(fi)
        if axis == 2:
            return float(np.exp(self.mesh.elem_hi[e, 2] if side else self.mesh.elem_lo[e, 2]))
        return float(np.exp(self.mesh.elem_hi[e, 2]))

    def norm_weights(self, e, fi):
        _, _, t1, t2 = self.face_axes(fi)
        hh = self.h(e) / 2.0
        R = self.G(e, fi)
        return (R * hh[t1] * hh[t2], R * hh[t2], R * hh[t1])

    def jump_forms(self, e, fi, Qf):
        _, _, t1, t2 = self.face_axes(fi)
        hh = self.h(e) / 2.0
        Mk = face_form(Qf, *self.norm_weights(e, fi))
        return [face_form(Qf, self.G(e, fi) * hh[t1] * hh[t2], 0.0, 0.0), Mk, Mk, Mk]

    def dirichlet_forms(self, e, fi, Qf):
        _, _, t1, t2 = self.face_axes(fi)
        hh = self.h(e) / 2.0
        Mk = face_form(Qf, *self.norm_weights(e, fi))
        return [face_form(Qf, self.G(e, fi) * hh[t1] * hh[t2], 0.0, 0.0), Mk, Mk]

    def corner_fields(self, p, c, e, Qf):
        """The corner constant on the face chi = ln rho_1: p, no derivatives."""
        z = np.zeros((Qf, Qf))
        return [np.full((Qf, Qf), float(p[0])), z, z, z]

    def corner_fields_T(self, gs, c, e, Qf):
        return np.array([gs[0].sum()])

    def dirichlet_data(self, e, fi, Qf, rhs):
        from .gll import diff_matrix
        axis, side, t1, t2 = self.face_axes(fi)
        phis, ths, chis = self.face_points(e, fi, Qf)
        gv = self.problem.g[rhs](phis, ths, np.exp(chis)).reshape(Qf, Qf)
        xf, _ = gll(Qf)
        D = diff_matrix(xf)
        s = self.scale(e)
        return [gv, s[t1] * (gv @ D.T), s[t2] * (D @ gv)]

    # --- Neumann faces (the last sum of eq. 4.3) ---------------------------
    # L^v u = -div(e^{chi/2} sqrt(sin phi) A^v grad u) + lower-order terms with
    # A^v = diag(1, 1/sin^2 phi, 1) for the Laplacian (the principal part of
    # L^v), so the conormal derivative of eq. 2.24 along the outward normal is
    # +-u_phi, +-u_theta / sin^2 phi or +-u_chi; a physical gradient field
    # q = (q_rho, q_phi, q_theta) gives h^v = +-rho q_phi, +-rho q_theta / sin phi
    # (the thesis's e^chi / sin phi factor of its theta = const faces) or
    # +-rho q_rho.
    def _conormal_factor(self, e, fi, Qf):
        axis, side, _, _ = self.face_axes(fi)
        sgn = 1.0 if side else -1.0
        if axis != 1:
            return sgn
        phis = self.face_points(e, fi, Qf)[0]
        return sgn * np.broadcast_to((1.0 / np.sin(phis) ** 2)[None, :], (Qf, Qf))

    def neumann_data(self, e, fi, Qf, rhs):
        axis, side, _, _ = self.face_axes(fi)
        phis, ths, chis = self.face_points(e, fi, Qf)
        rhos = np.exp(chis)
        shape = (len(chis), len(ths), len(phis))
        qr, qp, qt = self.problem.flux[rhs](phis, ths, rhos)
        rho = np.broadcast_to(rhos[:, None, None], shape)
        sp = np.broadcast_to(np.sin(phis)[None, None, :], shape)
        q = {0: rho * np.broadcast_to(qp, shape), 1: rho * np.broadcast_to(qt, shape) / sp,
             2: rho * np.broadcast_to(qr, shape)}[axis]
        return (1.0 if side else -1.0) * q.reshape(Qf, Qf)

    # --- the functional (literal norm sums, eq. 4.3) -----------------------
    def functional(self, U, rhs=0):
        from .edge import l2_literal
        R = 0.0
        for e in range(self.E):
            u = self.block(U, e)
            z = np.sqrt(self.vol_weight(e)) * (self.L_apply(u, e) - self.f_at(e, rhs))
            R += float(np.sum(z * z))
        for e in range(self.E):
            u = self.block(U, e)
            hh = self.h(e) / 2.0
            for fi in range(6):
                if (e, fi) in self.skip_faces:
                    continue
                Qf = self.Qf(e, fi)
                n = int(self.mesh.elem_nbr[e, fi])
                _, _, t1, t2 = self.face_axes(fi)
                Rf = self.G(e, fi)
                c = self.norm_weights(e, fi)
                if n == -1 and self.is_neumann(e, fi):
                    v = self.neumann_sample(u, e, fi, Qf) - self.neumann_data(e, fi, Qf, rhs)
                    R += self._norm_literal(v, Qf, c)
                    continue
                if n == -1:
                    sm = self.dirichlet_samples(u, e, fi, Qf)
                    dd = self.dirichlet_data(e, fi, Qf, rhs)
                    R += Rf * hh[t1] * hh[t2] * l2_literal(sm[0] - dd[0], Qf)
                    R += self._norm_literal(sm[1] - dd[1], Qf, c) + self._norm_literal(sm[2] - dd[2], Qf, c)
                    continue
                if n >= 0 and n < e:
                    continue
                fe = self.face_fields(u, e, fi, Qf)
                if n >= 0:
                    fn = self.face_fields(self.block(U, n), n, fi ^ 1, Qf)
                else:
                    fn = self.corner_fields(self.corner(U, -2 - n), -2 - n, e, Qf)
                R += Rf * hh[t1] * hh[t2] * l2_literal(fe[0] - fn[0], Qf)
                for k in range(1, 4):
                    R += self._norm_literal(fe[k] - fn[k], Qf, c)
        return R

    def corner_apply(self, U, c):
        p = self.corner(U, c)
        y = np.zeros_like(p)
        f = self.CORNER_FACE
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
        """fun(phi, theta, rho) on every finite element's nodes; each corner set
        takes fun at the centre of its first face chi = ln rho_1."""
        U = np.zeros(self.ndof)
        for e in range(self.E):
            xp, _ = gll(self.P[e])
            phs, ths, chs = (self.coord(e, a, xp) for a in range(3))
            U[self.off[e]:self.off[e + 1]] = fun(phs, ths, np.exp(chs)).ravel()
        for c in range(self.C):
            e = next(e for e in range(self.E) if int(self.mesh.elem_nbr[e, self.CORNER_FACE]) == -2 - c)
            lo, hi = self.mesh.elem_lo[e], self.mesh.elem_hi[e]
            U[self.coff[c]] = float(fun(np.array([0.5 * (lo[0] + hi[0])]), np.array([0.5 * (lo[1] + hi[1])]),
                                        np.array([np.exp(lo[2])])).ravel()[0])
        return U

    def h1_error_exact(self, U, nq=24):
        """(||u_h - w||_{H^1}^2, ||w||_{H^1}^2) over the vertex neighbourhood.
        Finite elements: Gauss-Legendre in (phi, theta, chi) with
        dx = e^{3 chi} sin(phi) dx^v, |grad v|^2 = e^{-2 chi} (v_chi^2 + v_phi^2 + v_theta^2 / sin^2 phi).
        Corner rho < rho_1: u_h is the constant there; integrated in
        (phi, theta, s) with rho = rho_1 s^3."""
        w_fun, gw = self.problem.u_exact, self.problem.grad_exact
        xg, wg = np.polynomial.legendre.leggauss(nq)
        err = nrm = 0.0
        for e in range(self.E):
            xp, _ = gll(self.P[e])
            B = [lagrange_eval(xp, xg, d) for d in range(2)]
            lo, hh = self.mesh.elem_lo[e], self.h(e) / 2.0
            phs, ths, chs = (lo[a] + (xg + 1.0) * hh[a] for a in range(3))
            rho = np.exp(chs)
            u = self.block(U, e)
            s = self.scale(e)
            v = eval_tensor(u, B[0], B[0], B[0])
            vp = s[0] * eval_tensor(u, B[1], B[0], B[0])
            vt = s[1] * eval_tensor(u, B[0], B[1], B[0])
            vc = s[2] * eval_tensor(u, B[0], B[0], B[1])
            wv = w_fun(phs, ths, rho)
            wr, wph, wth = gw(phs, ths, rho)   # w_rho, w_phi / rho, w_theta / (rho sin phi)
            Rr = rho[:, None, None]
            sp = np.sin(phs)[None, None, :]
            wc, wp, wt = Rr * wr, Rr * wph, Rr * sp * wth
            wq = wg[:, None, None] * wg[None, :, None] * wg[None, None, :] * float(np.prod(hh))
            e3, e1 = (Rr ** 3) * sp, Rr * sp
            err += float(np.sum(wq * (e3 * (v - wv) ** 2 + e1 * ((vc - wc) ** 2 + (vp - wp) ** 2 +
                                                                  (vt - wt) ** 2 / (sp * sp)))))
            nrm += float(np.sum(wq * (e3 * wv ** 2 + e1 * (wc ** 2 + wp ** 2 + wt ** 2 / (sp * sp)))))
        f = self.CORNER_FACE
        for c in range(self.C):
            for e in range(self.E):
                if int(self.mesh.elem_nbr[e, f]) != -2 - c:
                    continue
                rho1 = float(np.exp(self.mesh.elem_lo[e, 2]))
                lo, hh = self.mesh.elem_lo[e], self.h(e) / 2.0
                phs, ths = (lo[a] + (xg + 1.0) * hh[a] for a in (0, 1))
                sg = (xg + 1.0) / 2.0
                rho = rho1 * sg ** 3
                jr = 1.5 * rho1 * sg ** 2
                wv = w_fun(phs, ths, rho)
                wr, wph, wth = gw(phs, ths, rho)
                sp = np.sin(phs)[None, None, :]
                wq = ((wg * jr * rho * rho)[:, None, None] * (wg * hh[1])[None, :, None] *
                      (wg * hh[0])[None, None, :]) * sp
                pc = float(self.corner(U, c)[0])
                g2 = wr ** 2 + wph ** 2 + wth ** 2
                err += float(np.sum(wq * ((pc - wv) ** 2 + g2)))
                nrm += float(np.sum(wq * (wv ** 2 + g2)))
        return err, nrm


def h1_diff(disc, U, V):
    """(||u_h - v_h||_{H^1}^2, ||v_h||_{H^1}^2) of two discrete solutions on a
    vertex neighbourhood, in physical coordinates (Section 6.1).

    Finite elements in (phi, theta, chi), rho = e^chi: dx = e^{3 chi} sin(phi)
    dphi dtheta dchi and |grad v|^2 = e^{-2 chi} (v_chi^2 + v_phi^2 +
    v_theta^2 / sin^2(phi)), by the element's (2W+1)-point GLL rule (reading:
    the element rule of the regular region).  Corner set: the constant p on
    rho < rho_1 over the element's (phi, theta) box, integrated exactly:
    p^2 rho_1^3 / 3 (cos phi_lo - cos phi_hi) (theta_hi - theta_lo); its
    gradient is zero."""
    out = []
    for X in (U - V, V):
        tot = 0.0
        for e in range(disc.E):
            xp, _ = gll(disc.P[e])
            xg, wg = gll(2 * disc.W[e] + 1)
            B = [lagrange_eval(xp, xg, d) for d in range(2)]
            lo, hh = disc.mesh.elem_lo[e], disc.h(e) / 2.0
            phs = lo[0] + (xg + 1.0) * hh[0]
            chs = lo[2] + (xg + 1.0) * hh[2]
            s = disc.scale(e)
            u = disc.block(X, e)
            v = eval_tensor(u, B[0], B[0], B[0])
            vp = s[0] * eval_tensor(u, B[1], B[0], B[0])
            vt = s[1] * eval_tensor(u, B[0], B[1], B[0])
            vc = s[2] * eval_tensor(u, B[0], B[0], B[1])
            sp = np.sin(phs)[None, None, :]
            ec = np.exp(chs)[:, None, None]
            wq = wg[:, None, None] * wg[None, :, None] * wg[None, None, :] * float(np.prod(hh))
            tot += float(np.sum(wq * (ec ** 3 * sp * v * v + ec * sp * (vc * vc + vp * vp) + ec * vt * vt / sp)))
        f = disc.CORNER_FACE
        for c in range(disc.C):
            pc = float(disc.corner(X, c)[0])
            for e in range(disc.E):
                if int(disc.mesh.elem_nbr[e, f]) != -2 - c:
                    continue
                lo, hi = disc.mesh.elem_lo[e], disc.mesh.elem_hi[e]
                rho1 = float(np.exp(lo[2]))
                tot += pc * pc * rho1 ** 3 / 3.0 * (np.cos(lo[0]) - np.cos(hi[0])) * (hi[1] - lo[1])
        out.append(tot)
    return tuple(out)

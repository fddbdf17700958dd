"""Edge-neighbourhood least-squares functional in modified coordinates (oracle, FP64).

Test infrastructure only (see the package docstring).

Section 2.3 / Section 4.2: around an edge on the x3 axis the modified
coordinates are x^e = (tau, theta, x3) with tau = ln r, and the geometric mesh
makes every element a box in x^e.  Eq. (4.7) gives, for -Lap u = f,

  R_e(u) = sum_{finite l} int |L^e u_l - F^e|^2 dx^e
         + sum_{interior faces, finite measure} ( ||sqrt(H) [u]||_0^2 + |||[u_tau]|||^2
                                                 + |||[u_theta]|||^2 + |||G [u_x3]|||^2 )
         + sum_{Dirichlet faces, finite measure} ( ||u - g||_0^2 + |||(u - g)_t|||^2 ... )

with L^e u = r^2 L u written in x^e (eq. 2.35): for the Laplacian
L^e u = -(u_tautau + u_thetatheta + e^{2 tau} u_x3x3) and F^e = e^{2 tau} f
(eq. 4.7).  G = sup_face e^tau and, by eq. (2.34), the face norm |||v||| of a
face x3 = const is G (L2 + tau-difference quotient + theta-difference
quotient), of a face tau = const: L2 + theta-DQ + G x3-DQ, of a face
theta = const: L2 + tau-DQ + G x3-DQ; H = G on x3 = const faces, else 1.
The corner elements tau < ln r_1 carry one polynomial in x3 per x3-slab,
shared by all theta sectors; their volume and their infinite faces have
infinite measure and are left out, so they enter only through the faces
r = r_1 with layer 1.

Readings taken here (the thesis is silent or loose on them):

* Degrees: every finite element has the same degree W in tau, theta and x3
  (the thesis's W_q = [mu_1 i] capped at W, with mu_1 >= W), the corner
  polynomial degree W in x3.
* Norms are integrals in the modified coordinates as written in eq. (2.34):
  on a face with tangential half-lengths h1, h2 the L2 term carries h1 h2,
  the difference quotient along t1 carries h2 and along t2 carries h1 (the
  double integral of a difference quotient is invariant under the affine
  map to the reference face).  Quadrature and difference quotients are
  those of the regular region on the (2W+1)-point GLL face grid.
* Dirichlet faces: ||u - g||_0^2 plus |||.|||^2 of the derivatives of u - g
  along the face's two tangential modified coordinates, the x3 derivative
  multiplied by G (eq. 4.7 writes it for the faces theta = const, whose
  tangential coordinates are tau and x3); the tangential derivative of g is
  that of its interpolant on the face grid.
* Volume quadrature: the (2W+1)-point GLL rule per modified coordinate.

Layout: the finite elements' (W+1)^3 nodal blocks (x fastest, i.e. tau
fastest, then theta, then x3) in element order, then each corner set's W+1
nodal values in x3.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np

from .functional import eval_tensor, eval_tensor_T, half_norm_1d, tables, _face_eval_mats
from .gll import diff_matrix, gll, lagrange_eval


@lru_cache(maxsize=None)
def face_form(Qf: int, c0: float, c1: float, c2: float):
    """c0 L2 + c1 DQ(t1) + c2 DQ(t2) on a Qf x Qf face grid flattened [t2][t1]."""
    _, w = gll(Qf)
    Wd = np.diag(w)
    K = half_norm_1d(Qf)
    return c0 * np.kron(Wd, Wd) + c1 * np.kron(Wd, K) + c2 * np.kron(K, Wd)


def l2_literal(v, Qf):
    _, w = gll(Qf)
    return float(np.sum(w[:, None] * w[None, :] * v * v))


def dq_literal(v, Qf, along):
    """The difference-quotient part of the discrete H^{1/2} form (Section 5.3)
    along face direction ``along`` (1: t1, the second index of v[t2, t1];
    2: t2), weighted by the quadrature of the other direction, term by term."""
    x, w = gll(Qf)
    D = diff_matrix(x)
    a = v if along == 1 else v.T  # a[other, along]
    tot = 0.0
    n = Qf
    for o in range(n):
        for i in range(n):
            for ip in range(n):
                if ip != i:
                    tot += w[o] * w[i] * w[ip] * ((a[o, i] - a[o, ip]) / (x[i] - x[ip])) ** 2
            tot += w[o] * w[i] ** 2 * float(np.dot(D[i, :], a[o, :])) ** 2
    return tot


class EdgeDiscretisation:
    """Oracle discretisation of a workloads.EdgeProblem."""

    def __init__(self, problem):
        self.problem = problem
        m = problem.mesh
        self.mesh = m
        self.E = m.n_elem
        self.C = m.n_corner
        self.W = [int(w) for w in m.elem_W]
        self.P = [w + 1 for w in self.W]
        self.Wc = [int(w) for w in m.corner_W]
        off = [0]
        for e in range(self.E):
            off.append(off[-1] + self.P[e] ** 3)
        coff = []
        for c in range(self.C):
            coff.append(off[-1])
            off.append(off[-1] + self.Wc[c] + 1)
        self.off = np.array(off[:self.E + 1], dtype=np.int64)
        self.coff = np.array(coff, dtype=np.int64)
        self.ndof = int(off[-1])
        # (element, face) pairs whose terms a composite discretisation owns
        # (an interface with another region); skipped here
        self.skip_faces = set()

    # --- geometry ---------------------------------------------------------
    def h(self, e):
        return self.mesh.elem_hi[e] - self.mesh.elem_lo[e]

    def scale(self, e):
        return 2.0 / self.h(e)

    def jac(self, e):
        return float(np.prod(self.h(e) / 2.0))

    def coord(self, e, axis, lam):
        return self.mesh.elem_lo[e, axis] + (np.asarray(lam) + 1.0) * self.h(e)[axis] / 2.0

    def qpoints(self, e):
        t = tables(self.W[e])
        return tuple(self.coord(e, a, t["xq"]) for a in range(3))

    def block(self, U, e):
        P = self.P[e]
        return U[self.off[e]:self.off[e + 1]].reshape(P, P, P)

    def corner(self, U, c):
        return U[self.coff[c]:self.coff[c] + self.Wc[c] + 1]

    def vol_weight(self, e):
        wq = tables(self.W[e])["wq"]
        return wq[:, None, None] * wq[None, :, None] * wq[None, None, :] * self.jac(e)

    # --- volume term (eq. 2.35, 4.7) ----------------------------------------
    def L_apply(self, u, e):
        """L^e u = -(u_tautau + u_thetatheta + e^{2 tau} u_x3x3) at the (2W+1)^3 points [x3, theta, tau]."""
        B0, B1, B2 = tables(self.W[e])["B"]
        s = self.scale(e)
        taus = self.qpoints(e)[0]
        e2 = np.exp(2.0 * taus)[None, None, :]
        return -(s[0] ** 2 * eval_tensor(u, B2, B0, B0) + s[1] ** 2 * eval_tensor(u, B0, B2, B0) +
                 e2 * s[2] ** 2 * eval_tensor(u, B0, B0, B2))

    def L_apply_T(self, r, e):
        B0, B1, B2 = tables(self.W[e])["B"]
        s = self.scale(e)
        taus = self.qpoints(e)[0]
        e2 = np.exp(2.0 * taus)[None, None, :]
        return -(eval_tensor_T(s[0] ** 2 * r, B2, B0, B0) + eval_tensor_T(s[1] ** 2 * r, B0, B2, B0) +
                 eval_tensor_T(e2 * s[2] ** 2 * r, B0, B0, B2))

    def f_at(self, e, rhs):
        """F^e = e^{2 tau} f at the volume points."""
        taus, ths, zs = self.qpoints(e)
        fv = self.problem.f[rhs](np.exp(taus), ths, zs)
        return np.exp(2.0 * taus)[None, None, :] * fv

    # --- faces -----------------------------------------------------------
    @staticmethod
    def face_axes(fi):
        axis, side = fi // 2, fi % 2
        t1, t2 = [a for a in range(3) if a != axis]
        return axis, side, t1, t2

    def G(self, e, fi):
        """sup over the face of e^tau."""
        axis, side, _, _ = self.face_axes(fi)
        if axis == 0:
            return float(np.exp(self.mesh.elem_hi[e, 0] if side else self.mesh.elem_lo[e, 0]))
        return float(np.exp(self.mesh.elem_hi[e, 0]))

    def norm_weights(self, e, fi):
        """(c0, c1, c2) of |||.|||^2 on face fi in reference-face terms (eq. 2.34)."""
        axis, _, t1, t2 = self.face_axes(fi)
        hh = self.h(e) / 2.0
        G = self.G(e, fi)
        c = [hh[t1] * hh[t2], hh[t2], hh[t1]]
        if t1 == 2:
            c[1] *= G
        if t2 == 2:
            c[2] *= G
        if axis == 2:
            c = [G * v for v in c]
        return tuple(c)

    def jump_forms(self, e, fi, Qf):
        """Face matrices of the four jump terms: [u], [u_tau], [u_theta], G [u_x3]."""
        axis, _, t1, t2 = self.face_axes(fi)
        hh = self.h(e) / 2.0
        G = self.G(e, fi)
        Hf = G if axis == 2 else 1.0
        c = self.norm_weights(e, fi)
        Mk = face_form(Qf, *c)
        return [face_form(Qf, Hf * hh[t1] * hh[t2], 0.0, 0.0), Mk, Mk, G * G * Mk]

    def dirichlet_forms(self, e, fi, Qf):
        """Face matrices of ||u-g||_0^2 and of the two tangential derivative terms."""
        axis, _, t1, t2 = self.face_axes(fi)
        hh = self.h(e) / 2.0
        G = self.G(e, fi)
        Mk = face_form(Qf, *self.norm_weights(e, fi))
        return [face_form(Qf, hh[t1] * hh[t2], 0.0, 0.0),
                (G * G if t1 == 2 else 1.0) * Mk, (G * G if t2 == 2 else 1.0) * Mk]

    ORD = {0: (0, 0, 0), 1: (1, 0, 0), 2: (0, 1, 0), 3: (0, 0, 1)}

    def face_eval(self, u, e, fi, Qf, orders):
        Mx, My, Mz = _face_eval_mats(self.P[e], fi, Qf, tuple(orders))
        return eval_tensor(u, Mx, My, Mz).reshape(Qf, Qf)

    def face_eval_T(self, g, e, fi, Qf, orders):
        axis = fi // 2
        Mx, My, Mz = _face_eval_mats(self.P[e], fi, Qf, tuple(orders))
        shape = [Qf, Qf, Qf]
        shape[2 - axis] = 1
        return eval_tensor_T(g.reshape(shape), Mx, My, Mz)

    def face_fields(self, u, e, fi, Qf):
        """u and its modified-coordinate derivatives u_tau, u_theta, u_x3 on face fi."""
        s = self.scale(e)
        out = [self.face_eval(u, e, fi, Qf, self.ORD[0])]
        for k in range(3):
            out.append(s[k] * self.face_eval(u, e, fi, Qf, self.ORD[k + 1]))
        return out

    def face_fields_T(self, gs, e, fi, Qf):
        s = self.scale(e)
        out = self.face_eval_T(gs[0], e, fi, Qf, self.ORD[0])
        for k in range(3):
            out = out + s[k] * self.face_eval_T(gs[k + 1], e, fi, Qf, self.ORD[k + 1])
        return out

    def _corner_mats(self, c, Qf):
        xp, _ = gll(self.Wc[c] + 1)
        xf, _ = gll(Qf)
        return lagrange_eval(xp, xf, 0), lagrange_eval(xp, xf, 1)

    def corner_fields(self, p, c, e, Qf):
        """The corner polynomial's fields on the face r = r_1 of layer-1 element e
        (face 0, grid [x3 (t2), theta (t1)]): p, 0, 0, p_x3."""
        B0z, B1z = self._corner_mats(c, Qf)
        s3 = self.scale(e)[2]
        one = np.ones(Qf)
        return [np.outer(B0z @ p, one), np.zeros((Qf, Qf)), np.zeros((Qf, Qf)), s3 * np.outer(B1z @ p, one)]

    def corner_fields_T(self, gs, c, e, Qf):
        B0z, B1z = self._corner_mats(c, Qf)
        s3 = self.scale(e)[2]
        return B0z.T @ gs[0].sum(axis=1) + s3 * (B1z.T @ gs[3].sum(axis=1))

    def face_points(self, e, fi, Qf):
        axis, side, _, _ = self.face_axes(fi)
        xf, _ = gll(Qf)
        pts = []
        for a in range(3):
            lam = np.array([-1.0 if side == 0 else 1.0]) if a == axis else xf
            pts.append(self.coord(e, a, lam))
        return pts

    def dirichlet_samples(self, u, e, fi, Qf):
        """(u, u_t1, u_t2) on a boundary face, modified-coordinate derivatives."""
        axis, side, t1, t2 = self.face_axes(fi)
        s = self.scale(e)
        o1 = [0, 0, 0]
        o1[t1] = 1
        o2 = [0, 0, 0]
        o2[t2] = 1
        return [self.face_eval(u, e, fi, Qf, (0, 0, 0)), s[t1] * self.face_eval(u, e, fi, Qf, tuple(o1)),
                s[t2] * self.face_eval(u, e, fi, Qf, tuple(o2))]

    def dirichlet_samples_T(self, gs, e, fi, Qf):
        axis, side, t1, t2 = self.face_axes(fi)
        s = self.scale(e)
        o1 = [0, 0, 0]
        o1[t1] = 1
        o2 = [0, 0, 0]
        o2[t2] = 1
        return (self.face_eval_T(gs[0], e, fi, Qf, (0, 0, 0)) +
                s[t1] * self.face_eval_T(gs[1], e, fi, Qf, tuple(o1)) +
                s[t2] * self.face_eval_T(gs[2], e, fi, Qf, tuple(o2)))

    def dirichlet_data(self, e, fi, Qf, rhs):
        """(g, g_t1, g_t2) on the face grid [t2, t1] (derivatives of the interpolant)."""
        axis, side, t1, t2 = self.face_axes(fi)
        taus, ths, zs = self.face_points(e, fi, Qf)
        gv = self.problem.g[rhs](np.exp(taus), ths, zs).reshape(Qf, Qf)
        xf, _ = gll(Qf)
        D = diff_matrix(xf)
        s = self.scale(e)
        return [gv, s[t1] * (gv @ D.T), s[t2] * (D @ gv)]

    # --- Neumann faces (the last sum of eq. 2.38 / eq. 4.7) ----------------
    # L^e u = -div(A^e grad u) with A^e = diag(1, 1, e^{2 tau}) for the
    # Laplacian, so the conormal derivative along the outward normal is
    # +-u_tau, +-u_theta or +-e^{2 tau} u_x3; a physical flux q (q_r,
    # q_theta = u_theta / r, q_x3) gives h^e = +-r q_r, +-r q_theta, +-r^2 q_x3.
    def is_neumann(self, e, fi):
        bc = getattr(self.mesh, "elem_bc", None)
        return bc is not None and int(self.mesh.elem_nbr[e, fi]) == -1 and int(bc[e, fi]) == 1

    def _conormal_factor(self, e, fi, Qf):
        """+-1 or +-e^{2 tau} on the face grid [t2, t1] (outward normal)."""
        axis, side, _, _ = self.face_axes(fi)
        sgn = 1.0 if side else -1.0
        if axis != 2:
            return sgn
        taus = self.face_points(e, fi, Qf)[0]
        return sgn * np.broadcast_to(np.exp(2.0 * taus)[None, :], (Qf, Qf))

    def neumann_sample(self, u, e, fi, Qf):
        axis = fi // 2
        o = [0, 0, 0]
        o[axis] = 1
        return self._conormal_factor(e, fi, Qf) * self.scale(e)[axis] * self.face_eval(u, e, fi, Qf, tuple(o))

    def neumann_sample_T(self, g, e, fi, Qf):
        axis = fi // 2
        o = [0, 0, 0]
        o[axis] = 1
        return self.face_eval_T(self._conormal_factor(e, fi, Qf) * self.scale(e)[axis] * g, e, fi, Qf, tuple(o))

    def neumann_data(self, e, fi, Qf, rhs):
        axis, side, _, _ = self.face_axes(fi)
        taus, ths, zs = self.face_points(e, fi, Qf)
        rs = np.exp(taus)
        q = self.problem.flux[rhs](rs, ths, zs)[axis]
        q = np.broadcast_to(q, (len(zs), len(ths), len(rs))).reshape(Qf, Qf)
        r = np.broadcast_to(np.exp(taus)[None, None, :], (len(zs), len(ths), len(rs))).reshape(Qf, Qf)
        return (1.0 if side else -1.0) * (r * r if axis == 2 else r) * q

    def Qf(self, e, fi=None):
        """(2 W_f + 1)-point face grid, W_f the larger degree of the two sides
        of face fi (the element's own degree without fi)."""
        W = self.W[e]
        if fi is not None:
            n = int(self.mesh.elem_nbr[e, fi])
            if n >= 0:
                W = max(W, self.W[n])
            elif n <= -2:
                W = max(W, self.Wc[-2 - n])
        return 2 * W + 1

    # --- the functional (literal norm sums) -------------------------------
    def _norm_literal(self, v, Qf, c):
        return c[0] * l2_literal(v, Qf) + c[1] * dq_literal(v, Qf, 1) + c[2] * dq_literal(v, Qf, 2)

    def functional(self, U, rhs=0):
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
                axis, _, t1, t2 = self.face_axes(fi)
                G = self.G(e, fi)
                c = self.norm_weights(e, fi)
                if n == -1 and self.is_neumann(e, fi):
                    v = self.neumann_sample(u, e, fi, Qf) - self.neumann_data(e, fi, Qf, rhs)
                    R += self._norm_literal(v, Qf, c)
                    continue
                if n == -1:
                    sm = self.dirichlet_samples(u, e, fi, Qf)
                    dd = self.dirichlet_data(e, fi, Qf, rhs)
                    R += hh[t1] * hh[t2] * l2_literal(sm[0] - dd[0], Qf)
                    R += (G * G if t1 == 2 else 1.0) * self._norm_literal(sm[1] - dd[1], Qf, c)
                    R += (G * G if t2 == 2 else 1.0) * self._norm_literal(sm[2] - dd[2], Qf, c)
                    continue
                if n >= 0 and n < e:
                    continue
                fe = self.face_fields(u, e, fi, Qf)
                if n >= 0:
                    fn = self.face_fields(self.block(U, n), n, fi ^ 1, Qf)
                else:
                    cc = -2 - n
                    fn = self.corner_fields(self.corner(U, cc), cc, e, Qf)
                Hf = G if axis == 2 else 1.0
                R += Hf * hh[t1] * hh[t2] * l2_literal(fe[0] - fn[0], Qf)
                R += self._norm_literal(fe[1] - fn[1], Qf, c)
                R += self._norm_literal(fe[2] - fn[2], Qf, c)
                R += G * G * self._norm_literal(fe[3] - fn[3], Qf, c)
        return R

    # --- normal operator and right-hand side -------------------------------
    def element_apply(self, U, e):
        u = self.block(U, e)
        y = self.L_apply_T(self.vol_weight(e) * self.L_apply(u, e), e)
        for fi in range(6):
            if (e, fi) in self.skip_faces:
                continue
            Qf = self.Qf(e, fi)
            n = int(self.mesh.elem_nbr[e, fi])
            if n == -1 and self.is_neumann(e, fi):
                Mk = face_form(Qf, *self.norm_weights(e, fi))
                v = self.neumann_sample(u, e, fi, Qf)
                y = y + self.neumann_sample_T((Mk @ v.ravel()).reshape(Qf, Qf), e, fi, Qf)
                continue
            if n == -1:
                M = self.dirichlet_forms(e, fi, Qf)
                sm = self.dirichlet_samples(u, e, fi, Qf)
                gs = [(M[k] @ sm[k].ravel()).reshape(Qf, Qf) for k in range(3)]
                y = y + self.dirichlet_samples_T(gs, e, fi, Qf)
                continue
            fe = self.face_fields(u, e, fi, Qf)
            if n >= 0:
                fn = self.face_fields(self.block(U, n), n, fi ^ 1, Qf)
                M = self.jump_forms(e, fi, Qf)
            else:
                cc = -2 - n
                fn = self.corner_fields(self.corner(U, cc), cc, e, Qf)
                M = self.jump_forms(e, fi, Qf)
            gs = [(M[k] @ (fe[k] - fn[k]).ravel()).reshape(Qf, Qf) for k in range(4)]
            y = y + self.face_fields_T(gs, e, fi, Qf)
        return y.ravel()

    def corner_apply(self, U, c):
        """(A U) on corner set c: the transposed corner fields of every jump on its faces."""
        p = self.corner(U, c)
        y = np.zeros_like(p)
        for e in range(self.E):
            if int(self.mesh.elem_nbr[e, 0]) != -2 - c:
                continue
            Qf = self.Qf(e, 0)
            fe = self.face_fields(self.block(U, e), e, 0, Qf)
            fn = self.corner_fields(p, c, e, Qf)
            M = self.jump_forms(e, 0, Qf)
            gs = [(M[k] @ (fn[k] - fe[k]).ravel()).reshape(Qf, Qf) for k in range(4)]
            y = y + self.corner_fields_T(gs, c, e, Qf)
        return y

    def apply_A(self, U):
        y = np.zeros(self.ndof)
        for e in range(self.E):
            y[self.off[e]:self.off[e + 1]] = self.element_apply(U, e)
        for c in range(self.C):
            y[self.coff[c]:self.coff[c] + self.Wc[c] + 1] = self.corner_apply(U, c)
        return y

    def rhs_b(self, rhs=0):
        b = np.zeros(self.ndof)
        for e in range(self.E):
            y = self.L_apply_T(self.vol_weight(e) * self.f_at(e, rhs), e)
            for fi in range(6):
                if int(self.mesh.elem_nbr[e, fi]) != -1 or (e, fi) in self.skip_faces:
                    continue
                Qf = self.Qf(e, fi)
                if self.is_neumann(e, fi):
                    Mk = face_form(Qf, *self.norm_weights(e, fi))
                    hd = self.neumann_data(e, fi, Qf, rhs)
                    y = y + self.neumann_sample_T((Mk @ hd.ravel()).reshape(Qf, Qf), e, fi, Qf)
                    continue
                M = self.dirichlet_forms(e, fi, Qf)
                dd = self.dirichlet_data(e, fi, Qf, rhs)
                gs = [(M[k] @ dd[k].ravel()).reshape(Qf, Qf) for k in range(3)]
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
        """Nodal values of fun(r, theta, x3) on every finite element; the corner
        sets take fun on the face r = r_1 at theta of their first sector."""
        U = np.zeros(self.ndof)
        for e in range(self.E):
            xp, _ = gll(self.P[e])
            taus, ths, zs = (self.coord(e, a, xp) for a in range(3))
            U[self.off[e]:self.off[e + 1]] = fun(np.exp(taus), ths, zs).ravel()
        for c in range(self.C):
            e = next(e for e in range(self.E) if int(self.mesh.elem_nbr[e, 0]) == -2 - c)
            xp, _ = gll(self.Wc[c] + 1)
            zs = self.mesh.corner_lo[c] + (xp + 1.0) * (self.mesh.corner_hi[c] - self.mesh.corner_lo[c]) / 2.0
            r1 = np.exp(self.mesh.elem_lo[e, 0])
            U[self.coff[c]:self.coff[c] + self.Wc[c] + 1] = fun(np.array([r1]), self.mesh.elem_lo[e, 1:2], zs).ravel()
        return U

    # --- H^1 error in physical coordinates (Section 6.1) -------------------
    def h1_error_exact(self, U, nq=24):
        """(||u_h - w||_{H^1}^2, ||w||_{H^1}^2) over the whole edge neighbourhood.

        Finite elements: Gauss-Legendre in (tau, theta, x3) with
        dx = e^{2 tau} dtau dtheta dx3 and |grad v|^2 = e^{-2 tau}(v_tau^2 + v_theta^2) + v_x3^2.
        Corner r < r_1: u_h = p(x3) there; integrated in (rho, theta, x3) with
        r = r_1 rho^3, which makes r^{2 alpha - 1} dr smooth for the singular w."""
        w_fun, gw = self.problem.u_exact, self.problem.grad_exact
        xg, wg = np.polynomial.legendre.leggauss(nq)
        err = nrm = 0.0
        for e in range(self.E):
            P = self.P[e]
            xp, _ = gll(P)
            B = [lagrange_eval(xp, xg, d) for d in range(2)]
            lo, hh = self.mesh.elem_lo[e], self.h(e) / 2.0
            taus, ths, zs = (lo[a] + (xg + 1.0) * hh[a] for a in range(3))
            r = np.exp(taus)
            u = self.block(U, e)
            s = self.scale(e)
            v = eval_tensor(u, B[0], B[0], B[0])
            vt = s[0] * eval_tensor(u, B[1], B[0], B[0])
            vh = s[1] * eval_tensor(u, B[0], B[1], B[0])
            vz = s[2] * eval_tensor(u, B[0], B[0], B[1])
            wv = w_fun(r, ths, zs)
            wr, wth, wz = gw(r, ths, zs)   # w_r, w_theta / r, w_x3
            R = r[None, None, :]
            wt, wh = R * wr, R * wth       # w_tau = r w_r, w_theta = r (w_theta / r)
            wq = wg[:, None, None] * wg[None, :, None] * wg[None, None, :] * float(np.prod(hh))
            e2 = R * R
            err += float(np.sum(wq * (e2 * (v - wv) ** 2 + (vt - wt) ** 2 + (vh - wh) ** 2 + e2 * (vz - wz) ** 2)))
            nrm += float(np.sum(wq * (e2 * wv ** 2 + wt ** 2 + wh ** 2 + e2 * wz ** 2)))
        for c in range(self.C):
            for e in range(self.E):
                if int(self.mesh.elem_nbr[e, 0]) != -2 - c:
                    continue
                r1 = float(np.exp(self.mesh.elem_lo[e, 0]))
                lo, hh = self.mesh.elem_lo[e], self.h(e) / 2.0
                ths, zs = (lo[a] + (xg + 1.0) * hh[a] for a in (1, 2))
                rho = (xg + 1.0) / 2.0
                r = r1 * rho ** 3
                jr = 3.0 * r1 * rho ** 2 * 0.5  # dr / d(xg)
                xp, _ = gll(self.Wc[c] + 1)
                p = self.corner(U, c)
                pz = lagrange_eval(xp, xg, 0) @ p
                pdz = (2.0 / (self.mesh.corner_hi[c] - self.mesh.corner_lo[c])) * (lagrange_eval(xp, xg, 1) @ p)
                wv = w_fun(r, ths, zs)
                wr, wth, wz = gw(r, ths, zs)
                wq = (wg[:, None, None] * hh[2]) * (wg[None, :, None] * hh[1]) * (wg[None, None, :] * jr * r)[None, None, :]
                wq = wq.reshape(nq, nq, nq)
                err += float(np.sum(wq * ((pz[:, None, None] - wv) ** 2 + wr ** 2 + wth ** 2 +
                                          (pdz[:, None, None] - wz) ** 2)))
                nrm += float(np.sum(wq * (wv ** 2 + wr ** 2 + wth ** 2 + wz ** 2)))
        return err, nrm


def apply_separable_preconditioner(disc, R):
    """The separable preconditioner of an edge discretisation: on every finite
    element the C* form (eq. 5.30) with eta = sup e^tau over the element, on
    every corner set its exact block A_cc (the corner's rows and columns of A)."""
    from .precond import apply_Cstar_inv_block
    Z = np.zeros_like(R)
    for e in range(disc.E):
        P = disc.P[e]
        eta = float(np.exp(disc.mesh.elem_hi[e, 0]))
        blk = R[disc.off[e]:disc.off[e + 1]].reshape(P, P, P)
        Z[disc.off[e]:disc.off[e + 1]] = apply_Cstar_inv_block(blk, disc.W[e], eta).ravel()
    for c in range(disc.C):
        n = disc.Wc[c] + 1
        sl = slice(disc.coff[c], disc.coff[c] + n)
        Acc = np.zeros((n, n))
        for j in range(n):
            U = np.zeros(disc.ndof)
            U[disc.coff[c] + j] = 1.0
            Acc[:, j] = disc.corner_apply(U, c)
        Z[sl] = np.linalg.solve(Acc, R[sl])
    return Z


def h1_diff(disc, U, V, nq=None):
    """(||u_h - v_h||_{H^1}^2, ||v_h||_{H^1}^2) of two discrete solutions in
    physical coordinates.  Finite elements: e^{2 tau} v^2 + v_tau^2 + v_theta^2
    + e^{2 tau} v_x3^2 in modified coordinates with the (2W+1)-point GLL rule
    (reading: the element rule of the regular region), or an nq-point Gauss
    rule if nq is given; corner sets: p(x3) on r < r_1, integrated exactly in r
    and theta, with the (2W+1)-point GLL rule in x3 (exact for p^2)."""
    out = []
    for X in (U - V, V):
        tot = 0.0
        for e in range(disc.E):
            P = disc.P[e]
            xp, _ = gll(P)
            if nq is None:
                xg, wg = gll(2 * disc.W[e] + 1)
            else:
                xg, wg = np.polynomial.legendre.leggauss(nq)
            B = [lagrange_eval(xp, xg, d) for d in range(2)]
            lo, hh = disc.mesh.elem_lo[e], disc.h(e) / 2.0
            taus = lo[0] + (xg + 1.0) * hh[0]
            s = disc.scale(e)
            u = disc.block(X, e)
            v = eval_tensor(u, B[0], B[0], B[0])
            vt = s[0] * eval_tensor(u, B[1], B[0], B[0])
            vh = s[1] * eval_tensor(u, B[0], B[1], B[0])
            vz = s[2] * eval_tensor(u, B[0], B[0], B[1])
            e2 = np.exp(2.0 * taus)[None, None, :]
            wq = wg[:, None, None] * wg[None, :, None] * wg[None, None, :] * float(np.prod(hh))
            tot += float(np.sum(wq * (e2 * v * v + vt * vt + vh * vh + e2 * vz * vz)))
        for c in range(disc.C):
            n = disc.Wc[c] + 1
            xp, _ = gll(n)
            xg, wg = gll(2 * disc.Wc[c] + 1)
            p = disc.corner(X, c)
            for e in range(disc.E):
                if int(disc.mesh.elem_nbr[e, 0]) != -2 - c:
                    continue
                r1 = float(np.exp(disc.mesh.elem_lo[e, 0]))
                hth = disc.mesh.elem_hi[e, 1] - disc.mesh.elem_lo[e, 1]
                hz = disc.mesh.elem_hi[e, 2] - disc.mesh.elem_lo[e, 2]
                p0 = lagrange_eval(xp, xg, 0) @ p
                p1 = (2.0 / hz) * (lagrange_eval(xp, xg, 1) @ p)
                tot += 0.5 * r1 * r1 * hth * 0.5 * hz * float(np.sum(wg * (p0 * p0 + p1 * p1)))
        out.append(tot)
    return tuple(out)

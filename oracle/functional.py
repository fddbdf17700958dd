"""The regular-region least-squares functional and its normal equations (oracle).

Test infrastructure only (see the package docstring).

Eq. (4.2) defines, for box elements Omega_l mapped affinely onto the master
cube Q = (-1,1)^3 by x = lo + (lambda + 1) h / 2,

    R(u) = sum_l int_Q |L u_l - f|^2 J dlambda
         + sum_{interior faces} ( ||[u]||_0^2 + sum_k ||[u_{x_k}]||_{1/2}^2 )
         + sum_{Dirichlet faces} ||u_l - g||_{3/2}^2
         + sum_{Neumann faces} ||(du_l/dnu)_A - h||_{1/2}^2 ,

with L u = -div(a grad u) (a = 1 for the Poisson / Laplace problems) and
(du/dnu)_A = a grad u . nu the conormal derivative along the outward unit
normal (eq. 2.1).

Readings taken here (the thesis is silent or loose on them):

* Quadrature.  The volume integral is evaluated with the (2W+1)-point GLL rule
  in each variable (Section 5.3).  The face norms use the (2W_f+1)-point GLL
  rule on the face, W_f = max of the two sides' degrees.
* Face norms are taken in the reference-face coordinates lambda (eq. 2.17b):
  no area Jacobian and no h-scaling; the jumps of derivatives are jumps of the
  physical derivatives u_{x_k} (eq. 4.2), each side using its own map.
* The H^{1/2} norm is the one of eq. (2.17b) with sigma = 1/2, discretised as
  in Section 5.3: off-diagonal difference quotients plus the diagonal
  (w_i)^2 w_j (D l)_i^2 terms.  For polynomials of degree <= 2W_f - 1 per
  variable (every face trace of degree <= W_f) this GLL sum equals the exact
  double integral (pinned in tests).
* The H^{3/2} norm on a Dirichlet face is eq. (2.18) with sigma = 1/2:
  ||w||_0^2 + sum_i ||dw/dlambda_i||_{1/2}^2; the tangential derivative of the
  data g is the derivative of its interpolant on the face GLL grid (the
  differentiation matrix of eq. 5.47 applied to sampled g).
* Each interior face has one jump term (it is not counted from both sides).
* Neumann faces: the conormal derivative a du/dnu = +-a s_a du/dlambda_a
  (a sampled on the face) at the face's GLL points against h = nu . q of the
  problem's conormal field q, in the H^{1/2} norm of the other face terms.

The functional is R(U) = (S U - d)^T M (S U - d), S the sampling map (volume
samples weighted by sqrt(w J) so that M = I there; face samples unweighted with
M the L2 / H^{1/2} face matrices).  The normal equations (Section 5.3) are
A U = b with A = S^T M S and b = S^T M d; A is applied matrix-free.

Layout: the unknowns of element e are its nodal values on the (W+1)^3 GLL
grid, lexicographic with x fastest (Section 5.3), stored as an array
u[k, j, i] (z, y, x); elements are concatenated in element order; several
right-hand sides are stacked as U[r, :].
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np

from .gll import diff_matrix, gll, lagrange_eval


# ---------------------------------------------------------------------------
# 1-D tables
# ---------------------------------------------------------------------------
@lru_cache(maxsize=None)
def tables(W: int):
    """P = W+1 nodal grid, Q = 2W+1 quadrature grid and Q x P evaluation matrices."""
    P, Q = W + 1, 2 * W + 1
    xp, wp = gll(P)
    xq, wq = gll(Q)
    B0 = lagrange_eval(xp, xq, 0)
    B1 = lagrange_eval(xp, xq, 1)
    B2 = lagrange_eval(xp, xq, 2)
    return dict(P=P, Q=Q, xp=xp, wp=wp, xq=xq, wq=wq, B=(B0, B1, B2))


@lru_cache(maxsize=None)
def half_norm_1d(Qf: int):
    """1-D matrix K with l^T K l = the x-part of the discrete H^{1/2} form.

    l^T K l = sum_{i != i'} w_i w_i' ((l_i - l_i') / (x_i - x_i'))^2
              + sum_i w_i^2 (sum_k d_ik l_k)^2                    (Section 5.3)
    """
    x, w = gll(Qf)
    D = diff_matrix(x)
    K = D.T @ np.diag(w * w) @ D
    for i in range(Qf):
        for ip in range(Qf):
            if i == ip:
                continue
            c = w[i] * w[ip] / (x[i] - x[ip]) ** 2
            K[i, i] += c
            K[ip, ip] += c
            K[i, ip] -= c
            K[ip, i] -= c
    return K


@lru_cache(maxsize=None)
def face_mats(Qf: int):
    """(W2, H): L2 and H^{1/2} matrices on a Qf x Qf face grid flattened [t2][t1].

    ||l||_{1/2,S}^2 = sum w_i w_j l_ij^2 + sum_j w_j (x-part on row j)
                      + sum_i w_i (y-part on column i)                 (eq. 5.49)
    """
    x, w = gll(Qf)
    Wd = np.diag(w)
    K = half_norm_1d(Qf)
    W2 = np.kron(Wd, Wd)
    H = np.kron(Wd, Wd) + np.kron(Wd, K) + np.kron(K, Wd)
    return W2, H


def l2_face_literal(v, Qf):
    """||v||_{0,S}^2 by the GLL sum on the face (v indexed [j (t2), i (t1)])."""
    _, w = gll(Qf)
    return float(np.sum(w[:, None] * w[None, :] * v * v))


def h12_face_literal(v, Qf):
    """||v||_{1/2,S}^2 written out term by term as in Section 5.3 (v[j, i])."""
    x, w = gll(Qf)
    D = diff_matrix(x)
    tot = l2_face_literal(v, Qf)
    n = Qf
    for j in range(n):
        for i in range(n):
            for ip in range(n):
                if ip != i:
                    tot += w[j] * w[i] * w[ip] * ((v[j, i] - v[j, ip]) / (x[i] - x[ip])) ** 2
    for i in range(n):
        for j in range(n):
            for jp in range(n):
                if jp != j:
                    tot += w[i] * w[j] * w[jp] * ((v[j, i] - v[jp, i]) / (x[j] - x[jp])) ** 2
    for i in range(n):
        for j in range(n):
            tot += w[i] ** 2 * w[j] * float(np.dot(D[i, :], v[j, :])) ** 2
    for j in range(n):
        for i in range(n):
            tot += w[j] ** 2 * w[i] * float(np.dot(D[j, :], v[:, i])) ** 2
    return tot


# ---------------------------------------------------------------------------
# tensor-product evaluation and its adjoint
# ---------------------------------------------------------------------------
def eval_tensor(u, Mx, My, Mz):
    """out[c, b, a] = sum_{k,j,i} Mz[c,k] My[b,j] Mx[a,i] u[k,j,i]."""
    return np.einsum("ck,bj,ai,kji->cba", Mz, My, Mx, u, optimize=True)


def eval_tensor_T(r, Mx, My, Mz):
    """Adjoint of eval_tensor: out[k, j, i] = sum_{c,b,a} Mz[c,k] My[b,j] Mx[a,i] r[c,b,a]."""
    return np.einsum("ck,bj,ai,cba->kji", Mz, My, Mx, r, optimize=True)


@lru_cache(maxsize=None)
def _face_eval_mats(P: int, fi: int, Qf: int, orders: tuple):
    """Lagrange matrices (x, y, z) evaluating order-``orders`` derivatives on face fi."""
    axis, side = fi // 2, fi % 2
    xp, _ = gll(P)
    xf, _ = gll(Qf)
    mats = []
    for a in range(3):
        pts = np.array([-1.0 if side == 0 else 1.0]) if a == axis else xf
        mats.append(lagrange_eval(xp, pts, orders[a]))
    return tuple(mats)


# ---------------------------------------------------------------------------
# discretisation of one mesh (batch of problems) with its data
# ---------------------------------------------------------------------------
class Discretisation:
    """Oracle discretisation of a workloads.Problem (box elements, Dirichlet faces)."""

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
        self._coef_cache = {}

    def part(self, e):
        """The problem whose data element e uses (batches of independent problems)."""
        parts = getattr(self.problem, "parts", None)
        return parts[int(self.mesh.elem_problem[e])] if parts is not None else self.problem

    # --- geometry ---------------------------------------------------------
    def h(self, e):
        return self.mesh.elem_hi[e] - self.mesh.elem_lo[e]

    def scale(self, e):
        """s_k = d lambda_k / d x_k = 2 / h_k."""
        return 2.0 / self.h(e)

    def jac(self, e):
        """J = det(dx / dlambda) = prod h_k / 2."""
        return float(np.prod(self.h(e) / 2.0))

    def phys(self, e, axis, lam):
        lo = self.mesh.elem_lo[e, axis]
        return lo + (np.asarray(lam) + 1.0) * self.h(e)[axis] / 2.0

    def qpoints(self, e):
        t = tables(self.W[e])
        return tuple(self.phys(e, a, t["xq"]) for a in range(3))

    def block(self, U, e):
        P = self.P[e]
        return U[self.off[e]:self.off[e + 1]].reshape(P, P, P)

    # --- coefficient a and its gradient at the volume points ---------------
    def coef(self, e):
        if e in self._coef_cache:
            return self._coef_cache[e]
        Q = tables(self.W[e])["Q"]
        xs, ys, zs = self.qpoints(e)
        pb = self.part(e)
        if pb.a is None:
            a = np.ones((Q, Q, Q))
            g = (np.zeros((Q, Q, Q)),) * 3
        else:
            a = np.broadcast_to(pb.a(xs, ys, zs), (Q, Q, Q))
            g = tuple(np.broadcast_to(c, (Q, Q, Q)) for c in pb.grad_a(xs, ys, zs))
        self._coef_cache[e] = (a, g)
        return a, g

    def vol_weight(self, e):
        """w_a w_b w_c J at the (2W+1)^3 GLL points, indexed [c, b, a]."""
        wq = tables(self.W[e])["wq"]
        return wq[:, None, None] * wq[None, :, None] * wq[None, None, :] * self.jac(e)

    # --- the general operator of eq. (2.2), written out ---------------------
    # L u = sum_ij A_ij u_{x_i x_j} + sum_i b_i u_{x_i} + c u (A symmetric); the
    # divergence form -sum d_i(a_ij u_j) of eq. (2.2) is this with A = -a and
    # b_j -= sum_i d_i a_ij.  A problem gives it as op(xs, ys, zs) -> (A, b, c)
    # on tensor grids (3x3 nested A, 3 b, scalar c; arrays or constants).
    def _op_terms(self, e):
        """(coefficient [Q,Q,Q], x, y, z matrices) of every term of L."""
        B0, B1, B2 = tables(self.W[e])["B"]
        Q = tables(self.W[e])["Q"]
        s = self.scale(e)
        A, b, c = self.part(e).op(*self.qpoints(e))

        def full(v):
            return np.broadcast_to(np.asarray(v, dtype=np.float64), (Q, Q, Q))
        Bm = {0: B0, 1: B1, 2: B2}
        terms = []
        for i in range(3):
            for j in range(i, 3):
                order = [0, 0, 0]
                order[i] += 1
                order[j] += 1
                coef = (1.0 if i == j else 2.0) * full(A[i][j]) * s[i] * s[j]
                terms.append((coef, Bm[order[0]], Bm[order[1]], Bm[order[2]]))
        for i in range(3):
            order = [0, 0, 0]
            order[i] = 1
            terms.append((full(b[i]) * s[i], Bm[order[0]], Bm[order[1]], Bm[order[2]]))
        terms.append((full(c), B0, B0, B0))
        return terms

    # --- volume term: L u at the quadrature points (eq. 4.2) ---------------
    def L_apply(self, u, e):
        """L u = -a (u_xx + u_yy + u_zz) - grad a . grad u at the (2W+1)^3 points
        (or the problem's general operator)."""
        if getattr(self.part(e), "op", None) is not None:
            return sum(cf * eval_tensor(u, Mx, My, Mz) for cf, Mx, My, Mz in self._op_terms(e))
        B0, B1, B2 = tables(self.W[e])["B"]
        s = self.scale(e)
        a, (ax, ay, az) = self.coef(e)
        uxx = s[0] ** 2 * eval_tensor(u, B2, B0, B0)
        uyy = s[1] ** 2 * eval_tensor(u, B0, B2, B0)
        uzz = s[2] ** 2 * eval_tensor(u, B0, B0, B2)
        ux = s[0] * eval_tensor(u, B1, B0, B0)
        uy = s[1] * eval_tensor(u, B0, B1, B0)
        uz = s[2] * eval_tensor(u, B0, B0, B1)
        return -a * (uxx + uyy + uzz) - (ax * ux + ay * uy + az * uz)

    def L_apply_T(self, r, e):
        """Adjoint of L_apply (same coefficients, transposed evaluation matrices)."""
        if getattr(self.part(e), "op", None) is not None:
            return sum(eval_tensor_T(cf * r, Mx, My, Mz) for cf, Mx, My, Mz in self._op_terms(e))
        B0, B1, B2 = tables(self.W[e])["B"]
        s = self.scale(e)
        a, (ax, ay, az) = self.coef(e)
        out = eval_tensor_T(-a * s[0] ** 2 * r, B2, B0, B0)
        out += eval_tensor_T(-a * s[1] ** 2 * r, B0, B2, B0)
        out += eval_tensor_T(-a * s[2] ** 2 * r, B0, B0, B2)
        out += eval_tensor_T(-ax * s[0] * r, B1, B0, B0)
        out += eval_tensor_T(-ay * s[1] * r, B0, B1, B0)
        out += eval_tensor_T(-az * s[2] * r, B0, B0, B1)
        return out

    def f_at(self, e, rhs):
        xs, ys, zs = self.qpoints(e)
        return self.part(e).f[rhs](xs, ys, zs)

    # --- faces -----------------------------------------------------------
    @staticmethod
    def face_axes(fi):
        axis, side = fi // 2, fi % 2
        t1, t2 = [a for a in range(3) if a != axis]
        return axis, side, t1, t2

    def face_Qf(self, e, fi):
        n = int(self.mesh.elem_nbr[e, fi])
        Wf = self.W[e] if n < 0 else max(self.W[e], self.W[n])
        return 2 * Wf + 1

    def _face_mats(self, e, fi, Qf, orders):
        """Per-axis evaluation matrices for face fi of element e at its Qf^2 points."""
        return _face_eval_mats(self.P[e], fi, Qf, tuple(orders))

    def face_eval(self, u, e, fi, Qf, orders):
        """d^orders u / d lambda^orders on face fi at its Qf^2 GLL points, shape [t2, t1]."""
        Mx, My, Mz = self._face_mats(e, fi, Qf, orders)
        return eval_tensor(u, Mx, My, Mz).reshape(Qf, Qf)

    def face_eval_T(self, g, e, fi, Qf, orders):
        axis = fi // 2
        Mx, My, Mz = self._face_mats(e, fi, Qf, orders)
        shape = [Qf, Qf, Qf]
        shape[2 - axis] = 1
        return eval_tensor_T(g.reshape(shape), Mx, My, Mz)

    def face_points(self, e, fi, Qf):
        axis, side, _, _ = self.face_axes(fi)
        xf, _ = gll(Qf)
        pts = []
        for a in range(3):
            lam = np.array([-1.0 if side == 0 else 1.0]) if a == axis else xf
            pts.append(self.phys(e, a, lam))
        return pts

    def check_match(self, e, fi):
        n = int(self.mesh.elem_nbr[e, fi])
        axis = fi // 2
        for a in range(3):
            if a == axis:
                continue
            if not (np.isclose(self.mesh.elem_lo[e, a], self.mesh.elem_lo[n, a]) and
                    np.isclose(self.mesh.elem_hi[e, a], self.mesh.elem_hi[n, a])):
                raise ValueError("non-matching face between elements %d and %d" % (e, n))
        if int(self.mesh.elem_nbr[n, fi ^ 1]) != e:
            raise ValueError("face adjacency is not symmetric")

    ORD = {0: (0, 0, 0), 1: (1, 0, 0), 2: (0, 1, 0), 3: (0, 0, 1)}

    def face_fields(self, u, e, fi, Qf):
        """u and the physical gradient u_{x_k} on face fi (field 0 = u, 1..3 = x,y,z)."""
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

    def dirichlet_samples(self, u, e, fi, Qf):
        """(u, du/dlambda_t1, du/dlambda_t2) on a boundary face (the H^{3/2} norm, eq. 2.18)."""
        axis, side, t1, t2 = self.face_axes(fi)
        o1 = [0, 0, 0]
        o1[t1] = 1
        o2 = [0, 0, 0]
        o2[t2] = 1
        return [self.face_eval(u, e, fi, Qf, (0, 0, 0)),
                self.face_eval(u, e, fi, Qf, tuple(o1)),
                self.face_eval(u, e, fi, Qf, tuple(o2))]

    def dirichlet_samples_T(self, gs, e, fi, Qf):
        axis, side, t1, t2 = self.face_axes(fi)
        o1 = [0, 0, 0]
        o1[t1] = 1
        o2 = [0, 0, 0]
        o2[t2] = 1
        return (self.face_eval_T(gs[0], e, fi, Qf, (0, 0, 0)) +
                self.face_eval_T(gs[1], e, fi, Qf, tuple(o1)) +
                self.face_eval_T(gs[2], e, fi, Qf, tuple(o2)))

    def dirichlet_data(self, e, fi, Qf, rhs):
        """(g, dg/dlambda_t1, dg/dlambda_t2) on the face grid [t2, t1]."""
        xs, ys, zs = self.face_points(e, fi, Qf)
        gv = self.part(e).g[rhs](xs, ys, zs).reshape(Qf, Qf)
        xf, _ = gll(Qf)
        D = diff_matrix(xf)
        return [gv, gv @ D.T, D @ gv]

    # --- Neumann faces (eq. 2.1, the last sum of eq. 4.2) -------------------
    def is_neumann(self, e, fi):
        """A Neumann (bc 1) or Robin (bc 2) face."""
        bc = getattr(self.mesh, "elem_bc", None)
        return bc is not None and int(self.mesh.elem_nbr[e, fi]) == -1 and int(bc[e, fi]) in (1, 2)

    def _robin(self, e, fi):
        bc = getattr(self.mesh, "elem_bc", None)
        return float(getattr(self.part(e), "robin_gamma", 1.0)) if int(bc[e, fi]) == 2 else 0.0

    def _face_a(self, e, fi, Qf):
        pb = self.part(e)
        if pb.a is None:   # the Laplacian, or a general operator: the plain normal derivative
            return 1.0
        xs, ys, zs = self.face_points(e, fi, Qf)
        return np.broadcast_to(pb.a(xs, ys, zs), (len(zs), len(ys), len(xs))).reshape(Qf, Qf)

    def neumann_sample(self, u, e, fi, Qf):
        """a du/dnu (+ gamma u on a Robin face) on the face grid [t2, t1], nu
        the outward normal."""
        axis, side, _, _ = self.face_axes(fi)
        o = [0, 0, 0]
        o[axis] = 1
        sgn = 1.0 if side else -1.0
        v = sgn * self.scale(e)[axis] * self._face_a(e, fi, Qf) * self.face_eval(u, e, fi, Qf, tuple(o))
        gam = self._robin(e, fi)
        return v + gam * self.face_eval(u, e, fi, Qf, (0, 0, 0)) if gam else v

    def neumann_sample_T(self, g, e, fi, Qf):
        axis, side, _, _ = self.face_axes(fi)
        o = [0, 0, 0]
        o[axis] = 1
        sgn = 1.0 if side else -1.0
        y = self.face_eval_T(sgn * self.scale(e)[axis] * self._face_a(e, fi, Qf) * g, e, fi, Qf, tuple(o))
        gam = self._robin(e, fi)
        return y + self.face_eval_T(gam * g, e, fi, Qf, (0, 0, 0)) if gam else y

    def neumann_data(self, e, fi, Qf, rhs):
        """h = nu . q (+ gamma g on a Robin face) at the face grid [t2, t1] from
        the problem's conormal field q and boundary values g."""
        axis, side, _, _ = self.face_axes(fi)
        xs, ys, zs = self.face_points(e, fi, Qf)
        shape = (len(zs), len(ys), len(xs))
        q = self.part(e).flux[rhs](xs, ys, zs)[axis]
        h = (1.0 if side else -1.0) * np.broadcast_to(q, shape).reshape(Qf, Qf)
        gam = self._robin(e, fi)
        if gam:
            h = h + gam * np.broadcast_to(self.part(e).g[rhs](xs, ys, zs), shape).reshape(Qf, Qf)
        return h

    # --- the functional R (literal norm formulas) ------------------------
    def functional(self, U, rhs=0):
        """R(U) of eq. (4.2) with every norm summed term by term."""
        R = 0.0
        for e in range(self.E):
            u = self.block(U, e)
            z = np.sqrt(self.vol_weight(e)) * (self.L_apply(u, e) - self.f_at(e, rhs))
            R += float(np.sum(z * z))
        for e in range(self.E):
            u = self.block(U, e)
            for fi in range(6):
                n = int(self.mesh.elem_nbr[e, fi])
                Qf = self.face_Qf(e, fi)
                if n >= 0:
                    if n < e:
                        continue
                    self.check_match(e, fi)
                    fe = self.face_fields(u, e, fi, Qf)
                    fn = self.face_fields(self.block(U, n), n, fi ^ 1, Qf)
                    R += l2_face_literal(fe[0] - fn[0], Qf)
                    for k in range(1, 4):
                        R += h12_face_literal(fe[k] - fn[k], Qf)
                elif self.is_neumann(e, fi):
                    R += h12_face_literal(self.neumann_sample(u, e, fi, Qf) - self.neumann_data(e, fi, Qf, rhs), Qf)
                else:
                    sm = self.dirichlet_samples(u, e, fi, Qf)
                    dd = self.dirichlet_data(e, fi, Qf, rhs)
                    R += l2_face_literal(sm[0] - dd[0], Qf)
                    R += h12_face_literal(sm[1] - dd[1], Qf)
                    R += h12_face_literal(sm[2] - dd[2], Qf)
        return R

    # --- normal operator and right-hand side ------------------------------
    def element_apply(self, U, e):
        """(A U) restricted to element e: volume term plus every face of e."""
        u = self.block(U, e)
        y = self.L_apply_T(self.vol_weight(e) * self.L_apply(u, e), e)
        for fi in range(6):
            n = int(self.mesh.elem_nbr[e, fi])
            Qf = self.face_Qf(e, fi)
            W2, H = face_mats(Qf)
            if n >= 0:
                self.check_match(e, fi)
                fe = self.face_fields(u, e, fi, Qf)
                fn = self.face_fields(self.block(U, n), n, fi ^ 1, Qf)
                gs = [(W2 @ (fe[0] - fn[0]).ravel()).reshape(Qf, Qf)]
                for k in range(1, 4):
                    gs.append((H @ (fe[k] - fn[k]).ravel()).reshape(Qf, Qf))
                y = y + self.face_fields_T(gs, e, fi, Qf)
            elif self.is_neumann(e, fi):
                v = self.neumann_sample(u, e, fi, Qf)
                y = y + self.neumann_sample_T((H @ v.ravel()).reshape(Qf, Qf), e, fi, Qf)
            else:
                sm = self.dirichlet_samples(u, e, fi, Qf)
                gs = [(W2 @ sm[0].ravel()).reshape(Qf, Qf),
                      (H @ sm[1].ravel()).reshape(Qf, Qf),
                      (H @ sm[2].ravel()).reshape(Qf, Qf)]
                y = y + self.dirichlet_samples_T(gs, e, fi, Qf)
        return y.ravel()

    def apply_A(self, U, elems=None):
        """y = A U (one right-hand side); with ``elems`` only those blocks are filled."""
        y = np.zeros(self.ndof)
        for e in (range(self.E) if elems is None else elems):
            y[self.off[e]:self.off[e + 1]] = self.element_apply(U, e)
        return y

    def rhs_b(self, rhs=0):
        """b = S^T M d for right-hand side ``rhs``."""
        b = np.zeros(self.ndof)
        for e in range(self.E):
            y = self.L_apply_T(self.vol_weight(e) * self.f_at(e, rhs), e)
            for fi in range(6):
                if int(self.mesh.elem_nbr[e, fi]) >= 0:
                    continue
                Qf = self.face_Qf(e, fi)
                W2, H = face_mats(Qf)
                if self.is_neumann(e, fi):
                    hd = self.neumann_data(e, fi, Qf, rhs)
                    y = y + self.neumann_sample_T((H @ hd.ravel()).reshape(Qf, Qf), e, fi, Qf)
                    continue
                dd = self.dirichlet_data(e, fi, Qf, rhs)
                gs = [(W2 @ dd[0].ravel()).reshape(Qf, Qf),
                      (H @ dd[1].ravel()).reshape(Qf, Qf),
                      (H @ dd[2].ravel()).reshape(Qf, Qf)]
                y = y + self.dirichlet_samples_T(gs, e, fi, Qf)
            b[self.off[e]:self.off[e + 1]] = y.ravel()
        return b

    def dense_A(self):
        """Assemble A column by column from unit vectors (tiny meshes only)."""
        A = np.zeros((self.ndof, self.ndof))
        for j in range(self.ndof):
            v = np.zeros(self.ndof)
            v[j] = 1.0
            A[:, j] = self.apply_A(v)
        return A

    # --- interpolation of a function into the nodal space ----------------
    def nodal_interpolant(self, fun):
        """Nodal values of fun on every element's (W+1)^3 GLL grid."""
        U = np.zeros(self.ndof)
        for e in range(self.E):
            xp, _ = gll(self.P[e])
            xs, ys, zs = (self.phys(e, a, xp) for a in range(3))
            U[self.off[e]:self.off[e + 1]] = fun(xs, ys, zs).ravel()
        return U

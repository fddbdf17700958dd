"""Pins of the vertex-edge-neighbourhood oracle (eq. 2.27-2.29 in modified
coordinates (ln tan phi, theta, ln x3)).

* The operator: L^{v-e} applied to the nodal interpolant of a smooth function
  equals -e^{zeta/2} r^2 Lap w with the Laplacian taken in Cartesian
  coordinates; and int |L^{v-e} w|^2 dx^{v-e} equals int r^2 |Lap w|^2 dx
  integrated in physical coordinates (the defining identity of eq. 2.28).
* Face-norm weights E, F, G: the functional of a piecewise constant equals the
  hand-summed L2 jump weights; the anisotropic norms of eq. 2.27 against
  hand-computed integrals of linear traces.
* A solution inside the discrete space with both corner kinds makes R vanish
  and is returned by the normal equations.
* Variation identity (literal functional vs matrix-free A, Dirichlet data and
  both corner kinds); A symmetric positive definite.
* The H^1 norm of w = r^(2/3) sin(2 theta / 3) over the neighbourhood against
  its closed form; the H^1 error of least-squares solutions decays with W.
"""
import numpy as np
import pytest

import workloads as wl
from oracle.edge import face_form
from oracle.gll import gll
from oracle.vertex_edge import VertexEdgeDiscretisation


def _zero(ps, ts, zs):
    return 0.0 * wl._ve_grid(ps, ts, zs)[0]


def _box_problem(lo, hi, W, w_fun, f_fun):
    """One finite element with every face Dirichlet (no corner sets)."""
    mesh = wl.EdgeMeshDesc(np.array([lo], dtype=float), np.array([hi], dtype=float), np.array([W], dtype=np.int32),
                           -np.ones((1, 6), dtype=np.int32), np.zeros(1, dtype=np.int32),
                           np.zeros(0, dtype=np.int32), np.zeros(0), np.zeros(0), np.zeros(0, dtype=np.int32),
                           kind="vertex-edge")
    return wl.EdgeProblem(mesh, [f_fun], [w_fun])


def _w(ps, ts, zs):
    # w = x1 x2 x3^2 + x3^3 + r^3 with r = e^{psi + zeta}, x3 = e^zeta
    p, t, z = wl._ve_grid(ps, ts, zs)
    r, x3 = np.exp(p + z), np.exp(z)
    return 0.5 * r * r * np.sin(2 * t) * x3 * x3 + x3 ** 3 + r ** 3


def _lap_w(p, t, z):
    # Cartesian Laplacian: 2 x1 x2 + 6 x3 + 9 r
    r, x3 = np.exp(p + z), np.exp(z)
    return r * r * np.sin(2 * t) + 6.0 * x3 + 9.0 * r


LO, HI = (-0.3, 0.2, -1.0), (0.2, 0.9, -0.5)


def test_ve_operator_is_the_cartesian_laplacian():
    # interpolation error of the smooth w: 1e-3, 4e-7, 5e-11 at W = 6, 9, 12
    W = 12
    d = VertexEdgeDiscretisation(_box_problem(LO, HI, W, _w, _zero))
    xp, _ = gll(W + 1)
    u = _w(*(d.coord(0, a, xp) for a in range(3)))
    ps, ts, zs = d.qpoints(0)
    p, t, z = wl._ve_grid(ps, ts, zs)
    want = -np.exp(0.5 * z) * np.exp(2 * (p + z)) * _lap_w(p, t, z)
    got = d.L_apply(u, 0)
    assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()


def test_ve_residual_weight_is_the_physical_integral():
    # int |L^{v-e} w|^2 dx^{v-e} over the box = int r^2 |Lap w|^2 dx over its
    # physical image {e^psi_lo < r / x3 < e^psi_hi, theta, e^zeta_lo < x3 < e^zeta_hi}
    xg, wg = np.polynomial.legendre.leggauss(30)
    h = [(HI[a] - LO[a]) / 2 for a in range(3)]
    ps, ts, zs = (LO[a] + (xg + 1) * h[a] for a in range(3))
    p, t, z = wl._ve_grid(ps, ts, zs)
    Lv = -np.exp(0.5 * z) * np.exp(2 * (p + z)) * _lap_w(p, t, z)
    wq = np.einsum("i,j,k->ijk", wg, wg, wg) * h[0] * h[1] * h[2]
    lhs = float(np.sum(wq * Lv * Lv))
    # physical: (tt = r / x3, theta, x3), dx = r dr dtheta dx3 = tt x3^2 dtt dtheta dx3
    t0, t1 = np.exp(LO[0]), np.exp(HI[0])
    x0, x1 = np.exp(LO[2]), np.exp(HI[2])
    tt = t0 + (xg + 1) * (t1 - t0) / 2
    x3 = x0 + (xg + 1) * (x1 - x0) / 2
    X3, TH, TT = np.meshgrid(x3, ts, tt, indexing="ij")
    r = TT * X3
    lap = r * r * np.sin(2 * TH) + 6.0 * X3 + 9.0 * r
    wq2 = np.einsum("i,j,k->ijk", wg * (x1 - x0) / 2, wg * h[1], wg * (t1 - t0) / 2)
    rhs = float(np.sum(wq2 * r * r * lap * lap * TT * X3 * X3))
    assert lhs == pytest.approx(rhs, rel=1e-10)


def _sin_phi(psi):
    return np.sin(np.arctan(np.exp(psi)))


def test_ve_piecewise_constant_jump_weights():
    # U = 1 on one element's nodes (0 elsewhere, zero data): only [u] (and u on
    # Dirichlet faces) is non-zero; each face adds 4 hh_t1 hh_t2 F G with
    # F = sup e^zeta, G = sup sin(phi) on interior faces zeta = const, else 1
    mesh = wl.vertex_edge_mesh(3, 2, J=2)
    d = VertexEdgeDiscretisation(wl.EdgeProblem(mesh, [_zero], [_zero]))
    for e in (0, 4, 13):
        U = np.zeros(d.ndof)
        U[d.off[e]:d.off[e + 1]] = 1.0
        lo, hi = mesh.elem_lo[e], mesh.elem_hi[e]
        hh = (hi - lo) / 2
        want = 0.0
        for fi in range(6):
            a, side = fi // 2, fi % 2
            t1, t2 = [b for b in range(3) if b != a]
            zmax = lo[2] if (a == 2 and side == 0) else hi[2]
            pmax = lo[0] if (a == 0 and side == 0) else hi[0]
            G = _sin_phi(pmax) if (a == 2 and mesh.elem_nbr[e, fi] != -1) else 1.0
            want += 4 * hh[t1] * hh[t2] * np.exp(zmax) * G
        assert d.functional(U) == pytest.approx(want, rel=1e-12), e


def test_ve_face_norm_weights_closed_forms():
    d = VertexEdgeDiscretisation(wl.vertex_edge_polynomial(N=2, W=3))
    e = 3
    lo, hi = d.mesh.elem_lo[e], d.mesh.elem_hi[e]
    hp, ht, hz = d.h(e) / 2.0
    Qf = d.Qf(e)
    x, _ = gll(Qf)
    one = np.ones(Qf)
    F, E = np.exp(hi[2]), _sin_phi(hi[0])
    # v linear along t1 (unit slope in modified coordinates): L2 + quotient along t1;
    # along t2: L2 + quotient along t2 (grid [t2, t1])
    cases = [  # face, slope direction, tangential half-lengths (along, other), L2 weight, quotient weight
        (1, 1, ht, hz, F * ht * hz, F * hz),            # psi = const, along theta
        (1, 2, hz, ht, F * ht * hz, F * E * ht),        # psi = const, along zeta: E
        (3, 1, hp, hz, F * hp * hz, F * hz),            # theta = const, along psi
        (3, 2, hz, hp, F * hp * hz, F * E * hp),        # theta = const, along zeta: E
        (5, 1, hp, ht, E * F * hp * ht, E * F * ht),    # zeta = const: E F on everything
        (5, 2, ht, hp, E * F * hp * ht, E * F * hp),
    ]
    for fi, along, ha, hb, c0, cq in cases:
        v = np.outer(one, ha * x) if along == 1 else np.outer(ha * x, one)
        want = c0 * 4 * ha * ha / 3 + cq * 8 * ha * ha
        got = float(v.ravel() @ face_form(Qf, *d.norm_weights(e, fi)) @ v.ravel())
        assert got == pytest.approx(want, rel=1e-12), (fi, along)
    assert d.E_sup(e, 0) == pytest.approx(_sin_phi(lo[0]))
    assert d.F_sup(e, 4) == pytest.approx(np.exp(lo[2]))


def test_ve_polynomial_solution_is_reproduced():
    pb = wl.vertex_edge_polynomial(N=2, W=3)
    pb.mesh = wl.vertex_edge_mesh(2, 3, J=1)
    d = VertexEdgeDiscretisation(pb)
    assert d.cface == [0, 0, 4]
    U = d.nodal_interpolant(pb.u_exact)
    assert d.functional(U) <= 1e-22 * d.functional(np.zeros(d.ndof))
    x = np.linalg.solve(d.dense_A(), d.rhs_b())
    assert np.linalg.norm(x - U) <= 1e-8 * np.linalg.norm(U)


def test_ve_variation_identity_and_spd():
    pb = wl.vertex_edge_singular(N=2, W=2)
    pb.mesh = wl.vertex_edge_mesh(2, 2, J=2)
    d = VertexEdgeDiscretisation(pb)
    rng = np.random.default_rng(12)
    U, V = rng.standard_normal(d.ndof), rng.standard_normal(d.ndof)
    A, b = d.dense_A(), d.rhs_b()
    assert np.abs(A - A.T).max() <= 1e-11 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
    for eps in (0.6, -1.7):
        lhs = d.functional(U + eps * V)
        rhs = d.functional(U) + 2 * eps * V @ (A @ U - b) + eps ** 2 * V @ A @ V
        assert lhs == pytest.approx(rhs, rel=1e-10)


def test_ve_h1_norm_closed_form():
    # ||w||_{H^1}^2 over {0 < x3 < 1, phi < pi/4, 0 < theta < 3 pi/2} for
    # w = r^(2/3) sin(2 theta / 3): |grad w|^2 = (4/9) r^(-2/3), r < x3:
    # (3 pi / 2)(4/9)(3/4)(3/7) + (3 pi / 4)(3/10)(3/13)
    d = VertexEdgeDiscretisation(wl.vertex_edge_singular(N=3, W=2))
    err, nrm = d.h1_error_exact(np.zeros(d.ndof), nq=30)
    want = 1.5 * np.pi * (4 / 9) * (3 / 4) * (3 / 7) + 0.75 * np.pi * (3 / 10) * (3 / 13)
    assert nrm == pytest.approx(want, rel=1e-8)
    assert err == pytest.approx(nrm, rel=1e-12)


def _ls_h1(W, N):
    """Relative H^1 errors of the least-squares solution (block-Jacobi PCG to
    1e-10) and of the nodal interpolant; one theta sector, N layers."""
    import scipy.linalg as sla
    from oracle.pcg import pcg
    from oracle.precond import element_block
    pb = wl.vertex_edge_singular(N=N, W=W)
    pb.mesh = wl.vertex_edge_mesh(N, W, J=1)
    d = VertexEdgeDiscretisation(pb)
    fac = [sla.cho_factor(element_block(d, e)) for e in range(d.E)]
    cinv = []
    for c in range(d.C):
        n = d.Wc[c] + 1
        A = np.zeros((n, n))
        for j in range(n):
            U = np.zeros(d.ndof)
            U[d.coff[c] + j] = 1.0
            A[:, j] = d.corner_apply(U, c)
        cinv.append(np.linalg.inv(A))

    def M(r):
        z = np.zeros_like(r)
        for e in range(d.E):
            z[d.off[e]:d.off[e + 1]] = sla.cho_solve(fac[e], r[d.off[e]:d.off[e + 1]])
        for c in range(d.C):
            sl = slice(d.coff[c], d.coff[c] + d.Wc[c] + 1)
            z[sl] = cinv[c] @ r[sl]
        return z
    x, _, rel = pcg(d.apply_A, M, d.rhs_b(), tol=1e-10, maxit=5000)
    assert rel <= 1e-10
    err, nrm = d.h1_error_exact(x)
    ei, _ = d.h1_error_exact(d.nodal_interpolant(pb.u_exact))
    return np.sqrt(err / nrm), np.sqrt(ei / nrm)


@pytest.mark.slow
def test_ve_h1_error_decays_with_w():
    # one sector of opening 3 pi/2: the theta approximation of sin(2 theta / 3)
    # dominates at low W (measured: 12.8 % at W = 2, N = 3; 0.32 % at W = 4, N = 6)
    e2, i2 = _ls_h1(2, 3)
    e4, i4 = _ls_h1(4, 4)
    assert e4 < 0.1 * e2, (e2, e4)
    # the least-squares solution is as good as interpolation up to a modest factor
    assert e2 < 2 * i2 and e4 < 2 * i4, (e2, i2, e4, i4)


def _table_6_20_error(W, N, J):
    """Block-Jacobi PCG solution of Table 6.20's problem (the cone truncated by
    the plane x3 = cos(pi/6) inscribed in the table's unit sphere), relative
    H^1 error against w."""
    import scipy.linalg as sla
    from oracle.pcg import pcg
    from oracle.precond import element_block
    d = VertexEdgeDiscretisation(wl.vertex_edge_table_6_20(N, W, J=J))
    fac = [sla.cho_factor(element_block(d, e)) for e in range(d.E)]
    cinv = []
    for c in range(d.C):
        n = d.Wc[c] + 1
        A = np.zeros((n, n))
        for k in range(n):
            U = np.zeros(d.ndof)
            U[d.coff[c] + k] = 1.0
            A[:, k] = d.corner_apply(U, c)
        cinv.append(np.linalg.inv(A))

    def M(r):
        z = np.zeros_like(r)
        for e in range(d.E):
            z[d.off[e]:d.off[e + 1]] = sla.cho_solve(fac[e], r[d.off[e]:d.off[e + 1]])
        for c in range(d.C):
            sl = slice(d.coff[c], d.coff[c] + d.Wc[c] + 1)
            z[sl] = cinv[c] @ r[sl]
        return z
    x, _, rel = pcg(d.apply_A, M, d.rhs_b(), tol=1e-10, maxit=5000)
    assert rel <= 1e-10
    err, nrm = d.h1_error_exact(x)
    return np.sqrt(err / nrm)


def test_table_6_20_w2():
    # one theta sector, N = 3: measured 13.0 % against the table's 4.73 %
    from golden_tables import rel_error
    ref = rel_error("table6_20_vertex_edge.txt", 2)
    err = _table_6_20_error(2, 3, 1)
    assert ref / 5 < err < ref * 5, err


@pytest.mark.slow
def test_table_6_20_w3():
    # three theta sectors, N = 4: measured 3.00 % against 1.06 % (W = 2: 10.2 %)
    from golden_tables import rel_error
    ref = rel_error("table6_20_vertex_edge.txt", 3)
    err = _table_6_20_error(3, 4, 3)
    assert ref / 5 < err < ref * 5, err

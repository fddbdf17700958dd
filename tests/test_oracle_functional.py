"""Pins for the oracle functional, its normal operator and PCG (eq. 4.2, Section 5.3).

* closed-form values of R for simple functions (volume scaling, face conventions);
* the variation identity R(U + eV) = R(U) + 2e V^T(AU - b) + e^2 V^T A V, with R
  summed term by term and A applied matrix-free;
* adjointness of the sampling map and its transpose;
* symmetry / positive definiteness of A assembled by brute force, Cholesky = PCG;
* polynomial reproduction (exact solution inside the discrete space);
* the transposed interpolation G^T computed by the five Legendre-transform
  steps of Section 5.3 equals the explicit transpose used in the oracle.
"""
import numpy as np
import pytest

import workloads as wl
from oracle.functional import Discretisation, eval_tensor, eval_tensor_T, tables
from oracle.gll import gll, legendre
from oracle.pcg import cholesky_solve, pcg
from oracle.precond import apply_Cinv


def _zero_problem(mesh, a=None, grad_a=None):
    z = wl._zero
    return wl.Problem(mesh, [z], [z], a, grad_a)


def test_closed_form_volume_term():
    # one element [0,2]x[0,1]x[0,1], u = x^2, f = 0: Lu = -2, R_vol = int 4 = 8
    mesh = wl.box_mesh((1, 1, 1), (0, 0, 0), (2, 1, 1), W=3)
    d = Discretisation(_zero_problem(mesh))
    U = d.nodal_interpolant(lambda xs, ys, zs: np.broadcast_to(
        np.asarray(xs)[None, None, :] ** 2, (len(zs), len(ys), len(xs))).copy())
    e = 0
    z = np.sqrt(d.vol_weight(e)) * d.L_apply(d.block(U, e), e)
    assert abs(float(np.sum(z * z)) - 8.0) < 1e-12


def test_closed_form_variable_coefficient():
    # u = x, a = 1 + x: L u = -(a u')' = -1, R_vol = |Omega| = 1 on (0,1)^3
    mesh = wl.box_mesh((1, 1, 1), (0, 0, 0), (1, 1, 1), W=2)

    def a(xs, ys, zs):
        x, y, z = wl._grid(xs, ys, zs)
        return np.broadcast_to(1 + x, (len(zs), len(ys), len(xs))).copy()

    def ga(xs, ys, zs):
        s = (len(zs), len(ys), len(xs))
        return np.ones(s), np.zeros(s), np.zeros(s)

    d = Discretisation(_zero_problem(mesh, a, ga))
    U = d.nodal_interpolant(lambda xs, ys, zs: np.broadcast_to(
        np.asarray(xs)[None, None, :], (len(zs), len(ys), len(xs))).copy())
    Lu = d.L_apply(d.block(U, 0), 0)
    assert np.allclose(Lu, -1.0, atol=1e-12)


def test_closed_form_face_terms():
    # two elements along x; u = 1 on element 0 and 0 on element 1, f = g = 0.
    # volume terms vanish; the interior jump [u] = 1 has ||1||_0^2 = 4 on the
    # reference face; the 5 Dirichlet faces of element 0 carry ||1||_{3/2}^2 = 4.
    mesh = wl.box_mesh((2, 1, 1), (0, 0, 0), (1, 0.5, 0.5), W=2)
    d = Discretisation(_zero_problem(mesh))
    U = np.zeros(d.ndof)
    U[d.off[0]:d.off[1]] = 1.0
    assert abs(d.functional(U) - 24.0) < 1e-12


def test_closed_form_derivative_jump():
    # u = x on element 0, u = 0 on element 1 (both [0,1] x ... along x with h = 1/2):
    # interior face: [u] = 1/2, [u_x] = 1 (physical), ||1||_{1/2}^2 = ||1||_0^2 = 4.
    mesh = wl.box_mesh((2, 1, 1), (0, 0, 0), (1, 1, 1), W=2)
    d = Discretisation(_zero_problem(mesh))
    xp, _ = gll(3)
    U = np.zeros(d.ndof)
    u0 = np.broadcast_to(d.phys(0, 0, xp)[None, None, :], (3, 3, 3))
    U[d.off[0]:d.off[1]] = u0.ravel()
    e, fi, Qf = 0, 1, 5
    fe = d.face_fields(d.block(U, 0), 0, fi, Qf)
    fn = d.face_fields(d.block(U, 1), 1, fi ^ 1, Qf)
    assert np.allclose(fe[0] - fn[0], 0.5)
    assert np.allclose(fe[1] - fn[1], 1.0)
    assert np.allclose(fe[2] - fn[2], 0.0) and np.allclose(fe[3] - fn[3], 0.0)


@pytest.mark.parametrize("maker", [
    lambda: wl.varcoef_manufactured(n=(2, 1, 1), W=3),
    lambda: wl.laplace_sinh(n=(1, 2, 1), W=2),
])
def test_variation_identity(maker):
    pb = maker()
    d = Discretisation(pb)
    rng = np.random.default_rng(7)
    U = rng.standard_normal(d.ndof)
    V = rng.standard_normal(d.ndof)
    b = d.rhs_b()
    AU = d.apply_A(U)
    AV = d.apply_A(V)
    R0 = d.functional(U)
    for eps in (0.3, -1.7):
        lhs = d.functional(U + eps * V)
        rhs = R0 + 2 * eps * V @ (AU - b) + eps * eps * V @ AV
        assert abs(lhs - rhs) < 1e-11 * abs(lhs), (lhs, rhs)


def test_adjoint_of_sampling_map():
    pb = wl.varcoef_manufactured(n=(1, 1, 1), W=4)
    d = Discretisation(pb)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((5, 5, 5))
    r = rng.standard_normal((9, 9, 9))
    lhs = float(np.sum(d.L_apply(u, 0) * r))
    rhs = float(np.sum(u * d.L_apply_T(r, 0)))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    for fi in range(6):
        for orders in [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]:
            g = rng.standard_normal((9, 9))
            lhs = float(np.sum(d.face_eval(u, 0, fi, 9, orders) * g))
            rhs = float(np.sum(u * d.face_eval_T(g, 0, fi, 9, orders)))
            assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_brute_force_spd_and_cholesky_equals_pcg():
    pb = wl.varcoef_manufactured(n=(2, 1, 1), W=2)
    d = Discretisation(pb)
    A = d.dense_A()
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0
    b = d.rhs_b()
    x_direct = cholesky_solve(A, b)
    x_pcg, it, rel = pcg(d.apply_A, lambda r: apply_Cinv(d, r), b, tol=1e-13)
    assert rel <= 1e-13
    assert np.abs(x_pcg - x_direct).max() <= 1e-9 * np.abs(x_direct).max()


def test_polynomial_reproduction():
    pb = wl.polynomial_exact(n=2, W=3)
    d = Discretisation(pb)
    ui = d.nodal_interpolant(pb.u_exact[0])
    assert d.functional(ui) < 1e-22
    b = d.rhs_b()
    assert np.abs(d.apply_A(ui) - b).max() < 1e-10 * np.abs(b).max()
    x, it, rel = pcg(d.apply_A, lambda r: apply_Cinv(d, r), b, tol=1e-12)
    assert np.abs(x - ui).max() < 1e-9


def _G_transpose_by_legendre_steps(O, W):
    """J = G^T O by the five steps of Section 5.3 (discrete Legendre transforms)."""
    P, Q = W + 1, 2 * W + 1
    xq, wq = gll(Q)
    xp, wp = gll(P)

    def gam(n, N):
        m = np.arange(n)
        g = 1.0 / (m + 0.5)
        g[N] = 2.0 / N
        return g[:n]

    g2 = gam(Q, 2 * W)
    g1 = gam(P, W)
    Lq = np.array([legendre(m, xq) for m in range(Q)])  # [m, i]
    Lp = np.array([legendre(m, xp) for m in range(P)])
    # 1. divide by the weights
    O = O / (wq[:, None, None] * wq[None, :, None] * wq[None, None, :])
    # 2. Legendre transform on the 2N grid, times gamma^{2N}
    Dl = np.einsum("ck,bj,ai,kji->cba", Lq, Lq, Lq, O * (wq[:, None, None] * wq[None, :, None] * wq[None, None, :]))
    Dl = Dl / (g2[:, None, None] * g2[None, :, None] * g2[None, None, :])
    Dl = Dl * (g2[:, None, None] * g2[None, :, None] * g2[None, None, :])
    # 3. truncate to degree N and divide by gamma^N
    mu = Dl[:P, :P, :P] / (g1[:, None, None] * g1[None, :, None] * g1[None, None, :])
    # 4. inverse Legendre transform on the N grid, times the weights
    eps = np.einsum("ck,bj,ai,cba->kji", Lp, Lp, Lp, mu)
    return eps * (wp[:, None, None] * wp[None, :, None] * wp[None, None, :])


@pytest.mark.parametrize("W", [2, 4, 7])
def test_G_transpose_legendre_steps(W):
    # Reading: the Legendre transform of step 2 is the discrete one,
    # Delta_m = (1/gamma_m) sum_i w_i L_m(x_i) O_i; multiplying by gamma^{2N}
    # then leaves the plain weighted projection sum_i w_i L_m(x_i) O_i.
    rng = np.random.default_rng(W)
    Q = 2 * W + 1
    O = rng.standard_normal((Q, Q, Q))
    B0 = tables(W)["B"][0]
    J_explicit = eval_tensor_T(O, B0, B0, B0)
    J_steps = _G_transpose_by_legendre_steps(O, W)
    assert np.allclose(J_steps, J_explicit, atol=1e-12 * np.abs(J_explicit).max())
    # and G itself interpolates: V^{2N} = G V^N
    v = rng.standard_normal((W + 1,) * 3)
    assert np.allclose(np.sum(eval_tensor(v, B0, B0, B0) * O), np.sum(v * J_explicit))

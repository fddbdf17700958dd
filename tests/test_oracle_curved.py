"""Pins of the oracle for regular elements with a curved map (eq. 4.2 through
the chain rule of the map): the L-shaped prism's polar-blend sectors around
the re-entrant edge.

* The blend map's first and second derivatives against central differences.
* With affine maps the curved oracle equals the box oracle (operator,
  right-hand side and functional of a mesh with Dirichlet data).
* -Lap of a smooth function's interpolant through a curved map equals the
  Cartesian Laplacian at every quadrature point (W = 20, 2e-8).
* Variation identity and A symmetric positive definite on the six sectors.
* The H^1 error of w = r^(2/3) sin(2 theta'/3) (smooth for r >= 0.25) decays
  with W and stays within 5x of the interpolant's.
"""
import numpy as np
import pytest

import workloads as wl
from oracle.curved import CurvedDiscretisation, CurvedMesh, CurvedProblem
from oracle.functional import Discretisation

PI = np.pi


def test_blend_map_derivatives():
    maps, _, _, _, _, _ = wl.lprism_regular(3)
    rng = np.random.default_rng(3)
    h = 1e-5
    for m in maps:
        lam = [rng.uniform(-1, 1, size=5) for _ in range(3)]
        x, Dx, D2x = m(*lam)
        for a in range(3):
            lp = [v.copy() for v in lam]
            lm = [v.copy() for v in lam]
            lp[a] += h
            lm[a] -= h
            xp, Dp, _ = m(*lp)
            xm, Dm, _ = m(*lm)
            assert np.abs((xp - xm) / (2 * h) - Dx[:, a]).max() <= 1e-8 * (1 + np.abs(Dx).max())
            assert np.abs((Dp - Dm) / (2 * h) - D2x[:, :, a]).max() <= 1e-7 * (1 + np.abs(D2x).max())


def _sine(x, y, z):
    return np.sin(PI * x) * np.sin(PI * y) * np.sin(PI * z)


def test_affine_maps_equal_the_box_oracle():
    desc = wl.box_mesh((2, 1, 1), lo=(0.0, 0.0, 0.0), hi=(1.0, 0.6, 0.8), W=3)

    def g(x, y, z):
        return np.exp(x) * np.cos(y) + z * z

    def f(x, y, z):
        return 3 * PI * PI * _sine(x, y, z)

    def grid(fun):
        return lambda xs, ys, zs: fun(*wl._grid(xs, ys, zs))

    box = Discretisation(wl.Problem(desc, [grid(f)], [grid(g)]))
    maps, W, nbr = wl.curved_mesh_of_boxes(desc)
    cur = CurvedDiscretisation(CurvedProblem(CurvedMesh(maps, W, nbr), f, g))
    U = wl.random_dofs(box.ndof, seed=23)
    ya, yb = cur.apply_A(U), box.apply_A(U)
    assert np.abs(ya - yb).max() <= 1e-12 * np.abs(yb).max()
    ba, bb = cur.rhs_b(), box.rhs_b()
    assert np.abs(ba - bb).max() <= 1e-12 * np.abs(bb).max()
    assert cur.functional(U) == pytest.approx(box.functional(U), rel=1e-12)


def test_curved_operator_is_the_cartesian_laplacian():
    # w is not a polynomial in the reference coordinates of a curved map: the
    # gap is the interpolation error, 8e-5, 3e-7, 5e-9 of max at W = 12, 16, 20
    maps, _, _, _, _, _ = wl.lprism_regular(20)
    W = 20

    def w(x, y, z):
        return np.sin(1.3 * x) * np.exp(y) * z + x * x * y

    def lap(x, y, z):
        return -1.69 * np.sin(1.3 * x) * np.exp(y) * z + np.sin(1.3 * x) * np.exp(y) * z + 2 * y

    for j in (0, 2, 5):
        mesh = CurvedMesh([maps[j]], np.array([W]), -np.ones((1, 6), dtype=np.int32))
        d = CurvedDiscretisation(CurvedProblem(mesh, w, w))
        U = d.nodal_interpolant(w)
        x = d.vol_geom(0)[0]
        got = d.L_apply(d.block(U, 0), 0)
        want = -lap(x[0], x[1], x[2])
        assert np.abs(got - want).max() <= 2e-8 * np.abs(want).max(), j


def _lprism(W):
    maps, Ws, nbr, u, gu, f = wl.lprism_regular(W)
    return CurvedDiscretisation(CurvedProblem(CurvedMesh(maps, Ws, nbr), f, u, u, gu))


def test_curved_variation_identity_and_spd():
    d = _lprism(2)
    rng = np.random.default_rng(29)
    U, V = rng.standard_normal(d.ndof), rng.standard_normal(d.ndof)
    A, b = d.dense_A(), d.rhs_b()
    assert np.abs(A - A.T).max() <= 1e-11 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
    for eps in (0.5, -1.1):
        lhs = d.functional(U + eps * V)
        rhs = d.functional(U) + 2 * eps * V @ (A @ U - b) + eps ** 2 * V @ A @ V
        assert lhs == pytest.approx(rhs, rel=1e-10)


def _curved_errors(Ws):
    from oracle.pcg import pcg
    from oracle.precond import apply_block_inverse, block_factors
    errs, ints = {}, {}
    for W in Ws:
        d = _lprism(W)
        fac = block_factors(d)
        x, _, rel = pcg(d.apply_A, lambda r: apply_block_inverse(d, r, fac), d.rhs_b(), tol=1e-12, maxit=5000)
        assert rel <= 1e-12
        errs[W] = d.h1_error_exact(x)
        ints[W] = d.h1_error_exact(d.nodal_interpolant(d.problem.u_exact))
    return errs, ints


def test_curved_h1_error_decays_w2_w3():
    # measured: 13.0 %, 2.07 % at W = 2, 3 against the interpolant's 3.4 %, 0.65 %
    errs, ints = _curved_errors((2, 3))
    assert errs[3] < 0.5 * errs[2], errs
    for W in (2, 3):
        assert errs[W] < 5 * ints[W], (errs, ints)


@pytest.mark.slow
def test_curved_h1_error_decays():
    # measured: 13.0 %, 2.07 %, 0.31 % at W = 2, 3, 4 against the interpolant's
    # 3.4 %, 0.65 %, 0.14 % (block-Jacobi PCG to 1e-12)
    from oracle.pcg import pcg
    from oracle.precond import apply_block_inverse, block_factors
    errs, ints = {}, {}
    for W in (2, 3, 4):
        d = _lprism(W)
        fac = block_factors(d)
        x, _, rel = pcg(d.apply_A, lambda r: apply_block_inverse(d, r, fac), d.rhs_b(), tol=1e-12, maxit=5000)
        assert rel <= 1e-12
        errs[W] = d.h1_error_exact(x)
        ints[W] = d.h1_error_exact(d.nodal_interpolant(d.problem.u_exact))
    for W in (3, 4):
        assert errs[W] < 0.5 * errs[W - 1], errs
    for W in (2, 3, 4):
        assert errs[W] < 5 * ints[W], (errs, ints)


def test_h1_parts_gll_equals_the_gauss_rule_on_polynomials():
    # affine maps, a discrete u of degree W and a polynomial "exact" w of
    # degree <= W: every H^1 integrand has degree <= 2W, which both the
    # (2W+1)^3 GLL rule and the 20^3 Gauss rule integrate exactly
    desc = wl.box_mesh((2, 1, 1), lo=(0.0, 0.0, 0.0), hi=(1.0, 0.5, 0.7), W=3)
    maps, Ws, nbr = wl.curved_mesh_of_boxes(desc)

    def w(x, y, z):
        return x * x * y - z ** 3 + 0.5 * x * y * z

    def gw(x, y, z):
        return (2 * x * y + 0.5 * y * z, x * x + 0.5 * x * z, -3 * z * z + 0.5 * x * y)

    d = CurvedDiscretisation(CurvedProblem(CurvedMesh(maps, np.asarray(Ws), np.asarray(nbr)), w, w, w, gw))
    U = np.random.default_rng(2).standard_normal(d.ndof)
    a, b = d.h1_parts_gll(U), d.h1_parts(U, nq=20)
    assert a[0] == pytest.approx(b[0], rel=1e-12) and a[1] == pytest.approx(b[1], rel=1e-12)

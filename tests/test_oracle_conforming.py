"""Pins of the oracle's conforming correction (Remark 4.3.0, Appendix C.1).

* The corrected function is conforming: the traces of the two elements of
  every interior face coincide node by node, and it vanishes on every
  Dirichlet face (random nodal data, batches of two problems, ragged meshes,
  degrees 2 and 3).
* It is a projection: a function that is already conforming and vanishes on
  the Dirichlet boundary (the nodal interpolant of sin(pi x) sin(pi y)
  sin(pi z) on matching GLL grids) is returned unchanged; the correction is
  linear in u.
* Half jumps: two elements with traces a and b on their common face take
  (a + b) / 2 there, and the face correction blends linearly,
  (1 + lambda) / 2, along the normal lines of the element.
* The H^1 error of the corrected solution of the 2 x 2 x 2 Poisson problem
  stays within 1.5x of the nonconforming solution's (W = 2, 3: 0.146 -> 0.160,
  0.0208 -> 0.0159) and decays with W (Remark 4.3.0: exponentially small).
"""
import numpy as np
import pytest

import workloads as wl
from oracle.conforming import conforming_correction
from oracle.functional import Discretisation
from oracle.gll import gll
from oracle.h1 import h1_error_exact
from oracle.pcg import pcg
from oracle.precond import apply_Cinv


def _trace(B, fi, P):
    a, side = fi >> 1, fi & 1
    n = P - 1 if side else 0
    return [B[:, :, n], B[:, n, :], B[n, :, :]][a]


def _conformity_error(d, p):
    worst = 0.0
    for e in range(d.E):
        B = d.block(p, e)
        for fi in range(6):
            nb = int(d.mesh.elem_nbr[e, fi])
            tr = _trace(B, fi, d.P[e])
            if nb >= 0:
                worst = max(worst, float(np.abs(tr - _trace(d.block(p, nb), fi ^ 1, d.P[nb])).max()))
            else:
                worst = max(worst, float(np.abs(tr).max()))
    return worst


def _mesh_cases():
    a = wl.varcoef_manufactured(n=(3, 2, 1), W=2)
    b = wl.poisson_sine(n=2, W=3)
    return {"ragged_W2": a, "cube_W3": b, "batch": wl.batch_problems([wl.poisson_sine(n=2, W=2),
                                                                       wl.poisson_sine(n=(2, 1, 1), W=2)])}


@pytest.mark.parametrize("name", ["ragged_W2", "cube_W3", "batch"])
def test_correction_is_conforming_and_vanishes_on_dirichlet_faces(name):
    d = Discretisation(_mesh_cases()[name])
    U = np.random.default_rng(3).standard_normal(d.ndof)
    p = conforming_correction(d, U)
    assert _conformity_error(d, p) <= 1e-14 * np.abs(p).max()
    assert _conformity_error(d, U) > 0.1  # the data were not conforming


def test_correction_is_a_linear_projection():
    pb = wl.poisson_sine(n=2, W=3)
    d = Discretisation(pb)
    U = d.nodal_interpolant(pb.u_exact[0])
    assert np.abs(conforming_correction(d, U) - U).max() <= 1e-14 * np.abs(U).max()
    rng = np.random.default_rng(4)
    X, Y = rng.standard_normal(d.ndof), rng.standard_normal(d.ndof)
    lhs = conforming_correction(d, 2.0 * X - 3.0 * Y)
    rhs = 2.0 * conforming_correction(d, X) - 3.0 * conforming_correction(d, Y)
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(rhs).max()


def test_half_jump_on_a_face_and_its_linear_blend():
    # two elements side by side along x on (0,1)^3 (x < 1/2 and x > 1/2), W = 3,
    # with s = sin(pi y) sin(pi z) (zero on the y and z faces, hence on every
    # edge and vertex): element 0 holds x s, element 1 holds (x + 1) s.  Only
    # the faces x = 1/2 (jump s) and x = 1 (Dirichlet, trace 2 s) need
    # corrections; the common face takes the average s and element 0's
    # correction s / 2 blends linearly to 0 at x = 0.
    pb = wl.poisson_sine(n=(2, 1, 1), W=3)
    d = Discretisation(pb)
    s_ = lambda y, z: np.sin(np.pi * y) * np.sin(np.pi * z)  # noqa: E731
    U = d.nodal_interpolant(lambda x, y, z: x[None, None, :] * s_(y[None, :, None], z[:, None, None]))
    shift = d.nodal_interpolant(lambda x, y, z: s_(y[None, :, None], z[:, None, None]) + 0 * x[None, None, :])
    U[d.off[1]:d.off[2]] += shift[d.off[1]:d.off[2]]
    p = conforming_correction(d, U)
    xp, _ = gll(d.P[0])
    B0, B1 = d.block(p, 0), d.block(p, 1)
    for k in range(d.P[0]):
        for j in range(d.P[0]):
            y, z = (xp[j] + 1) / 2, (xp[k] + 1) / 2
            sv = s_(y, z)
            assert B1[k, j, 0] == pytest.approx(B0[k, j, -1], abs=1e-14)
            for i in range(d.P[0]):
                x = (xp[i] + 1) / 4
                assert B0[k, j, i] == pytest.approx(x * sv + 0.5 * sv * (1 + xp[i]) / 2, abs=1e-14)
            assert B1[k, j, -1] == pytest.approx(0.0, abs=1e-14)


def test_corrected_solution_keeps_the_h1_error():
    errs = {}
    for W in (2, 3):
        pb = wl.poisson_sine(n=2, W=W)
        d = Discretisation(pb)
        x, _, rel = pcg(d.apply_A, lambda r: apply_Cinv(d, r), d.rhs_b(), tol=1e-12, maxit=20000)
        assert rel <= 1e-12
        p = conforming_correction(d, x)
        eu, ep = h1_error_exact(d, x), h1_error_exact(d, p)
        assert ep <= 1.5 * eu, (W, eu, ep)
        errs[W] = ep
    assert errs[3] < 0.2 * errs[2], errs

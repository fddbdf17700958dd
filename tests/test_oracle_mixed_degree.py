"""Pins of the oracle on box meshes whose degree differs across interior faces
(the face terms on the (2 max(W, W') + 1)-point grid of the face).

* Reproduction: u = (1-x^2)(1-y^2)(1-z^2)(1+xy) (degree 3 per variable) is in
  the discrete space of every element of degree >= 3, so the least-squares
  minimiser on a mesh of degrees 3 and 5 is its nodal interpolant.
* The normal operator is the functional's: R(U + tV) - R(U) = 2t <AU - b, V> +
  t^2 <AV, V> for random U, V, and A is symmetric.
* The Laplacian's relative H^1 error on a mesh of degrees 2 and 4 lies between
  the uniform W = 2 and W = 4 errors.
"""
import numpy as np

import workloads as wl
from oracle.functional import Discretisation
from oracle.h1 import h1_error_exact


def _mixed(pb, Ws):
    m = pb.mesh
    m.elem_W = np.asarray(Ws, dtype=np.int32)
    return pb


def test_polynomial_reproduced_on_a_mixed_degree_mesh():
    pb = _mixed(wl.polynomial_exact(n=(2, 1, 1), W=3), [3, 5])
    d = Discretisation(pb)
    U = np.linalg.solve(d.dense_A(), d.rhs_b())
    Ui = d.nodal_interpolant(pb.u_exact[0])
    assert np.abs(U - Ui).max() <= 1e-10 * np.abs(Ui).max()
    assert d.functional(Ui) <= 1e-20


def test_operator_is_the_functional_variation_and_symmetric():
    pb = _mixed(wl.varcoef_manufactured(n=(2, 1, 2), W=2), [2, 4, 3, 2])
    d = Discretisation(pb)
    rng = np.random.default_rng(12)
    U, V = rng.standard_normal(d.ndof), rng.standard_normal(d.ndof)
    b = d.rhs_b()
    AU, AV = d.apply_A(U), d.apply_A(V)
    for t in (0.3, -1.7):
        lhs = d.functional(U + t * V) - d.functional(U)
        rhs = 2 * t * float((AU - b) @ V) + t * t * float(AV @ V)
        assert abs(lhs - rhs) <= 1e-10 * abs(rhs)
    assert abs(float(V @ AU) - float(U @ AV)) <= 1e-12 * abs(float(V @ AU))


def test_mixed_degree_error_between_the_uniform_ones():
    errs = {}
    for name, Ws in (("W2", [2, 2]), ("mixed", [2, 4]), ("W4", [4, 4])):
        pb = _mixed(wl.poisson_sine(n=(2, 1, 1), W=2), Ws)
        d = Discretisation(pb)
        U = np.linalg.solve(d.dense_A(), d.rhs_b())
        errs[name] = h1_error_exact(d, U)
    assert errs["W4"] < errs["mixed"] < errs["W2"], errs

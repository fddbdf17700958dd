"""Pins of the oracle's second-order adjoint quantities (oracle/adjoint.py,
DenseAdjoint): the solution functional J(theta) of the data at the volume
points, its adjoint gradient and Hessian-vector products.

* The dense system at the problem's own data reproduces the Discretisation's
  A and b (by construction of the face parts) and its solution.
* The adjoint gradient agrees with central differences of J (every datum
  kind: f, a, grad a) along a random direction.
* Hessian-vector products: v^T H v equals the second difference of J
  (Richardson-extrapolated), and the Hessian is symmetric, w^T H v =
  v^T H w, for two random directions.
"""
import numpy as np
import pytest

import workloads as wl
from oracle.adjoint import DenseAdjoint, point_data
from oracle.functional import Discretisation


def _target(disc):
    out = []
    for e in range(disc.E):
        x, y, z = wl._grid(*disc.qpoints(e))
        out.append((np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)).ravel())
    return np.concatenate(out)


@pytest.fixture(scope="module")
def setup():
    pb = wl.varcoef_manufactured(n=(2, 1, 1), W=2)
    disc = Discretisation(pb)
    dn = DenseAdjoint(disc, _target(disc))
    theta = point_data(disc)
    rng = np.random.default_rng(6)
    nq = theta[0].size
    v = (rng.standard_normal(nq), 0.1 * rng.standard_normal(nq), 0.1 * rng.standard_normal((3, nq)))
    w = (rng.standard_normal(nq), 0.1 * rng.standard_normal(nq), 0.1 * rng.standard_normal((3, nq)))
    return disc, dn, theta, v, w


def _dot(x, y):
    return sum(float(np.sum(a * b)) for a, b in zip(x, y))


def test_dense_system_reproduces_the_discretisation(setup):
    disc, dn, theta, _, _ = setup
    A, U = dn.solve(*theta)
    assert np.abs(A - disc.dense_A()).max() <= 1e-12 * np.abs(A).max()
    Ud = np.linalg.solve(disc.dense_A(), disc.rhs_b())
    assert np.abs(U - Ud).max() <= 1e-10 * np.abs(Ud).max()


def test_gradient_against_differences_of_J(setup):
    _, dn, theta, v, _ = setup
    g = dn.gradient(*theta)
    h = 1e-5
    Jp = dn.J(*(t + h * d for t, d in zip(theta, v)))
    Jm = dn.J(*(t - h * d for t, d in zip(theta, v)))
    fd = (Jp - Jm) / (2 * h)
    assert abs(_dot(g, v) - fd) <= 1e-6 * abs(fd)


def test_hessian_vector_second_difference_and_symmetry(setup):
    _, dn, theta, v, w = setup
    Hv = dn.hessian_vector(*theta, v, 1e-4)
    Hw = dn.hessian_vector(*theta, w, 1e-4)
    J0 = dn.J(*theta)

    def d2(h):
        Jp = dn.J(*(t + h * d for t, d in zip(theta, v)))
        Jm = dn.J(*(t - h * d for t, d in zip(theta, v)))
        return (Jp - 2 * J0 + Jm) / h ** 2
    # J is not quadratic in a: Richardson's extrapolation of the second
    # difference (truncation O(h^4)); its rounding is that of J (about 1e-13
    # relative, through the dense solves) over h^2, 1e-9 of J at h = 1e-2,
    # i.e. about 1e-7 of v^T H v here: the bound 2e-6
    h = 1e-2
    ref = (4.0 * d2(h / 2) - d2(h)) / 3.0
    assert abs(_dot(v, Hv) - ref) <= 2e-6 * abs(ref)
    assert abs(_dot(w, Hv) - _dot(v, Hw)) <= 1e-7 * max(abs(_dot(w, Hv)), 1e-30)

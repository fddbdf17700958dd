"""Pin of the oracle's adjoint data gradient: central finite differences of J
with respect to single pointwise data values (f_q, a_q, (d_k a)_q), with the
normal equations solved exactly (dense Cholesky) on a tiny mesh.

Finite differences: Richardson extrapolation of central differences with
steps h and h/2, h = 1e-3 (relative), which cancels the O(h^2) truncation term
while keeping the roundoff term O(eps kappa(A) J / h) small (plain central
differences on this mesh: 3e-7 relative at h = 1e-3, 4e-6 at h = 1e-6).
Tolerance: |g - fd| <= 1e-6 max(|fd|, 1e-3 |g|_inf), the gradient field's
sup norm setting the scale for entries near zero."""
import numpy as np
import pytest

import workloads as wl
from oracle.adjoint import data_gradient, l2_misfit, l2_misfit_gradient
from oracle.functional import Discretisation
from oracle.pcg import cholesky_solve


def u_target(xs, ys, zs):
    x, y, z = wl._grid(xs, ys, zs)
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def solve_J(disc):
    A = disc.dense_A()
    U = cholesky_solve(A, disc.rhs_b())
    return A, U, l2_misfit(disc, U, u_target)


@pytest.fixture(scope="module")
def setup():
    pb = wl.varcoef_manufactured(n=(2, 1, 1), W=2)
    disc = Discretisation(pb)
    for e in range(disc.E):  # fill the coefficient cache with writable arrays
        a, g = disc.coef(e)
        disc._coef_cache[e] = (np.array(a), tuple(np.array(c) for c in g))
    A, U, J = solve_J(disc)
    lam = cholesky_solve(A, l2_misfit_gradient(disc, U, u_target))
    grads = data_gradient(disc, U, lam)
    return pb, disc, grads


POINTS = [(0, (1, 2, 3)), (1, (4, 0, 2)), (0, (2, 2, 2))]


@pytest.mark.parametrize("e,idx", POINTS)
@pytest.mark.parametrize("which", ["a", "ax", "ay", "az"])
def test_coefficient_gradient_fd(setup, e, idx, which):
    pb, disc, grads = setup
    a, (ax, ay, az) = disc._coef_cache[e]
    arr = {"a": a, "ax": ax, "ay": ay, "az": az}[which]
    k = {"a": 1, "ax": 2, "ay": 3, "az": 4}[which]
    h = 1e-3 * max(1.0, abs(arr[idx]))
    old = arr[idx]

    def central(step):
        arr[idx] = old + step
        Jp = solve_J(disc)[2]
        arr[idx] = old - step
        Jm = solve_J(disc)[2]
        arr[idx] = old
        return (Jp - Jm) / (2 * step)

    fd = (4 * central(h / 2) - central(h)) / 3
    g = grads[e][k][idx]
    scale = max(abs(fd), 1e-3 * max(np.abs(gr[kk]).max() for gr in grads for kk in range(1, 5)))
    assert abs(g - fd) <= 1e-6 * scale, (which, g, fd)


@pytest.mark.parametrize("e,idx", POINTS)
def test_source_gradient_fd(setup, e, idx):
    pb, disc, grads = setup
    base = disc.f_at
    # J is exactly quadratic in f (U is linear in f): the central difference has
    # no truncation error, so a large step only lowers the roundoff
    h = 0.1 * max(1.0, abs(float(np.asarray(base(e, 0))[idx])))

    def shifted(delta):
        def f_at(ee, rhs):
            v = np.array(base(ee, rhs))
            if ee == e:
                v[idx] += delta
            return v
        return f_at

    def central(step):
        disc.f_at = shifted(+step)
        Jp = solve_J(disc)[2]
        disc.f_at = shifted(-step)
        Jm = solve_J(disc)[2]
        disc.f_at = base
        return (Jp - Jm) / (2 * step)

    fd = (4 * central(h / 2) - central(h)) / 3
    g = grads[e][0][idx]
    scale = max(abs(fd), 1e-3 * max(np.abs(gr[0]).max() for gr in grads))
    assert abs(g - fd) <= 1e-6 * scale, (g, fd)

"""Pins of the oracle's integration-by-parts form of the volume variation
(eq. 5.45-5.48).

* Constant coefficients (the Laplacian of a box element, anisotropic scales;
  a Helmholtz-type operator with first-order and reaction terms): the
  integration-by-parts form equals the direct transpose of the sum
  factorisation, sum_q w_q (L phi_k)(xi_q) z_q written out with the Lagrange
  matrices, for random point values z, W = 2..6 (the two are the same
  integral of polynomials the GLL rule integrates exactly).
* The boundary terms matter: the volume part alone misses by O(1).
* The element's Laplacian transpose of the oracle's Discretisation
  (L_apply_T of a box element) agrees with it.
* Pointwise-sampled variable coefficients (applied to z before the
  interpolation, the (c z)_{xi xi} of eq. 5.46) keep the equality: the
  -div(a grad u) form with a non-polynomial a and first-order terms.
* W = 1: the Laplacian of the trilinear basis vanishes, and so does the
  integration-by-parts form (its volume and face terms cancel).
"""
import numpy as np
import pytest

import workloads as wl
from oracle.functional import Discretisation, eval_tensor_T, tables
from oracle.gll import gll
from oracle.ibp import ibp_transpose


def _direct(W, z, alpha, beta=(0.0, 0.0, 0.0), gamma=0.0):
    B0, B1, B2 = tables(W)["B"]
    Q = 2 * W + 1
    _, wq = gll(Q)
    r = wq[:, None, None] * wq[None, :, None] * wq[None, None, :] * z
    y = gamma * eval_tensor_T(r, B0, B0, B0)
    y = y + alpha[0] * eval_tensor_T(r, B2, B0, B0) + alpha[1] * eval_tensor_T(r, B0, B2, B0) \
        + alpha[2] * eval_tensor_T(r, B0, B0, B2)
    y = y + beta[0] * eval_tensor_T(r, B1, B0, B0) + beta[1] * eval_tensor_T(r, B0, B1, B0) \
        + beta[2] * eval_tensor_T(r, B0, B0, B1)
    return y


def test_w1_laplacian_vanishes():
    z = np.random.default_rng(1).standard_normal((3, 3, 3))
    assert np.abs(ibp_transpose(1, z, (-4.0, -1.0, -16.0))).max() <= 1e-13 * 16 * np.abs(z).max()


@pytest.mark.parametrize("W", [2, 3, 4, 5, 6])
def test_laplacian_ibp_equals_direct_transpose(W):
    Q = 2 * W + 1
    z = np.random.default_rng(W).standard_normal((Q, Q, Q))
    alpha = (-4.0, -1.0, -16.0)   # -s_a^2 of a 1 x 2 x 0.5 box
    got = ibp_transpose(W, z, alpha)
    want = _direct(W, z, alpha)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("W", [2, 5])
def test_first_order_and_reaction_terms(W):
    Q = 2 * W + 1
    z = np.random.default_rng(10 + W).standard_normal((Q, Q, Q))
    args = ((-1.0, -2.5, -0.3), (0.4, -0.7, 1.1), 1.3)
    got = ibp_transpose(W, z, *args)
    want = _direct(W, z, *args)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_boundary_terms_are_needed():
    W, Q = 3, 7
    z = np.random.default_rng(7).standard_normal((Q, Q, Q))
    alpha = (-1.0, -1.0, -1.0)
    want = _direct(W, z, alpha)
    # the volume part alone (no face terms) is far off
    import oracle.ibp as ib
    Z = z
    _, wq = gll(Q)
    from oracle.gll import diff_matrix
    xq, _ = gll(Q)
    DQ = diff_matrix(xq)
    V = sum(alpha[a] * ib._along(DQ, ib._along(DQ, Z, a), a) for a in range(3))
    w3 = wq[:, None, None] * wq[None, :, None] * wq[None, None, :]
    vol_only = eval_tensor_T(w3 * V, *[tables(W)["B"][0]] * 3)
    assert np.abs(vol_only - want).max() > 0.1 * np.abs(want).max()


def test_matches_box_element_transpose_of_the_discretisation():
    pb = wl.poisson_sine(n=(1, 1, 1), W=4)
    pb.mesh.elem_hi[0] = [1.0, 0.5, 2.0]
    d = Discretisation(pb)
    Q = 9
    z = np.random.default_rng(3).standard_normal((Q, Q, Q))
    s = d.scale(0)
    # L = -Lap: L_apply_T(w J z) = sum_q w_q J (L phi)(x_q) z_q
    want = d.L_apply_T(d.vol_weight(0) * z, 0)
    got = d.jac(0) * ibp_transpose(4, z, tuple(-s[a] ** 2 for a in range(3)))
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("W", [3, 6])
def test_pointwise_variable_coefficients_stay_exact(W):
    # -div(a grad u) = -a Lap u - grad a . grad u on a box: alpha_a = -a s_a^2,
    # beta_a = -(d_a a) s_a per point, with a = 1 + 0.5 sin(3x) cos(y) e^{z/2}
    Q = 2 * W + 1
    xq, wq = gll(Q)
    x, y, zc = xq[None, None, :], xq[None, :, None], xq[:, None, None]
    a = 1.0 + 0.5 * np.sin(3 * x) * np.cos(y) * np.exp(zc / 2)
    ax = 1.5 * np.cos(3 * x) * np.cos(y) * np.exp(zc / 2)
    ay = -0.5 * np.sin(3 * x) * np.sin(y) * np.exp(zc / 2)
    az = 0.25 * np.sin(3 * x) * np.cos(y) * np.exp(zc / 2)
    s = (2.0, 1.0, 4.0)
    alpha = tuple(-a * s[k] ** 2 for k in range(3))
    beta = (-ax * s[0], -ay * s[1], -az * s[2])
    z = np.random.default_rng(20 + W).standard_normal((Q, Q, Q))
    B0, B1, B2 = tables(W)["B"]
    r = wq[:, None, None] * wq[None, :, None] * wq[None, None, :] * z
    want = (eval_tensor_T(alpha[0] * r, B2, B0, B0) + eval_tensor_T(alpha[1] * r, B0, B2, B0)
            + eval_tensor_T(alpha[2] * r, B0, B0, B2) + eval_tensor_T(beta[0] * r, B1, B0, B0)
            + eval_tensor_T(beta[1] * r, B0, B1, B0) + eval_tensor_T(beta[2] * r, B0, B0, B1))
    got = ibp_transpose(W, z, alpha, beta)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()

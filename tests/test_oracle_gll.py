"""Pins for the oracle's GLL rules and Lagrange matrices (eq. 5.47, Section 5.3).

Checked against closed forms: the W=2 rule, exact integration of monomials,
and exact differentiation / interpolation of polynomials.
"""
import numpy as np
import pytest

from oracle.gll import diff_matrix, gll, lagrange_eval, legendre


def test_gll_w2_closed_form():
    x, w = gll(3)
    assert np.allclose(x, [-1.0, 0.0, 1.0], atol=1e-15)
    assert np.allclose(w, [1.0 / 3, 4.0 / 3, 1.0 / 3], atol=1e-15)


def test_gll_w3_closed_form():
    # 4-point GLL: nodes +-1, +-1/sqrt(5); weights 1/6, 5/6
    x, w = gll(4)
    s = 1.0 / np.sqrt(5.0)
    assert np.allclose(x, [-1, -s, s, 1], atol=1e-15)
    assert np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)


@pytest.mark.parametrize("n", [2, 3, 5, 9, 13, 17, 21, 25])
def test_gll_exact_monomials(n):
    x, w = gll(n)
    for m in range(0, 2 * n - 2):  # exact up to degree 2n-3
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.dot(w, x ** m) - exact) < 1e-13 * max(1.0, exact)
    # degree 2N = 2n-2 is not exact: the GLL sum of L_N^2 is 2/N, not 2/(2N+1)
    N = n - 1
    assert abs(np.dot(w, legendre(N, x) ** 2) - 2.0 / N) < 1e-12


def test_legendre_recurrence_values():
    t = np.linspace(-1, 1, 7)
    assert np.allclose(legendre(2, t), 0.5 * (3 * t * t - 1))
    assert np.allclose(legendre(3, t), 0.5 * (5 * t ** 3 - 3 * t))
    assert np.allclose(legendre(7, np.array([1.0, -1.0])), [1.0, -1.0])


@pytest.mark.parametrize("W", [1, 2, 4, 8, 10])
def test_lagrange_reproduces_polynomials(W):
    xp, _ = gll(W + 1)
    xq, _ = gll(2 * W + 1)
    rng = np.random.default_rng(W)
    c = rng.standard_normal(W + 1)  # p(x) = sum c_m x^m, degree W
    p = np.polynomial.Polynomial(c)
    B0, B1, B2 = (lagrange_eval(xp, xq, o) for o in range(3))
    assert np.allclose(B0 @ p(xp), p(xq), atol=1e-12)
    assert np.allclose(B1 @ p(xp), p.deriv(1)(xq), atol=1e-10 * W ** 2)
    assert np.allclose(B2 @ p(xp), p.deriv(2)(xq), atol=1e-9 * W ** 4)


@pytest.mark.parametrize("n", [3, 5, 9, 17])
def test_diff_matrix(n):
    x, _ = gll(n)
    D = diff_matrix(x)
    assert np.allclose(D.sum(axis=1), 0.0, atol=1e-11)
    # exact derivative of x^(n-1)
    assert np.allclose(D @ x ** (n - 1), (n - 1) * x ** (n - 2), atol=1e-9)
    # classical corner entry d_00 = -N(N+1)/4
    N = n - 1
    assert abs(D[0, 0] + N * (N + 1) / 4.0) < 1e-10

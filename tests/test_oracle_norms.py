"""Pins for the discrete face norms (eq. 2.17b, 2.18, 5.49).

The discrete H^{1/2} form of Section 5.3 must equal the exact double integral
of eq. (2.17b) for polynomials of degree <= Qf-2 per variable (every product
the Qf-point GLL rule then meets has degree <= 2Qf-3; face traces of degree
W on the 2W+1 grid are in this class).  The exact integral is
computed here independently with high-order Gauss-Legendre quadrature of the
difference quotient polynomial.
"""
import numpy as np
import pytest

from oracle.functional import face_mats, h12_face_literal, half_norm_1d, l2_face_literal
from oracle.gll import gll


def exact_h12_1d_seminorm(p):
    """int int ((p(s) - p(t)) / (s - t))^2 ds dt on (-1,1)^2 for a numpy Polynomial p."""
    # (p(s) - p(t)) / (s - t) = sum_m c_m sum_{a+b=m-1} s^a t^b, a polynomial in (s, t)
    c = p.coef
    xg, wg = np.polynomial.legendre.leggauss(40)
    S, T = np.meshgrid(xg, xg, indexing="ij")
    q = np.zeros_like(S)
    for m in range(1, len(c)):
        for a in range(m):
            q += c[m] * S ** a * T ** (m - 1 - a)
    return float(np.sum(wg[:, None] * wg[None, :] * q * q))


def test_h12_closed_form_quadratic():
    # l(x1, x2) = x1^2: ||l||_0^2 = 4/5; x-part = 2 * int int (s + t)^2 = 16/3; y-part 0
    Qf = 9
    x, _ = gll(Qf)
    v = np.tile(x ** 2, (Qf, 1))  # v[j, i] = x_i^2
    assert abs(h12_face_literal(v, Qf) - (4.0 / 5 + 16.0 / 3)) < 1e-12


@pytest.mark.parametrize("Qf", [5, 9, 17])
def test_h12_exact_for_polynomials(Qf):
    rng = np.random.default_rng(Qf)
    x, w = gll(Qf)
    deg = Qf - 2
    p = np.polynomial.Polynomial(rng.standard_normal(deg + 1))
    q = np.polynomial.Polynomial(rng.standard_normal(deg + 1))
    v = np.outer(q(x), p(x))  # l(x1, x2) = p(x1) q(x2), v[j, i]
    # exact: ||pq||_0^2 + |p|^2 ||q||_0^2 + |q|^2 ||p||_0^2
    xg, wg = np.polynomial.legendre.leggauss(40)
    pp = float(np.sum(wg * p(xg) ** 2))
    qq = float(np.sum(wg * q(xg) ** 2))
    exact = pp * qq + exact_h12_1d_seminorm(p) * qq + exact_h12_1d_seminorm(q) * pp
    got = h12_face_literal(v, Qf)
    assert abs(got - exact) < 1e-11 * exact


@pytest.mark.parametrize("Qf", [3, 7, 11])
def test_matrix_form_matches_literal(Qf):
    rng = np.random.default_rng(100 + Qf)
    W2, H = face_mats(Qf)
    for _ in range(3):
        v = rng.standard_normal((Qf, Qf))
        assert abs(v.ravel() @ H @ v.ravel() - h12_face_literal(v, Qf)) < 1e-11 * h12_face_literal(v, Qf)
        assert abs(v.ravel() @ W2 @ v.ravel() - l2_face_literal(v, Qf)) < 1e-13 * l2_face_literal(v, Qf)


@pytest.mark.parametrize("Qf", [3, 9, 21])
def test_half_norm_matrix_properties(Qf):
    K = half_norm_1d(Qf)
    assert np.allclose(K, K.T, atol=1e-12 * np.abs(K).max())
    ev = np.linalg.eigvalsh(K)
    assert ev.min() > -1e-10 * ev.max()
    # constants have zero H^{1/2} seminorm
    assert np.abs(K @ np.ones(Qf)).max() < 1e-10 * np.abs(K).max()
    W2, H = face_mats(Qf)
    assert np.linalg.eigvalsh(H).min() > 0  # SPD (Section 5.3)

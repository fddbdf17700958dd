"""Separable C-form preconditioner and the H^2 form B (oracle, FP64).

Test infrastructure only (see the package docstring).

Section 5.2.1: on the master cube the preconditioner corresponds to the form
C(u) = int_Q (u_11^2 + u_22^2 + u_33^2 + u_1^2 + u_2^2 + u_3^2 + u^2) (eq. 5.19),
spectrally equivalent to B(u) = ||u||_{H^2(Q)}^2 (eq. 5.7/5.9).  With the 1-D
forms E(v) = int (v'')^2 + (v')^2 and F(v) = int v^2 (eq. 5.11/5.12) and the
generalised eigenpairs (E - mu F) b = 0, b_i^T F b_j = delta_ij (eq. 5.15/5.16),
C is diagonal in the tensor eigenbasis with eigenvalues mu_i + mu_j + mu_k + 1
(eq. 5.20), so C^{-1} r costs O(W^4).

Reading: every 1-D integral is evaluated with the (W+1)-point GLL rule on the
nodal grid (so F = diag(w)); in B each mixed second derivative is counted once.
With exactly these conventions Table 5.1 is reproduced to 1e-12 (tests).
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np
import scipy.linalg as sla

from .gll import diff_matrix, gll


@lru_cache(maxsize=None)
def one_d_forms(W: int):
    """E and F of eq. (5.11)-(5.14) in the nodal GLL basis, (W+1)-point quadrature."""
    x, w = gll(W + 1)
    D1 = diff_matrix(x)
    D2 = D1 @ D1
    Wd = np.diag(w)
    E = D2.T @ Wd @ D2 + D1.T @ Wd @ D1
    F = Wd
    return E, F, D1, D2, Wd


@lru_cache(maxsize=None)
def eigenbasis(W: int):
    """(mu, S): E S = F S diag(mu), S^T F S = I (eq. 5.15/5.16)."""
    E, F, *_ = one_d_forms(W)
    mu, S = sla.eigh(E, F)
    return mu, S


def kron3(a, b, c):
    return np.kron(a, np.kron(b, c))


def dense_C(W: int):
    """C of eq. (5.19) as a (W+1)^3 matrix on u[k,j,i] flattened (x fastest)."""
    E, F, *_ = one_d_forms(W)
    # ordering kron(z-part, y-part, x-part) matches the flattening of u[k, j, i]
    return kron3(F, F, E) + kron3(F, E, F) + kron3(E, F, F) + kron3(F, F, F)


def dense_B(W: int):
    """B = ||u||_{H^2(Q)}^2 (eq. 5.9): all |alpha| <= 2, each multi-index once."""
    _, _, D1, D2, Wd = one_d_forms(W)
    I = np.eye(W + 1)
    ops = {0: I, 1: D1, 2: D2}
    alphas = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0),
              (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
    Wq = kron3(Wd, Wd, Wd)
    B = np.zeros(((W + 1) ** 3,) * 2)
    for ax, ay, az in alphas:
        G = kron3(ops[az], ops[ay], ops[ax])
        B += G.T @ Wq @ G
    return B


def kappa_C_B(W: int) -> float:
    """Condition number of C^{-1} B (the quantity of Table 5.1)."""
    ev = sla.eigh(dense_B(W), dense_C(W), eigvals_only=True)
    return float(ev.max() / ev.min())


def apply_Cinv_block(r, W: int):
    """z = C^{-1} r for one element block r[k, j, i] by fast diagonalisation."""
    mu, S = eigenbasis(W)
    t = np.einsum("kc,jb,ia,kji->cba", S, S, S, r, optimize=True)
    sig = mu[:, None, None] + mu[None, :, None] + mu[None, None, :] + 1.0
    t = t / sig
    return np.einsum("kc,jb,ia,cba->kji", S, S, S, t, optimize=True)


def apply_Cinv(disc, R):
    """Block-diagonal preconditioner on every element of an oracle Discretisation."""
    Z = np.zeros_like(R)
    for e in range(disc.E):
        P = disc.P[e]
        blk = R[disc.off[e]:disc.off[e + 1]].reshape(P, P, P)
        Z[disc.off[e]:disc.off[e + 1]] = apply_Cinv_block(blk, disc.W[e]).ravel()
    return Z


# ---------------------------------------------------------------------------
# Element-block preconditioner (block Jacobi on the element blocks of A).
# Not the thesis's preconditioner; its plain definition is z_e = A_ee^{-1} r_e
# with A_ee the rows and columns of element e of the normal operator of
# eq. (4.2) -- the element's volume term and its own side of every face term.
# ---------------------------------------------------------------------------
def element_block(disc, e):
    """A_ee: column j is (A u)_e for u the j-th unit vector of element e."""
    n = disc.off[e + 1] - disc.off[e]
    B = np.zeros((n, n))
    U = np.zeros(disc.ndof)
    for j in range(n):
        U[disc.off[e] + j] = 1.0
        B[:, j] = np.asarray(disc.element_apply(U, e)).ravel()
        U[disc.off[e] + j] = 0.0
    return B


def block_factors(disc):
    """Cholesky factors of every A_ee (scipy cho_factor)."""
    return [sla.cho_factor(element_block(disc, e), lower=True) for e in range(disc.E)]


def apply_block_inverse(disc, R, factors=None):
    """z_e = A_ee^{-1} r_e on every element."""
    if factors is None:
        factors = block_factors(disc)
    Z = np.zeros_like(R)
    for e in range(disc.E):
        Z[disc.off[e]:disc.off[e + 1]] = sla.cho_solve(factors[e], R[disc.off[e]:disc.off[e + 1]])
    return Z


# ---------------------------------------------------------------------------
# C* form of edge (and vertex-edge) elements, eq. (5.29)-(5.30): with a small
# factor eta in the third variable, C*(u) = int u_xx^2 + u_yy^2 + eta^4 u_zz^2
# + u_x^2 + u_y^2 + eta^2 u_z^2 + u^2, diagonal in the tensor basis of the
# generalised eigenpairs (E - mu F) b = 0 in x, y and (G - nu H) d = 0 in z with
# G(v) = int eta^4 v''^2 + eta^2 v'^2, H(v) = int v^2 (eq. 5.31-5.38); the
# eigenvalues are mu_i + mu_j + nu_k + 1 (eq. 5.42).  1-D integrals with the
# (W+1)-point GLL rule, as for the C-form.
# ---------------------------------------------------------------------------
def one_d_G(W: int, eta: float):
    """G and H of eq. (5.33)-(5.34) in the nodal GLL basis."""
    _, _, D1, D2, Wd = one_d_forms(W)
    return eta ** 4 * D2.T @ Wd @ D2 + eta ** 2 * D1.T @ Wd @ D1, Wd


def cstar_eigen_z(W: int, eta: float):
    G, H = one_d_G(W, eta)
    nu, S = sla.eigh(G, H)
    return np.maximum(nu, 0.0), S


def dense_Cstar(W: int, eta: float):
    """C* of eq. (5.30) on u[k, j, i] flattened (x fastest)."""
    E, F, *_ = one_d_forms(W)
    G, H = one_d_G(W, eta)
    return kron3(H, F, E) + kron3(H, E, F) + kron3(G, F, F) + kron3(H, F, F)


def dense_Bstar(W: int, eta: float):
    """B* of eq. (5.29): second derivatives (the mixed x-y one included, as in
    its transformed form and in B of the edge elements), z-derivatives weighted
    by eta per derivative, first derivatives and u itself."""
    _, _, D1, D2, Wd = one_d_forms(W)
    I = np.eye(W + 1)
    ops = {0: I, 1: D1, 2: D2}
    terms = [((2, 0, 0), 1.0), ((0, 2, 0), 1.0), ((1, 1, 0), 1.0), ((1, 0, 1), eta ** 2), ((0, 1, 1), eta ** 2),
             ((0, 0, 2), eta ** 4), ((1, 0, 0), 1.0), ((0, 1, 0), 1.0), ((0, 0, 1), eta ** 2), ((0, 0, 0), 1.0)]
    Wq = kron3(Wd, Wd, Wd)
    B = np.zeros(((W + 1) ** 3,) * 2)
    for (ax, ay, az), c in terms:
        Gm = kron3(ops[az], ops[ay], ops[ax])
        B += c * Gm.T @ Wq @ Gm
    return B


def apply_Cstar_inv_block(r, W: int, eta: float):
    """z = C*^{-1} r for one block r[k, j, i] by fast diagonalisation."""
    mu, S = eigenbasis(W)
    nu, Sz = cstar_eigen_z(W, eta)
    t = np.einsum("kc,jb,ia,kji->cba", Sz, S, S, r, optimize=True)
    t = t / (nu[:, None, None] + mu[None, :, None] + mu[None, None, :] + 1.0)
    return np.einsum("kc,jb,ia,cba->kji", Sz, S, S, t, optimize=True)
